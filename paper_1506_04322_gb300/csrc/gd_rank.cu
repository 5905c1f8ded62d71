// gd_rank.cu -- ranking and feature vectors built on the exact counts.
//
// Ranking: the k largest entries of a uint64 column (a per-edge graphlet
// column, or per-node sums of one), as used to surface the edges and nodes
// with the most triangles, 4-cliques, stars (the paper's visual analytics of
// top-ranked edges/nodes, Sec. 6 and Fig. 6).  Radix selection over 8-bit
// digits finds the k-th largest value; an order-preserving compaction keeps
// the larger values and the lowest-indexed ties; a bitonic sort orders them
// by (value descending, index ascending), so the answer is unique.
//
// Features: graphlet frequency vectors (Sec. 6, graph classification with
// graphlet features): every count divided by the number of k-subsets,
// C(n, k), as the exact rational rounded once to the nearest double.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "gd_device.cuh"
#include "gd_internal.h"

namespace gdi {

namespace {

using namespace gdi::dev;

int rank_fail(gd_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int rank_cuda(gd_ctx *ctx, cudaError_t e, const char *where) {
    return rank_fail(ctx, GD_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define RK_CK(ctx, call)                                                  \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return rank_cuda((ctx), e_, #call);        \
    } while (0)

// Scratch blocks of one call, returned to the context's cache on exit.
struct Scratch {
    gd_ctx *ctx;
    std::vector<std::pair<void *, size_t>> blocks;
    explicit Scratch(gd_ctx *c) : ctx(c) {}
    ~Scratch() {
        for (auto &b : blocks) scratch_release(ctx, b.first, b.second);
    }
    template <typename T>
    int get(T **p, int64_t count) {
        const size_t bytes = sizeof(T) * (size_t)std::max<int64_t>(count, 1);
        int rc = scratch_alloc(ctx, (void **)p, bytes);
        if (rc == GD_OK) blocks.emplace_back((void *)*p, bytes);
        return rc;
    }
};

__global__ void k_topk_gather(const uint64_t *__restrict__ vals, int64_t count, int64_t stride, uint64_t *keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = vals[i * stride];
}

// histogram of digit (key >> shift) & 255 over the keys whose digits above
// `shift` equal `prefix`
__global__ void k_topk_hist(const uint64_t *__restrict__ keys, int64_t count, int shift, uint64_t prefix,
                            unsigned long long *hist) {
    __shared__ unsigned int h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int hi = shift + 8;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        if (hi < 64 && (k >> hi) != prefix) continue;
        atomicAdd(&h[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(hist + i, (unsigned long long)h[i]);
}

__global__ void k_topk_flags(const uint64_t *__restrict__ keys, int64_t count, uint64_t thr, int64_t *gt,
                             int64_t *eq) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        gt[i] = k > thr;
        eq[i] = k == thr;
    }
}

// the keys > thr, in index order, to (gkey, gidx); the first want_eq keys
// == thr (in index order) to out[ngt ...]
__global__ void k_topk_scatter(const uint64_t *__restrict__ keys, int64_t count, uint64_t thr,
                               const int64_t *__restrict__ pgt, const int64_t *__restrict__ peq, int64_t ngt,
                               int64_t want_eq, uint64_t *gkey, int64_t *gidx, uint64_t *out_key, int64_t *out_idx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        if (k > thr) {
            gkey[pgt[i]] = k;
            gidx[pgt[i]] = i;
        } else if (k == thr && peq[i] < want_eq) {
            out_key[ngt + peq[i]] = k;
            out_idx[ngt + peq[i]] = i;
        }
    }
}

// one compare-exchange stage of a bitonic sort of len (a power of two)
// entries into (key descending, index ascending)
__global__ void k_bitonic(uint64_t *key, int64_t *idx, int64_t len, int64_t size, int64_t stride) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i ^ stride;
        if (j <= i) continue;
        const bool up = (i & size) == 0;
        const uint64_t ki = key[i], kj = key[j];
        const int64_t ii = idx[i], ij = idx[j];
        // "i before j" in the final order
        const bool first = ki > kj || (ki == kj && ii < ij);
        if (first != up) {
            key[i] = kj; key[j] = ki;
            idx[i] = ij; idx[j] = ii;
        }
    }
}

__global__ void k_fill_sentinel(uint64_t *key, int64_t *idx, int64_t from, int64_t to) {
    for (int64_t i = from + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < to; i += (int64_t)gridDim.x * blockDim.x) {
        key[i] = 0;
        idx[i] = INT64_MAX;          // after every real entry
    }
}

__global__ void k_node_sums(int64_t m, const int32_t *__restrict__ eu, const int32_t *__restrict__ ev,
                            const uint64_t *__restrict__ per_edge, int column, unsigned long long *node) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long x = per_edge[e * 15 + column];
        if (x == 0) continue;
        atomicAdd(node + eu[e], x);
        atomicAdd(node + ev[e], x);
    }
}

unsigned grid_of(int64_t items, int sms) {
    const int64_t b = (items + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sms * 16));
}

}  // namespace

// ---------------------------------------------------------------------------
// exact u128 / u128 -> nearest double (ties to even), 0 <= a <= b
// ---------------------------------------------------------------------------

__host__ __device__ inline bool u128_lt(uint64_t ahi, uint64_t alo, uint64_t bhi, uint64_t blo) {
    return ahi < bhi || (ahi == bhi && alo < blo);
}

// The rational a / b rounded once: restoring long division yields the
// leading 1, 52 fraction bits and one rounding bit; the remainder is the
// sticky bit.
__host__ __device__ inline double ratio_nearest(uint64_t ahi, uint64_t alo, uint64_t bhi, uint64_t blo) {
    if ((ahi | alo) == 0 || (bhi | blo) == 0) return 0.0;
    // r = a; scale r by 2 until b <= r (a / b = r / b * 2^-e)
    uint64_t rhi = ahi, rlo = alo;
    int e = 0;
    while (u128_lt(rhi, rlo, bhi, blo)) {
        rhi = (rhi << 1) | (rlo >> 63);
        rlo <<= 1;
        e++;
    }
    // when a > b (not used by the callers) r / b may exceed 2: shift b up
    int bshift = 0;
    uint64_t bh = bhi, bl = blo;
    while (!u128_lt(rhi, rlo, (bh << 1) | (bl >> 63), bl << 1) && bh < (1ull << 62)) {
        bh = (bh << 1) | (bl >> 63);
        bl <<= 1;
        bshift++;
    }
    uint64_t mant = 0;
    for (int i = 0; i < 54; i++) {
        mant <<= 1;
        if (!u128_lt(rhi, rlo, bh, bl)) {
            const uint64_t lo = rlo - bl;
            rhi = rhi - bh - (rlo < bl ? 1 : 0);
            rlo = lo;
            mant |= 1;
        }
        rhi = (rhi << 1) | (rlo >> 63);
        rlo <<= 1;
    }
    const bool sticky = (rhi | rlo) != 0;
    uint64_t m53 = mant >> 1;
    const bool round_bit = mant & 1;
    if (round_bit && (sticky || (m53 & 1))) m53++;
    int exp2 = bshift - e - 52;
    if (m53 == (1ull << 53)) { m53 >>= 1; exp2++; }
    return ldexp((double)m53, exp2);
}

// C(n, k) as u128 (k <= 4)
__host__ __device__ inline void choose_u128(int64_t n, int k, uint64_t *hi, uint64_t *lo) {
    if (n < k) { *hi = 0; *lo = 0; return; }
    unsigned __int128 c = 1;
    for (int i = 0; i < k; i++) c = c * (unsigned __int128)(n - i) / (unsigned __int128)(i + 1);
    *hi = (uint64_t)(c >> 64);
    *lo = (uint64_t)c;
}

__host__ __device__ inline void gfd_one(int64_t n, int64_t m, const uint64_t *chi, const uint64_t *clo, double *out) {
    uint64_t h2, l2, h3, l3, h4, l4;
    choose_u128(n, 2, &h2, &l2);
    choose_u128(n, 3, &h3, &l3);
    choose_u128(n, 4, &h4, &l4);
    const unsigned __int128 c2 = ((unsigned __int128)h2 << 64) | l2;
    const unsigned __int128 non = c2 - (unsigned __int128)m;
    out[0] = ratio_nearest(0, (uint64_t)m, h2, l2);
    out[1] = ratio_nearest((uint64_t)(non >> 64), (uint64_t)non, h2, l2);
    for (int i = 0; i < 4; i++) out[2 + i] = ratio_nearest(chi[i], clo[i], h3, l3);
    for (int i = 4; i < 15; i++) out[2 + i] = ratio_nearest(chi[i], clo[i], h4, l4);
}

__global__ void k_gfd_batch(int32_t G, const int32_t *__restrict__ node_ptr, const int32_t *__restrict__ row_ptr,
                            const uint64_t *__restrict__ counts, double *out) {
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const int64_t n = node_ptr[g + 1] - node_ptr[g];
        const int64_t m = ((int64_t)row_ptr[node_ptr[g + 1]] - row_ptr[node_ptr[g]]) / 2;
        uint64_t hi[15], lo[15];
        for (int i = 0; i < 15; i++) { hi[i] = 0; lo[i] = counts[(int64_t)g * 15 + i]; }
        gfd_one(n, m, hi, lo, out + (int64_t)g * 17);
    }
}

}  // namespace gdi

using namespace gdi;

extern "C" {

int gd_topk(gd_ctx *ctx, const uint64_t *values, int64_t count, int64_t stride, int flags, int64_t k,
            int64_t *idx_out, uint64_t *val_out, void *cuda_stream) {
    if (!ctx) return GD_EINVAL;
    if (count < 0 || stride < 1 || k < 0 || k > count || (k > 0 && (!values || !idx_out)))
        return rank_fail(ctx, GD_EINVAL, "gd_topk: bad arguments");
    if (k == 0) return GD_OK;
    RK_CK(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    gd_graph tmp;                      // launch bookkeeping only
    tmp.ctx = ctx;
    tmp.stream = st;
    const int sms = ctx->num_sms > 0 ? ctx->num_sms : 152;
    Scratch sc(ctx);
    int rc;
    uint64_t *keys = nullptr;
    const uint64_t *src = values;
    if (!(flags & GD_DEVICE_PTRS)) {
        uint64_t *dv = nullptr;
        const int64_t span = (count - 1) * stride + 1;
        if ((rc = sc.get(&dv, span))) return rc;
        RK_CK(ctx, cudaMemcpyAsync(dv, values, sizeof(uint64_t) * (size_t)span, cudaMemcpyHostToDevice, st));
        src = dv;
    }
    if ((rc = sc.get(&keys, count))) return rc;
    GD_LAUNCH(&tmp, "k_topk_gather", k_topk_gather, grid_of(count, sms), 256, 0, src, count, stride, keys);
    // radix selection of the k-th largest key
    unsigned long long *hist = nullptr;
    if ((rc = sc.get(&hist, 256))) return rc;
    uint64_t prefix = 0;
    int64_t want = k;
    for (int shift = 56; shift >= 0; shift -= 8) {
        RK_CK(ctx, cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned long long), st));
        GD_LAUNCH(&tmp, "k_topk_hist", k_topk_hist, grid_of(count, sms), 256, 0, keys, count, shift, prefix, hist);
        unsigned long long h[256];
        RK_CK(ctx, cudaMemcpyAsync(h, hist, sizeof(h), cudaMemcpyDeviceToHost, st));
        RK_CK(ctx, cudaStreamSynchronize(st));
        int d = 255;
        for (; d > 0; d--) {
            if ((int64_t)h[d] >= want) break;
            want -= (int64_t)h[d];
        }
        prefix = (prefix << 8) | (uint64_t)d;
    }
    const uint64_t thr = prefix;       // the k-th largest; `want` of the entries equal to it are taken
    const int64_t ngt = k - want;
    int64_t *gt = nullptr, *eq = nullptr, *pgt = nullptr, *peq = nullptr, *tmpscan = nullptr;
    const int64_t tmp_len = 2 * ((count + 1023) / 1024) + 4096;
    if ((rc = sc.get(&gt, count)) || (rc = sc.get(&eq, count)) || (rc = sc.get(&pgt, count + 1)) ||
        (rc = sc.get(&peq, count + 1)) || (rc = sc.get(&tmpscan, tmp_len)))
        return rc;
    GD_LAUNCH(&tmp, "k_topk_flags", k_topk_flags, grid_of(count, sms), 256, 0, keys, count, thr, gt, eq);
    RK_CK(ctx, exclusive_scan_i64(&tmp, gt, pgt, count, tmpscan));
    RK_CK(ctx, exclusive_scan_i64(&tmp, eq, peq, count, tmpscan));
    int64_t l2 = 1;
    while (l2 < ngt) l2 <<= 1;
    uint64_t *okey = nullptr, *gkey = nullptr;
    int64_t *oidx = nullptr, *gidx = nullptr;
    if ((rc = sc.get(&okey, k)) || (rc = sc.get(&oidx, k)) || (rc = sc.get(&gkey, l2)) || (rc = sc.get(&gidx, l2)))
        return rc;
    GD_LAUNCH(&tmp, "k_topk_scatter", k_topk_scatter, grid_of(count, sms), 256, 0, keys, count, thr, pgt, peq, ngt,
              want, gkey, gidx, okey, oidx);
    // the entries above the threshold need ordering; the ties follow in index order
    if (ngt > 1) {
        if (l2 > ngt)
            GD_LAUNCH(&tmp, "k_fill_sentinel", k_fill_sentinel, grid_of(l2 - ngt, sms), 256, 0, gkey, gidx, ngt, l2);
        for (int64_t size = 2; size <= l2; size <<= 1)
            for (int64_t stride2 = size >> 1; stride2 > 0; stride2 >>= 1)
                GD_LAUNCH(&tmp, "k_bitonic", k_bitonic, grid_of(l2, sms), 256, 0, gkey, gidx, l2, size, stride2);
    }
    if (ngt > 0) {
        RK_CK(ctx, cudaMemcpyAsync(okey, gkey, sizeof(uint64_t) * (size_t)ngt, cudaMemcpyDeviceToDevice, st));
        RK_CK(ctx, cudaMemcpyAsync(oidx, gidx, sizeof(int64_t) * (size_t)ngt, cudaMemcpyDeviceToDevice, st));
    }
    RK_CK(ctx, cudaMemcpyAsync(idx_out, oidx, sizeof(int64_t) * (size_t)k, cudaMemcpyDeviceToHost, st));
    if (val_out) RK_CK(ctx, cudaMemcpyAsync(val_out, okey, sizeof(uint64_t) * (size_t)k, cudaMemcpyDeviceToHost, st));
    RK_CK(ctx, cudaStreamSynchronize(st));
    return GD_OK;
}

int gd_node_sums(gd_graph *g, const uint64_t *per_edge, int flags, int column, uint64_t *node_out, int out_flags) {
    if (!g) return GD_EINVAL;
    gd_ctx *ctx = g->ctx;
    if (!per_edge || !node_out || column < 0 || column >= 15)
        return rank_fail(ctx, GD_EINVAL, "gd_node_sums: bad arguments");
    RK_CK(ctx, cudaSetDevice(ctx->device));
    if (!g->prepared || !g->ws.eu)
        return rank_fail(ctx, GD_EINVAL, "count the graph first (its edge list gives the rows)");
    const int sms = ctx->num_sms > 0 ? ctx->num_sms : 152;
    Scratch sc(ctx);
    int rc;
    const uint64_t *pe = per_edge;
    if (!(flags & GD_DEVICE_PTRS)) {
        uint64_t *d = nullptr;
        if ((rc = sc.get(&d, 15 * g->m))) return rc;
        RK_CK(ctx, cudaMemcpyAsync(d, per_edge, sizeof(uint64_t) * 15 * (size_t)g->m, cudaMemcpyHostToDevice, g->stream));
        pe = d;
    }
    unsigned long long *node = nullptr;
    if (out_flags & GD_OUT_DEVICE) node = (unsigned long long *)node_out;
    else if ((rc = sc.get(&node, g->n))) return rc;
    RK_CK(ctx, cudaMemsetAsync(node, 0, sizeof(uint64_t) * (size_t)std::max<int32_t>(g->n, 0), g->stream));
    if (g->m > 0)
        GD_LAUNCH(g, "k_node_sums", k_node_sums, grid_of(g->m, sms), 256, 0, g->m, g->ws.eu, g->ws.ev, pe, column, node);
    if (!(out_flags & GD_OUT_DEVICE))
        RK_CK(ctx, cudaMemcpyAsync(node_out, node, sizeof(uint64_t) * (size_t)g->n, cudaMemcpyDeviceToHost, g->stream));
    RK_CK(ctx, cudaStreamSynchronize(g->stream));
    return GD_OK;
}

int gd_gfd(int64_t n, int64_t m, const gd_u128 counts[15], double out[17]) {
    if (!counts || !out || n < 0 || m < 0 || (n >= 2 && m > n * (n - 1) / 2)) return GD_EINVAL;
    uint64_t hi[15], lo[15];
    for (int i = 0; i < 15; i++) { hi[i] = counts[i].hi; lo[i] = counts[i].lo; }
    gfd_one(n, m, hi, lo, out);
    return GD_OK;
}

int gd_gfd_batch(gd_ctx *ctx, int32_t num_graphs, const int32_t *graph_node_ptr, const int32_t *row_ptr,
                 const uint64_t *counts, int flags, double *out, void *cuda_stream) {
    if (!ctx) return GD_EINVAL;
    if (num_graphs < 0 || (num_graphs > 0 && (!graph_node_ptr || !row_ptr || !counts || !out)))
        return rank_fail(ctx, GD_EINVAL, "gd_gfd_batch: bad arguments");
    if (num_graphs == 0) return GD_OK;
    if (!(flags & GD_DEVICE_PTRS)) return rank_fail(ctx, GD_EINVAL, "gd_gfd_batch: device pointers expected");
    RK_CK(ctx, cudaSetDevice(ctx->device));
    gd_graph tmp;
    tmp.ctx = ctx;
    tmp.stream = (cudaStream_t)cuda_stream;
    const int sms = ctx->num_sms > 0 ? ctx->num_sms : 152;
    GD_LAUNCH(&tmp, "k_gfd_batch", k_gfd_batch, grid_of(num_graphs, sms), 256, 0, num_graphs, graph_node_ptr, row_ptr,
              counts, out);
    RK_CK(ctx, cudaGetLastError());
    RK_CK(ctx, cudaStreamSynchronize(tmp.stream));
    return GD_OK;
}

}  // extern "C"
