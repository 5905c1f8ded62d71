// gd_batch.cu -- per-graph global 3/4-node graphlet counts for a batch of
// many small graphs in one persistent launch (the graph-classification
// workloads of Sec. 6: thousands of graphs of tens to hundreds of nodes).
//
// One CTA takes one graph at a time (dynamic work index).  For a graph of
// n <= NMAX nodes it builds the adjacency matrix as n rows of n bits in
// shared memory; then, with codeg(i,j) = popcount(row_i & row_j):
//   Step 1  |Tri_e| = codeg(u,v) for every edge (u,v)
//   Step 2  cliq_e = edges inside Tri_e = (1/2) sum_{c in Tri_e} popc(row_c & Tri_e)
//           4-cycles (not necessarily induced) = (1/2) sum_{u<y} C(codeg(u,y), 2)
//           sum_e cyc_e = 4 C4 - 2 sum T^2 + 2 sum T + 2 sum cliq
//           (sum over edges of: 4-cycles through e minus the chordal/clique
//            cycles through e, i.e. identity D6 summed)
//   Step 3  the unrestricted counts of Algorithm 2 per edge
//   Step 4  the Lemmas of Sec. 4.3 (exact u128), one result row per graph.
// Graphs with more than NMAX nodes are counted by the single-graph path.
#include <cuda_runtime.h>

#include <algorithm>
#include <stdint.h>

#include "gd_device.cuh"
#include "gd_internal.h"

namespace gdi {

namespace {

using namespace gdi::dev;

// per-graph sums: 0 T, 1 S, 2 I, 3 C(T,2), 4 SuSv, 5 T(Su+Sv), 6 C(Su,2)+C(Sv,2),
// 7 T*I, 8 (Su+Sv)*I, 9 C(I,2), 10 |E|-du-dv+1, 11 T^2, 12 cliq, 13 sum_{u<y} C(codeg,2)
constexpr int NB = 14;

enum { BERR_EDGE = 1, BERR_ARITH = 2, BERR_WIDTH = 4 };

template <int NMAX, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)
k_batch_bitmatrix(int32_t num_graphs, const int32_t *__restrict__ gnp, const int32_t *__restrict__ rp,
                  const int32_t *__restrict__ ci, int32_t *work, unsigned long long *out, int32_t *gstatus,
                  int32_t *big_list, int32_t *big_count) {
    constexpr int W = NMAX / 32;
    constexpr int NW = THREADS / 32;
    extern __shared__ __align__(16) uint32_t M[];          // [NMAX][W + 1]: rows at an odd stride
    __shared__ unsigned long long red[NB][NW];
    __shared__ int32_t cur, bad;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) cur = atomicAdd(work, 1);
    __syncthreads();
    while (true) {
        const int32_t gi = cur;
        if (gi >= num_graphs) break;
        const int32_t n0 = gnp[gi], n = gnp[gi + 1] - n0;
        if (n > NMAX) {
            if (threadIdx.x == 0) big_list[atomicAdd(big_count, 1)] = gi;
        } else {
            const int Wn = (n + 31) >> 5;
            // odd row stride: the lanes of a warp read word w of 32 consecutive
            // rows, which then fall in 32 different banks
            const int Sn = Wn | 1;
            const int64_t e0 = rp[n0];
            const int64_t mg = ((int64_t)rp[n0 + n] - e0) / 2;
            for (int k = threadIdx.x; k < n * Sn; k += THREADS) M[k] = 0;
            if (threadIdx.x == 0) bad = 0;
            __syncthreads();
            // rows of bits; every edge must stay inside the graph
            for (int i = warp; i < n; i += NW) {
                const int32_t b = rp[n0 + i], e = rp[n0 + i + 1];
                for (int32_t p = b + lane; p < e; p += WARP) {
                    const int32_t j = ci[p] - n0;
                    if (j < 0 || j >= n || j == i) { atomicOr(&bad, BERR_EDGE); continue; }
                    atomicOr(&M[i * Sn + (j >> 5)], 1u << (j & 31));
                }
            }
            __syncthreads();
            // u64 partials are exact here: a graph has n <= NMAX <= 1024 nodes,
            // so every per-pair term is at most n^2 <= 2^20 and a sum over the
            // C(n,2) < 2^19 pairs stays below 2^39
            unsigned long long acc[NB];
#pragma unroll
            for (int k = 0; k < NB; k++) acc[k] = 0;
            // pairs i < j: codegree; edges get the Step 3 terms and cliq_e
            for (int i = warp; i < n; i += NW) {
                const int64_t di = rp[n0 + i + 1] - rp[n0 + i];
                for (int j = i + 1 + lane; j < n; j += WARP) {
                    uint32_t c = 0;
                    for (int w = 0; w < Wn; w++) c += __popc(M[i * Sn + w] & M[j * Sn + w]);
                    acc[13] += (unsigned long long)c * (c - 1) / 2;
                    if (!((M[i * Sn + (j >> 5)] >> (j & 31)) & 1u)) continue;
                    const int64_t dj = rp[n0 + j + 1] - rp[n0 + j];
                    const int64_t T = c, Su = di - 1 - T, Sv = dj - 1 - T, I = (int64_t)n - di - dj + T;
                    acc[0] += T; acc[1] += Su + Sv; acc[2] += I;
                    acc[3] += T * (T - 1) / 2;
                    acc[4] += Su * Sv;
                    acc[5] += T * (Su + Sv);
                    acc[6] += Su * (Su - 1) / 2 + Sv * (Sv - 1) / 2;
                    acc[7] += T * I;
                    acc[8] += (Su + Sv) * I;
                    acc[9] += (uint64_t)I * (uint64_t)(I - 1) / 2;
                    acc[10] += mg - di - dj + 1;
                    acc[11] += T * T;
                    // cliq_e: ordered adjacent pairs inside Tri_e, halved
                    if (T >= 2) {
                        unsigned long long pairs = 0;
                        for (int w = 0; w < Wn; w++) {
                            uint32_t cw = M[i * Sn + w] & M[j * Sn + w];
                            while (cw) {
                                const int bit = __ffs(cw) - 1;
                                cw &= cw - 1;
                                const int x = w * 32 + bit;
                                for (int w2 = 0; w2 < Wn; w2++)
                                    pairs += __popc(M[x * Sn + w2] & M[i * Sn + w2] & M[j * Sn + w2]);
                            }
                        }
                        acc[12] += pairs >> 1;
                    }
                }
            }
            for (int k = 0; k < NB; k++) {
                const unsigned long long x = warp_sum(acc[k]);
                if (lane == 0) red[k][warp] = x;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                u128 s[NB];
                for (int k = 0; k < NB; k++) {
                    s[k] = 0;
                    for (int w = 0; w < NW; w++) s[k] += red[k][w];
                }
                int err = bad;
                // sum cyc_e from the 4-cycle total (C4 = s13 / 2, sum_e C4(e) = 4 C4)
                const u128 scliq = s[12];
                const u128 plus = 2 * s[13] + 2 * s[0] + 2 * scliq, minus = 2 * s[11];
                if (minus > plus) err |= BERR_ARITH;
                const u128 scyc = plus - minus;
                const u128 N = (u128)n;
                const u128 C3 = N < 3 ? 0 : N * (N - 1) / 2 * (N - 2) / 3;
                const u128 C4 = N < 4 ? 0 : N * (N - 1) / 2 * (N - 2) / 3 * (N - 3) / 4;
                auto dv_ = [&](u128 x, unsigned d) -> u128 { if (x % d) err |= BERR_ARITH; return x / d; };
                auto sb_ = [&](u128 x, u128 y) -> u128 { if (y > x) err |= BERR_ARITH; return x - y; };
                u128 f[15];
                f[0] = dv_(s[0], 3);
                f[1] = dv_(s[1], 2);
                f[2] = s[2];
                f[3] = sb_(C3, f[0] + f[1] + f[2]);
                const u128 f41 = dv_(scliq, 6);
                const u128 f44 = dv_(scyc, 4);
                const u128 f42 = sb_(s[3], 6 * f41);
                const u128 f46 = sb_(s[4], 4 * f44);
                const u128 f43 = dv_(sb_(s[5], 4 * f42), 2);
                const u128 f45 = dv_(sb_(s[6], f43), 3);
                const u128 f47 = dv_(sb_(s[7], f43), 3);
                const u128 f48 = dv_(sb_(s[8], 2 * f46), 2);
                const u128 f49 = dv_(sb_(s[10], 6 * f41 + 4 * f42 + 2 * f43 + 4 * f44 + 2 * f46), 2);
                const u128 f410 = sb_(s[9], 2 * f49);
                const u128 f411 = sb_(C4, f41 + f42 + f43 + f44 + f45 + f46 + f47 + f48 + f49 + f410);
                f[4] = f41; f[5] = f42; f[6] = f43; f[7] = f44; f[8] = f45; f[9] = f46;
                f[10] = f47; f[11] = f48; f[12] = f49; f[13] = f410; f[14] = f411;
                for (int k = 0; k < 15; k++) {
                    if (f[k] >> 64) err |= BERR_WIDTH;
                    out[(int64_t)gi * 15 + k] = (unsigned long long)f[k];
                }
                if (err) atomicOr(gstatus, err);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) cur = atomicAdd(work, 1);
        __syncthreads();
    }
}

// Relabel one graph of the batch to local ids (fallback for large graphs).
__global__ void k_batch_slice(int32_t n0, int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              int32_t *lrp, int32_t *lci) {
    const int32_t e0 = rp[n0];
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x)
        lrp[i] = rp[n0 + i] - e0;
    const int32_t ne = rp[n0 + n] - e0;
    for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < ne; p += gridDim.x * blockDim.x)
        lci[p] = ci[e0 + p] - n0;
}

// Gather graphs held as separate device CSRs into one packed batch: a warp
// per graph copies its row offsets shifted by the graph's slot offset and
// its neighbour ids shifted by its node offset.  Graph i's row_ptr must
// start at 0 and end at its slot count; otherwise bit BERR_EDGE of the
// status is set and the graph's rows are left empty (the packed CSR stays
// well formed and the call is refused afterwards).
__global__ void k_batch_gather(int32_t num_graphs, const int32_t *const *__restrict__ rps,
                               const int32_t *const *__restrict__ cis, const int32_t *__restrict__ gnp,
                               const int32_t *__restrict__ eoff, int32_t *rp_out, int32_t *ci_out,
                               int32_t *gstatus) {
    const int lane = lane_id();
    for (int64_t i = global_warp(); i < num_graphs; i += num_warps()) {
        const int32_t n0 = gnp[i], n = gnp[i + 1] - n0;
        const int32_t e0 = eoff[i], ne = eoff[i + 1] - e0;
        const int32_t *rp = rps[i];
        const int32_t *ci = cis[i];
        const bool ok = n == 0 ? true : (rp[0] == 0 && rp[n] == ne);
        if (!ok) {
            if (lane == 0) atomicOr(gstatus, BERR_EDGE);
            for (int32_t u = lane; u < n; u += WARP) rp_out[n0 + u] = e0;
            for (int32_t p = lane; p < ne; p += WARP) ci_out[e0 + p] = n0;
            continue;
        }
        for (int32_t u = lane; u < n; u += WARP) rp_out[n0 + u] = e0 + rp[u];
        for (int32_t p = lane; p < ne; p += WARP) ci_out[e0 + p] = n0 + ci[p];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rp_out[gnp[num_graphs]] = eoff[num_graphs];
}

}  // namespace

size_t batch_smem_bytes(int nmax) { return (size_t)nmax * (nmax / 32 + 1) * 4; }

template <int NMAX, int THREADS>
static cudaError_t launch_bitmatrix(gd_graph *g, int32_t num_graphs, const int32_t *gnp, const int32_t *rp,
                                    const int32_t *ci, int32_t *work, unsigned long long *out, int32_t *gstatus,
                                    int32_t *big_list, int32_t *big_count) {
    cudaError_t e;
    int per_sm = 0;
    const size_t smem = batch_smem_bytes(NMAX);
    if ((e = cudaFuncSetAttribute(k_batch_bitmatrix<NMAX, THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_bitmatrix<NMAX, THREADS>, THREADS, smem))) return e;
    const int grid = g->ctx->num_sms * (per_sm > 0 ? per_sm : 1);
    GD_LAUNCH(g, "k_batch_bitmatrix", (k_batch_bitmatrix<NMAX, THREADS>), (unsigned)grid, THREADS, smem,
              num_graphs, gnp, rp, ci, work, out, gstatus, big_list, big_count);
    return cudaGetLastError();
}

cudaError_t launch_batch_count(gd_ctx *ctx, cudaStream_t st, int32_t num_graphs, const int32_t *gnp,
                               const int32_t *rp, const int32_t *ci, int32_t *work, unsigned long long *out,
                               int32_t *gstatus, int32_t *big_list, int32_t *big_count, int nmax) {
    gd_graph tmp;     // carrier for the launch macro (context + stream)
    tmp.ctx = ctx;
    tmp.stream = st;
    gd_graph *g = &tmp;
    const int t = ctx->opt.batch_threads;
    if (nmax == 512) {
        if (t > 0 && t <= 192)
            return launch_bitmatrix<512, 128>(g, num_graphs, gnp, rp, ci, work, out, gstatus, big_list, big_count);
        if (t > 384)
            return launch_bitmatrix<512, 512>(g, num_graphs, gnp, rp, ci, work, out, gstatus, big_list, big_count);
        return launch_bitmatrix<512, 256>(g, num_graphs, gnp, rp, ci, work, out, gstatus, big_list, big_count);
    }
    if (t > 0 && t <= 384)
        return launch_bitmatrix<1024, 256>(g, num_graphs, gnp, rp, ci, work, out, gstatus, big_list, big_count);
    if (t > 768)
        return launch_bitmatrix<1024, 1024>(g, num_graphs, gnp, rp, ci, work, out, gstatus, big_list, big_count);
    return launch_bitmatrix<1024, 512>(g, num_graphs, gnp, rp, ci, work, out, gstatus, big_list, big_count);
}

cudaError_t launch_batch_gather(gd_ctx *ctx, cudaStream_t st, int32_t num_graphs, const int32_t *const *rps,
                                const int32_t *const *cis, const int32_t *gnp, const int32_t *eoff,
                                int32_t *rp_out, int32_t *ci_out, int32_t *gstatus) {
    gd_graph tmp;
    tmp.ctx = ctx;
    tmp.stream = st;
    gd_graph *g = &tmp;
    const int64_t warps = std::max<int32_t>(num_graphs, 1);
    const unsigned grid = (unsigned)std::min<int64_t>((warps * 32 + 255) / 256, (int64_t)ctx->num_sms * 8);
    GD_LAUNCH(g, "k_batch_gather", k_batch_gather, grid, 256, 0, num_graphs, rps, cis, gnp, eoff, rp_out, ci_out,
              gstatus);
    return cudaGetLastError();
}

cudaError_t launch_batch_slice(gd_ctx *ctx, cudaStream_t st, int32_t n0, int32_t n, const int32_t *rp,
                               const int32_t *ci, int32_t *lrp, int32_t *lci) {
    gd_graph tmp;
    tmp.ctx = ctx;
    tmp.stream = st;
    gd_graph *g = &tmp;
    GD_LAUNCH(g, "k_batch_slice", k_batch_slice, (unsigned)(ctx->num_sms * 4), 256, 0, n0, n, rp, ci, lrp, lci);
    return cudaGetLastError();
}

}  // namespace gdi
