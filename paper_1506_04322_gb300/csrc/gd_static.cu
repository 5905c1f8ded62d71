// gd_static.cu -- gd_count_global_static: global 3/4-node graphlet counts of
// a small graph without allocating any memory.
//
// Who needs this.  Some callers cannot call cudaMalloc: code that runs while
// a latency-critical pipeline is in flight (cudaMalloc / cudaFree may
// synchronize the device and stall every other stream), plug-ins hosted by a
// framework whose own caching allocator must own every device byte, and
// processes under a hard device-memory quota that was planned before they
// started.  The regular entry points (gd_create_csr + gd_count_global)
// allocate per-graph work arrays; this one allocates nothing.  Its scratch
// is one fixed array in the library's device image: every GPU on which that
// image is loaded holds those bytes until the process exits.  The CUDA
// runtime loads device code lazily by default, so on a device where nothing
// of this file has run yet, the first call's set-up (below) loads it, and
// the runtime reserves the array then; make that first call early, outside
// any latency-critical section.
//
// What it computes: exactly the 15 counts of gd_count_global (same order,
// same exact u128 arithmetic), for graphs within the limits below, in ONE
// kernel launch with one CTA of 1024 threads (32 warps):
//   validate the CSR -> |Tri_e| per slot (Step 1) -> edge sums of
//   Algorithm 2 (Step 3) -> 4-cliques counted once under the degree
//   ordering -> 4-cycles counted once from their highest-ranked node with a
//   per-warp wedge table -> completion (Step 4).
// The scratch holds the per-slot |Tri_e|, the 32 per-warp wedge tables and
// the 32 per-warp candidate lists.  The kernel clears the wedge tables and
// its status word itself at the start of every call.
//
// Sharing and races: every call on a device uses the same scratch array, and
// it keeps the last call's contents.  Two calls whose kernels overlap on the
// GPU (different streams, or different host threads) race on it and give
// wrong results; serialize them (one stream, or events).
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress while that device is current; make that first
// call before any stream capture begins on the device.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/gd.h"

namespace {

constexpr int SW = 32;                       // warps in the CTA
constexpr int32_t MAX_N = GD_STATIC_MAX_N;
constexpr int64_t MAX_NNZ = GD_STATIC_MAX_NNZ;
constexpr int32_t TRICAP = 1024;             // >= sqrt(MAX_NNZ) + 1 (bound on |Tri+|)

constexpr size_t OFF_TSLOT = 0;                                             // u32[MAX_NNZ]
constexpr size_t OFF_TABLE = OFF_TSLOT + sizeof(uint32_t) * MAX_NNZ;       // u32[SW][MAX_N]
constexpr size_t OFF_TRI = OFF_TABLE + sizeof(uint32_t) * SW * MAX_N;      // i32[SW][TRICAP]
constexpr size_t OFF_STATUS = OFF_TRI + sizeof(int32_t) * SW * TRICAP;     // i32[4]
constexpr size_t SCRATCH_BYTES = OFF_STATUS + 256;
static_assert(SCRATCH_BYTES <= GD_STATIC_SCRATCH_BYTES, "scratch layout exceeds the stated size");

// The scratch array (the only device memory this entry point uses).
static __device__ __align__(256) unsigned char gd_static_scratch[GD_STATIC_SCRATCH_BYTES];

enum { ST_BAD_CSR = 1, ST_ARITH = 2, ST_CAP = 4 };

__device__ __forceinline__ bool ranks_below(int32_t da, int32_t a, int32_t db, int32_t b) {
    return da < db || (da == db && a < b);
}

__device__ __forceinline__ int32_t bsearch_pos(const int32_t *a, int32_t len, int32_t key) {
    int32_t lo = 0, hi = len;
    while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return (lo < len && a[lo] == key) ? lo : -1;
}

__device__ __forceinline__ unsigned long long wsum(unsigned long long x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

typedef unsigned __int128 u128;

// sums: 0 T, 1 S, 2 I, 3 C(T,2), 4 SuSv, 5 T(Su+Sv), 6 C(Su,2)+C(Sv,2), 7 T*I,
//       8 (Su+Sv)*I, 9 C(I,2), 10 |E|-du-dv+1, 11 T^2, 12 K4, 13 2*C4
constexpr int NS = 14;

__global__ void __launch_bounds__(SW * 32, 1)
k_static_global(int32_t n, int64_t nnz, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                unsigned char *scratch, unsigned long long *out) {
    uint32_t *tslot = (uint32_t *)(scratch + OFF_TSLOT);
    uint32_t *tables = (uint32_t *)(scratch + OFF_TABLE);
    int32_t *tri = (int32_t *)(scratch + OFF_TRI);
    int32_t *status = (int32_t *)(scratch + OFF_STATUS);
    __shared__ unsigned long long red[NS][SW];
    __shared__ int32_t bad;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // clear what must start at zero: status and the first n entries of every wedge table
    if (threadIdx.x == 0) { bad = 0; status[0] = 0; }
    for (int64_t i = threadIdx.x; i < (int64_t)SW * MAX_N; i += blockDim.x)
        if ((i % MAX_N) < n) tables[i] = 0;
    __syncthreads();

    // validate: row bounds, ascending rows, ids in range, no self-loops, symmetric
    if (threadIdx.x == 0 && (rp[0] != 0 || (int64_t)rp[n] != nnz)) bad = ST_BAD_CSR;
    __syncthreads();
    if (!bad) {
        for (int32_t u = warp; u < n; u += SW) {
            const int32_t b = rp[u], e = rp[u + 1];
            bool ok = (b >= 0 && e >= b && (int64_t)e <= nnz);
            if (ok) {
                for (int32_t p = b + lane; p < e; p += 32) {
                    const int32_t v = ci[p];
                    bool good = v >= 0 && v < n && v != u && (p == b || ci[p - 1] < v);
                    if (good) {
                        const int32_t vb = rp[v], ve = rp[v + 1];
                        good = vb >= 0 && ve >= vb && (int64_t)ve <= nnz && bsearch_pos(ci + vb, ve - vb, u) >= 0;
                    }
                    if (!good) ok = false;
                }
            }
            if (__any_sync(0xffffffffu, !ok) && lane == 0) atomicOr(&bad, ST_BAD_CSR);
        }
    }
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) status[0] = bad;
        return;
    }

    // Step 1: |Tri_e| for every slot
    for (int32_t u = warp; u < n; u += SW) {
        const int32_t bu = rp[u], du = rp[u + 1] - bu;
        for (int32_t p = bu; p < bu + du; p++) {
            const int32_t v = ci[p], bv = rp[v], dv = rp[v + 1] - bv;
            const int32_t *s = du <= dv ? ci + bu : ci + bv;
            const int32_t *l = du <= dv ? ci + bv : ci + bu;
            const int32_t sd = du <= dv ? du : dv, ld = du <= dv ? dv : du;
            unsigned long long c = 0;
            for (int32_t i = lane; i < sd; i += 32) c += bsearch_pos(l, ld, s[i]) >= 0;
            c = wsum(c);
            if (lane == 0) tslot[p] = (uint32_t)c;
        }
    }
    __syncthreads();

    // u64 partials are exact here: n <= MAX_N = 2^15, so every per-edge term
    // is at most n^2 = 2^30, and a sum over the at most 2^17 edges stays
    // below 2^47
    unsigned long long acc[NS];
    for (int i = 0; i < NS; i++) acc[i] = 0;
    const int64_t m = nnz / 2;

    // Step 3: edge sums over each undirected edge once (u < v)
    for (int32_t u = warp; u < n; u += SW) {
        const int32_t bu = rp[u], du = rp[u + 1] - bu;
        for (int32_t p = bu + lane; p < bu + du; p += 32) {
            const int32_t v = ci[p];
            if (v < u) continue;
            const int64_t dv = rp[v + 1] - rp[v];
            const int64_t T = tslot[p], Su = du - 1 - T, Sv = dv - 1 - T;
            const int64_t I = (int64_t)n - du - dv + T;
            acc[0] += T; acc[1] += Su + Sv; acc[2] += I;
            acc[3] += T * (T - 1) / 2;
            acc[4] += Su * Sv;
            acc[5] += T * (Su + Sv);
            acc[6] += Su * (Su - 1) / 2 + Sv * (Sv - 1) / 2;
            acc[7] += T * I;
            acc[8] += (Su + Sv) * I;
            acc[9] += (uint64_t)I * (uint64_t)(I - 1) / 2;
            acc[10] += m - du - dv + 1;
            acc[11] += T * T;
        }
    }

    // 4-cliques, each once: from the edge (a, b) of its two lowest-ranked
    // nodes, pairs of Tri+ = {c in N(a) n N(b) ranked above b} joined by an edge
    int32_t *mytri = tri + warp * TRICAP;
    for (int32_t a = warp; a < n; a += SW) {
        const int32_t ba = rp[a], da = rp[a + 1] - ba;
        for (int32_t p = ba; p < ba + da; p++) {
            const int32_t b = ci[p], bb = rp[b], db = rp[b + 1] - bb;
            if (!ranks_below(da, a, db, b)) continue;
            int32_t cnt = 0;
            for (int32_t i0 = 0; i0 < da; i0 += 32) {
                const int32_t i = i0 + lane;
                bool keep = false;
                int32_t c = 0;
                if (i < da) {
                    c = ci[ba + i];
                    if (bsearch_pos(ci + bb, db, c) >= 0) keep = ranks_below(db, b, rp[c + 1] - rp[c], c);
                }
                const unsigned mask = __ballot_sync(0xffffffffu, keep);
                const int32_t pos = cnt + __popc(mask & ((1u << lane) - 1));
                if (keep) {
                    if (pos < TRICAP) mytri[pos] = c; else atomicOr(status, ST_CAP);
                }
                cnt += __popc(mask);
            }
            __syncwarp();
            if (cnt > TRICAP) cnt = TRICAP;
            for (int32_t i = 0; i + 1 < cnt; i++) {
                const int32_t c = mytri[i], bc = rp[c], dc = rp[c + 1] - bc;
                for (int32_t j = i + 1 + lane; j < cnt; j += 32) acc[12] += bsearch_pos(ci + bc, dc, mytri[j]) >= 0;
            }
            __syncwarp();
        }
    }

    // 4-cycles, each once: from its highest-ranked node u with opposite node
    // y; cnt[y] = number of v below u adjacent to both; sum over wedges of
    // (cnt[y]-1) = 2 * (4-cycles with top node u)
    uint32_t *tab = tables + (int64_t)warp * MAX_N;
    for (int32_t u = warp; u < n; u += SW) {
        const int32_t bu = rp[u], du = rp[u + 1] - bu;
        for (int pass = 0; pass < 3; pass++) {
            for (int32_t i = 0; i < du; i++) {
                const int32_t v = ci[bu + i], bv = rp[v], dv = rp[v + 1] - bv;
                if (!ranks_below(dv, v, du, u)) continue;
                for (int32_t j = lane; j < dv; j += 32) {
                    const int32_t y = ci[bv + j];
                    if (!ranks_below(rp[y + 1] - rp[y], y, du, u)) continue;
                    if (pass == 0) atomicAdd(tab + y, 1u);
                    else if (pass == 1) acc[13] += tab[y] - 1;
                    else tab[y] = 0;
                }
            }
            __syncwarp();
        }
    }

    // block reduction
    for (int i = 0; i < NS; i++) {
        const unsigned long long x = wsum(acc[i]);
        if (lane == 0) red[i][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    u128 s[NS];
    for (int i = 0; i < NS; i++) {
        s[i] = 0;
        for (int w = 0; w < SW; w++) s[i] += red[i][w];
    }
    // Step 4 (Lemmas of Sec. 4.3): sum cliq_e = 6 K4; sum cyc_e = 4 C4 minus
    // the chordal and clique cycles: sum cyc = 4 C4 - 2 sum T^2 + 2 sum T + 2 sum cliq
    int err = status[0];
    const u128 scliq = 6 * s[12];
    const u128 plus = 2 * s[13] + 2 * s[0] + 2 * scliq, minus = 2 * s[11];
    if (minus > plus) err |= ST_ARITH;
    const u128 scyc = plus - minus;
    const u128 N = (u128)n;
    const u128 C3 = N < 3 ? 0 : N * (N - 1) / 2 * (N - 2) / 3;
    const u128 C4 = N < 4 ? 0 : N * (N - 1) / 2 * (N - 2) / 3 * (N - 3) / 4;
    auto dv_ = [&](u128 a, unsigned d) -> u128 { if (a % d) err |= ST_ARITH; return a / d; };
    auto sb_ = [&](u128 a, u128 b) -> u128 { if (b > a) err |= ST_ARITH; return a - b; };
    u128 f[15];
    f[0] = dv_(s[0], 3);
    f[1] = dv_(s[1], 2);
    f[2] = s[2];
    f[3] = sb_(C3, f[0] + f[1] + f[2]);
    const u128 f41 = s[12];
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
    for (int i = 0; i < 15; i++) {
        out[2 * i] = (unsigned long long)f[i];
        out[2 * i + 1] = (unsigned long long)(f[i] >> 64);
    }
    status[0] = err;
}

// per-device address of gd_static_scratch, looked up once with the device current
constexpr int MAX_DEVICES = 64;
unsigned char *g_scratch_addr[MAX_DEVICES] = {nullptr};
std::mutex g_setup_mu;

}  // namespace

extern "C" int gd_count_global_static(int32_t n, int64_t nnz, const int32_t *row_ptr,
                                      const int32_t *col_idx, gd_u128 *out, void *cuda_stream) {
    if (n < 0 || nnz < 0 || (nnz & 1) || !row_ptr || (nnz > 0 && !col_idx) || !out) return GD_EINVAL;
    if (n > MAX_N || nnz > MAX_NNZ) return GD_EOVERFLOW;   // beyond the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return GD_ECUDA;
    unsigned char *scratch;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, gd_static_scratch);
            if (e != cudaSuccess || !p) { cudaGetLastError(); return GD_ECUDA; }
            g_scratch_addr[dev] = (unsigned char *)p;
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    k_static_global<<<1, SW * 32, 0, st>>>(n, nnz, row_ptr, col_idx, scratch, (unsigned long long *)out);
    if (cudaGetLastError() != cudaSuccess) return GD_ECUDA;
    int32_t status = 0;
    if (cudaMemcpyAsync(&status, scratch + OFF_STATUS, sizeof(status), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return GD_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GD_ECUDA;
    if (status & ST_BAD_CSR) return GD_EINVAL;
    if (status) return GD_EARITH;
    return GD_OK;
}
