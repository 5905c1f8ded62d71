// gd_count.cu -- single-graph kernels of the edge-centric graphlet method.
//
// Steps (Ahmed et al. 2015, Sec. 3-4, Algorithm 2):
//   Step 1  per edge e=(u,v): |Tri_e| = |N(u) n N(v)|, |Star_u|, |Star_v|
//   Step 2  per edge: cliq_e (edges inside Tri_e, Cor. 1) and cyc_e (edges
//           between Star_u and Star_v, Cor. 3)
//   Step 3  per edge: the unrestricted counts of Sec. 4.2 (Eqs. for
//           N_{a,a} = C(|W|,2) and N_{a,b} = |W_a||R_b|)
//   Step 4  sums over edges and the Lemmas of Sec. 4.3 (completion kernel)
//
// GPU form.  Neighbour lists are sorted int32 CSR rows.  Each undirected edge
// is one work item (canonical slot: row u, col v > u).  Intersections are done
// by a warp: lanes take the elements of the shorter list and binary-search the
// longer one, so the work per edge is min(du,dv) * log(max).  Step 2 is done
// either literally (GD_VARIANT_LITERAL: scan the lists of Tri_e / Star_u as
// CliqueCount / CycleCount do) or by enumerating every 4-clique and 4-cycle
// once under the degree ordering (a precedes b iff (d_a, a) < (d_b, b)) and
// crediting the edges it contains; the per-edge cyc_e then follows from the
// number of 4-cycles through e minus the chordal/clique cycles (identity
// stated at run_final).  All counts are exact integers.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gd_device.cuh"
#include "gd_internal.h"

namespace gdi {

namespace {

using namespace gdi::dev;

// ---------------------------------------------------------------------------
// CSR validation: sorted rows, ids in range, no self-loops, symmetric.
// ---------------------------------------------------------------------------
// CSR check: row bounds (a thread per row), then the entries, every warp
// taking an equal range of them (hub rows of tens of thousands of entries
// would otherwise hold one warp for milliseconds): ids in [0, n), strictly
// ascending rows (no duplicates), no self-loops, and for every entry above
// the diagonal (u < v) its reverse u in N(v).  A warp finds the row of its
// first entry by binary search over row_ptr and walks forward; every index
// stays in bounds even when row_ptr is invalid (the row pass reports that).
// status[2] / status[3] receive the numbers of entries above / below the
// diagonal: every upper entry having its reverse and the two numbers being
// equal makes the CSR symmetric (the reverse map of the distinct upper
// entries is injective into the lower ones).
__global__ void __launch_bounds__(256) k_validate(int32_t n, int64_t nnz, const int32_t *__restrict__ rp,
                                                  const int32_t *__restrict__ ci, int32_t *status) {
    const int lane = lane_id();
    int32_t up_all = 0, lo_all = 0;
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int32_t b = rp[u], e = rp[u + 1];
        if (b < 0 || e < b || (int64_t)e > nnz) { atomicOr(status, ERR_CSR); atomicMin(status + 1, u); }
    }
    const int64_t W = num_warps(), w = global_warp();
    const int64_t p0 = nnz * w / W, p1 = nnz * (w + 1) / W;
    if (n > 0 && p0 < p1) {
        // the last row r with rp[r] <= p0
        int32_t r = 0, hi = n - 1;
        while (r < hi) {
            const int32_t mid = (r + hi + 1) >> 1;
            if ((int64_t)rp[mid] <= p0) r = mid; else hi = mid - 1;
        }
        for (int64_t q0 = p0; q0 < p1; q0 += WARP) {
            const int64_t p = q0 + lane;
            int32_t u = r;
            bool bad = false;
            if (p < p1) {
                while (u < n - 1 && (int64_t)rp[u + 1] <= p) u++;
                const int32_t v = ci[p];
                const int64_t b = rp[u];
                bad = v < 0 || v >= n || v == u || (p > 0 && p > b && v <= ci[p - 1]);
                if (!bad && v > u) {
                    up_all++;
                    const int32_t vb = rp[v], ve = rp[v + 1];
                    bad = vb < 0 || ve < vb || (int64_t)ve > nnz;
                    if (!bad) bad = find_in(ci + vb, ve - vb, u) < 0;
                } else if (!bad) {
                    lo_all++;
                }
            }
            if (bad) { atomicOr(status, ERR_CSR); atomicMin(status + 1, u); }
            r = __reduce_max_sync(0xffffffffu, (unsigned)u);
        }
    }
    // one pair of atomics per CTA
    __shared__ int32_t su, sl;
    if (threadIdx.x == 0) { su = 0; sl = 0; }
    __syncthreads();
    up_all = warp_sum(up_all);
    lo_all = warp_sum(lo_all);
    if (lane == 0) { atomicAdd(&su, up_all); atomicAdd(&sl, lo_all); }
    __syncthreads();
    if (threadIdx.x == 0) { atomicAdd(status + 2, su); atomicAdd(status + 3, sl); }
}

// ---------------------------------------------------------------------------
// Edge list: canonical slots (u, v) with u < v, in CSR order.
// ---------------------------------------------------------------------------
__global__ void k_upper_count(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              int32_t *first_up, int64_t *cnt) {
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        int32_t b = rp[u], e = rp[u + 1];
        int32_t f = b + lower_bound(ci + b, e - b, u + 1);
        first_up[u] = f;
        cnt[u] = e - f;
    }
}

// exclusive scan helpers (int64), three-phase
constexpr int SCAN_T = 256;
constexpr int SCAN_PER = 8;
constexpr int SCAN_TILE = SCAN_T * SCAN_PER;

__global__ void k_scan_tiles(const int64_t *in, int64_t *out, int64_t len, int64_t *tile_sums) {
    __shared__ int64_t sh[SCAN_T];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_PER;
    int64_t v[SCAN_PER];
    int64_t s = 0;
    for (int i = 0; i < SCAN_PER; i++) {
        int64_t x = (base + i < len) ? in[base + i] : 0;
        v[i] = s; s += x;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < SCAN_T; o <<= 1) {
        int64_t t = (threadIdx.x >= o) ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    int64_t off = sh[threadIdx.x] - s;
    for (int i = 0; i < SCAN_PER; i++)
        if (base + i < len) out[base + i] = v[i] + off;
    if (threadIdx.x == SCAN_T - 1) tile_sums[blockIdx.x] = sh[SCAN_T - 1];
}

__global__ void k_scan_add(int64_t *out, int64_t len, const int64_t *tile_offs) {
    int64_t i = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x;
    int64_t add = tile_offs[blockIdx.x];
    for (int k = 0; k < SCAN_PER; k++, i += SCAN_T)
        if (i < len) out[i] += add;
}

// exclusive scan of len values; out[len] receives the total.  tmp needs
// >= 2 * ceil(len / SCAN_TILE) + 64 entries per level.
cudaError_t exclusive_scan(gd_graph *g, const int64_t *in, int64_t *out, int64_t len, int64_t *tmp) {
    cudaStream_t st = g->stream;
    int64_t tiles = (len + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 0) {
        return cudaMemsetAsync(out, 0, sizeof(int64_t), st);
    }
    int64_t *sums = tmp, *offs = tmp + tiles;
    GD_LAUNCH(g, "k_scan_tiles", k_scan_tiles, (unsigned)tiles, SCAN_T, 0, in, out, len, sums);
    if (tiles > 1) {
        cudaError_t e = exclusive_scan(g, sums, offs, tiles, tmp + 2 * tiles + 1);
        if (e != cudaSuccess) return e;
        GD_LAUNCH(g, "k_scan_add", k_scan_add, (unsigned)tiles, SCAN_T, 0, out, len, offs);
        // total = offs[tiles]
        return cudaMemcpyAsync(out + len, offs + tiles, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    }
    return cudaMemcpyAsync(out + len, sums, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
}

__global__ void k_narrow(const int64_t *in, int32_t *out, int64_t len) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)in[i];
}

__global__ void k_edge_list(int32_t n, int64_t nnz, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const int32_t *__restrict__ first_up, const int32_t *__restrict__ eoff,
                            int32_t *eu, int32_t *ev, int32_t *eslot) {
    // every warp an equal range of the slots (a warp per row would leave one
    // warp with each hub row); slot p of row u above the diagonal is edge
    // eoff[u] + p - first_up[u].  The row of the range's first slot comes from
    // a binary search over row_ptr, the next ones from walking forward.
    const int lane = lane_id();
    const int64_t W = num_warps(), w = global_warp();
    const int64_t p0 = nnz * w / W, p1 = nnz * (w + 1) / W;
    if (n == 0 || p0 >= p1) return;
    int32_t r = 0, hi = n - 1;
    while (r < hi) {
        const int32_t mid = (r + hi + 1) >> 1;
        if ((int64_t)rp[mid] <= p0) r = mid; else hi = mid - 1;
    }
    for (int64_t q0 = p0; q0 < p1; q0 += WARP) {
        const int64_t p = q0 + lane;
        int32_t u = r;
        if (p < p1) {
            while (u < n - 1 && (int64_t)rp[u + 1] <= p) u++;
            const int32_t f = first_up[u];
            if (p >= f) {
                const int32_t k = eoff[u] + (int32_t)(p - f);
                eu[k] = u; ev[k] = ci[p]; eslot[k] = (int32_t)p;
            }
        }
        r = __reduce_max_sync(0xffffffffu, (unsigned)u);
    }
}

__global__ void k_mate(int64_t m, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                       const int32_t *__restrict__ eu, const int32_t *__restrict__ ev,
                       const int32_t *__restrict__ eslot, int32_t *mate) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = eu[k], v = ev[k], p = eslot[k];
        int32_t q = rp[v] + lower_bound(ci + rp[v], rp[v + 1] - rp[v], u);
        mate[p] = q;
        mate[q] = p;
    }
}

// ---------------------------------------------------------------------------
// Step 1: |Tri_e| per edge (Alg. 2 marking loops; Eq. triangle)
// ---------------------------------------------------------------------------
__global__ void k_triangles(int64_t m, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const int32_t *__restrict__ eu, const int32_t *__restrict__ ev,
                            const int32_t *__restrict__ eslot, const int32_t *__restrict__ mate,
                            uint32_t *tslot) {
    const int lane = lane_id();
    for (int64_t k = global_warp(); k < m; k += num_warps()) {
        int32_t u = eu[k], v = ev[k];
        int32_t bu = rp[u], du = rp[u + 1] - bu, bv = rp[v], dv = rp[v + 1] - bv;
        int32_t sb = bu, sd = du, lb = bv, ld = dv;
        if (dv < du) { sb = bv; sd = dv; lb = bu; ld = du; }
        uint32_t c = 0;
        for (int32_t i = lane; i < sd; i += WARP) {
            int32_t x = ldg(ci + sb + i);
            c += find_in(ci + lb, ld, x) >= 0;
        }
        c = warp_sum(c);
        if (lane == 0) {
            int32_t p = eslot[k];
            tslot[p] = c;
            tslot[mate[p]] = c;
        }
    }
}

// ---------------------------------------------------------------------------
// Node quantities: t(x) = edges inside N(x) = sum_y T(x,y)/2; S1(x) = sum d_y
// ---------------------------------------------------------------------------
// nd (nullable): degree of each slot's neighbour, read in order instead of
// through row_ptr when the schedule has built it.
__global__ void k_node(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                       const int32_t *__restrict__ nd, const uint32_t *__restrict__ tslot, uint64_t *tnode,
                       uint64_t *s1) {
    const int lane = lane_id();
    for (int32_t x = global_warp(); x < n; x += num_warps()) {
        uint64_t a = 0, b = 0;
        for (int32_t p = rp[x] + lane; p < rp[x + 1]; p += WARP) {
            a += tslot[p];
            if (nd) {
                b += (uint64_t)nd[p];
            } else {
                const int32_t y = ci[p];
                b += (uint64_t)(rp[y + 1] - rp[y]);
            }
        }
        a = warp_sum(a); b = warp_sum(b);
        if (lane == 0) { tnode[x] = a >> 1; s1[x] = b; }
    }
}

// Per edge: A_u + A_v = sum_{w in Tri} (T(u,w) + T(v,w)) and
// D_T = sum_{w in Tri} d_w (the per-edge identities need only the sum).
__global__ void k_tri_sums(int64_t m, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const int32_t *__restrict__ eu, const int32_t *__restrict__ ev,
                           const uint32_t *__restrict__ tslot, uint64_t *au, uint64_t *dt) {
    const int lane = lane_id();
    for (int64_t k = global_warp(); k < m; k += num_warps()) {
        int32_t u = eu[k], v = ev[k];
        int32_t bu = rp[u], du = rp[u + 1] - bu, bv = rp[v], dv = rp[v + 1] - bv;
        bool su = du <= dv;   // shorter list is u's
        int32_t sb = su ? bu : bv, sd = su ? du : dv, lb = su ? bv : bu, ld = su ? dv : du;
        uint64_t a_s = 0, a_l = 0, d = 0;
        for (int32_t i = lane; i < sd; i += WARP) {
            int32_t x = ldg(ci + sb + i);
            int32_t j = find_in(ci + lb, ld, x);
            if (j >= 0) {
                a_s += tslot[sb + i];
                a_l += tslot[lb + j];
                d += (uint64_t)(rp[x + 1] - rp[x]);
            }
        }
        a_s = warp_sum(a_s); a_l = warp_sum(a_l); d = warp_sum(d);
        if (lane == 0) {
            au[k] = a_s + a_l;      // A_u + A_v
            dt[k] = d;
        }
    }
}

// ---------------------------------------------------------------------------
// Step 2, literal (Algorithm 2 CliqueCount / CycleCount), warp per edge.
// cliq_e: for w in Tri_e, r in N(w): r in Tri_e (each internal edge seen
// twice; the paper's X(w)=0 reset halves it the same way).
// cyc_e: for w in Star_u, r in N(w): r in Star_v.
// ---------------------------------------------------------------------------
__global__ void k_literal(int64_t m, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                          const int32_t *__restrict__ eu, const int32_t *__restrict__ ev,
                          const int32_t *__restrict__ eslot,
                          int32_t *tribuf, int32_t tricap, unsigned long long *cacc,
                          unsigned long long *yacc, int32_t *status) {
    const int lane = lane_id();
    const int gw = global_warp();
    int32_t *buf = tribuf + (int64_t)gw * tricap * 3;
    for (int64_t k = gw; k < m; k += num_warps()) {
        int32_t u = eu[k], v = ev[k], p = eslot[k];
        int32_t bu = rp[u], du = rp[u + 1] - bu, bv = rp[v], dv = rp[v + 1] - bv;
        // Tri_e in ascending order (scan N(u), test membership in N(v))
        int32_t cnt = 0;
        for (int32_t i0 = 0; i0 < du; i0 += WARP) {
            int32_t i = i0 + lane;
            bool keep = false;
            int32_t x = 0;
            if (i < du) { x = ldg(ci + bu + i); keep = find_in(ci + bv, dv, x) >= 0; }
            unsigned mask = __ballot_sync(0xffffffffu, keep);
            int32_t pos = cnt + __popc(mask & ((1u << lane) - 1));
            if (keep) {
                if (pos < tricap) buf[pos] = x; else atomicOr(status, ERR_CAPACITY);
            }
            cnt += __popc(mask);
        }
        __syncwarp();
        if (cnt > tricap) cnt = tricap;
        // CliqueCount
        unsigned long long cl = 0;
        for (int32_t i = 0; i < cnt; i++) {
            int32_t w = buf[i];
            int32_t bw = rp[w], dw = rp[w + 1] - bw;
            for (int32_t j = lane; j < dw; j += WARP) cl += find_in(buf, cnt, ldg(ci + bw + j)) >= 0;
        }
        cl = warp_sum(cl);
        // CycleCount over Star_u = N(u) \ {v} \ N(v)
        unsigned long long cy = 0;
        for (int32_t i = 0; i < du; i++) {
            int32_t w = ldg(ci + bu + i);
            if (w == v || find_in(ci + bv, dv, w) >= 0) continue;
            int32_t bw = rp[w], dw = rp[w + 1] - bw;
            for (int32_t j = lane; j < dw; j += WARP) {
                int32_t r = ldg(ci + bw + j);
                // r in Star_v: r in N(v), r != u, r not in N(u)
                if (r != u && find_in(ci + bv, dv, r) >= 0 && find_in(ci + bu, du, r) < 0) cy++;
            }
        }
        cy = warp_sum(cy);
        if (lane == 0) { cacc[p] = cl >> 1; yacc[p] = cy; }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Steps 3-4 per edge: restricted counts from the identities, per-edge
// columns (Corollaries 1-14) and the 13 sums of Algorithm 2.
//
// With s = T + cliq etc. (all per edge e = (u,v)):
//   N_TSu1 = A_u - T - 2cliq                 (edges Tri-Star_u)
//   N_SuSu1 = t(u) - T - cliq - N_TSu1       (edges inside Star_u)
//   N_TI1  = D_T - 2T - 2cliq - N_TS1
//   cyc    = C4(e) - N_TS1 - 2cliq           (oriented variant)
//   N_SuI1 = (S1(u) - d_v - D_T - Su) - N_TSu1 - 2N_SuSu1 - cyc
//   N_II1  = |E| - (du-1) - (dv-1) - 1 - (all edges touching the egonet)
// ---------------------------------------------------------------------------
struct FinalArgs {
    const int32_t *nd;        // degree of each slot's neighbour (null: from row_ptr)
    int64_t m;
    int32_t n;
    int variant;              // 1 literal, 2 oriented
    int per_edge;             // write columns
    int need_restricted;      // per-edge restricted counts available
    int cliq_credits;         // cliq_e from the per-slot credits (else summed by the clique kernel)
    const int32_t *rp, *eu, *ev, *eslot, *mate;
    const uint32_t *tslot;
    const uint64_t *tnode, *s1, *au, *dt;        // au: A_u + A_v per edge
    const unsigned long long *qcred;             // per slot: triangle-perimeter credit, then degree-sum credit
    int qr_credits;                              // A_u + A_v and D_T from the credits
    const unsigned long long *cacc, *yacc;
    const uint32_t *y32;                         // oriented credits as 32-bit words, when so kept
    uint64_t *out;
    unsigned long long *sums;
    int32_t *status;
};

constexpr int FINAL_THREADS = 256;

// Every per-edge term below is at most n^2 < 2^62 (T, Su + Sv and I are
// parts of one partition of the n nodes), but their sums are not: C(I,2)
// alone sums to about m n^2 / 2, past 2^64 for a sparse graph of 2^28 nodes
// and 10^6 edges.  So every partial -- per thread, per warp, per CTA -- is
// kept in 128 bits and reaches the global words as one 128-bit addend.
__global__ void __launch_bounds__(FINAL_THREADS) k_final(FinalArgs a) {
    __shared__ u128 red[S_NUM + X_NUM][FINAL_THREADS / 32];
    u128 loc[S_NUM + X_NUM];
    for (int i = 0; i < S_NUM + X_NUM; i++) loc[i] = 0;
    // adds a per-edge term (non-negative for a consistent input; a negative
    // one raises ERR_NEGATIVE below, so its value here does not matter)
    auto acc = [&](int i, int64_t x) { loc[i] += (u128)(uint64_t)x; };
    int bad = 0;
    const int64_t nn = a.n, mm = a.m;
    // per-edge rows go through shared memory so that a tile of blockDim
    // consecutive edges is written with coalesced stores (a row is 120 bytes)
    __shared__ uint64_t stage[FINAL_THREADS * 15];
    for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x; k0 < a.m; k0 += (int64_t)gridDim.x * blockDim.x) {
      const int64_t k = k0 + threadIdx.x;
      if (k < a.m) {
        const int32_t u = a.eu[k], v = a.ev[k], p = a.eslot[k];
        const int64_t du = a.rp[u + 1] - a.rp[u], dv = a.nd ? a.nd[p] : a.rp[v + 1] - a.rp[v];
        const int64_t T = a.tslot[p];
        const int64_t Su = du - 1 - T, Sv = dv - 1 - T;
        const int64_t I = nn - du - dv + T;
        const int64_t II = mm - du - dv + 1;      // |E| - (du-1) - (dv-1) - 1
        acc(S_T, T); acc(S_S, Su + Sv); acc(S_I, I);
        acc(S_TT, T * (T - 1) / 2);
        acc(S_SUSV, Su * Sv);
        acc(S_TS, T * (Su + Sv));
        acc(S_SS, Su * (Su - 1) / 2 + Sv * (Sv - 1) / 2);
        acc(S_TI, T * I);
        acc(S_SI, (Su + Sv) * I);
        acc(S_II, (int64_t)((uint64_t)I * (uint64_t)(I - 1) / 2));
        acc(S_II1, II);
        acc(X_T2 + S_NUM, T * T);
        int64_t cliq = 0, cyc = 0, c4 = 0;
        if (a.variant == GD_VARIANT_LITERAL) {
            cliq = (int64_t)a.cacc[p];
            cyc = (int64_t)a.yacc[p];
            acc(S_CLIQ, cliq);
        } else if (a.cliq_credits) {
            const int32_t q = a.mate[p];
            cliq = (int64_t)(a.cacc[p] + a.cacc[q]);
            acc(S_CLIQ, cliq);
        }
        if (!a.need_restricted) {
            acc(S_CYC, cyc);
            continue;
        }
        if (a.variant != GD_VARIANT_LITERAL) {
            const int32_t q = a.mate[p];
            c4 = a.y32 ? (int64_t)a.y32[p] + a.y32[q] : (int64_t)(a.yacc[p] + a.yacc[q]);
        }
        // A = A_u + A_v and D_T, then the restricted counts summed over both
        // endpoints (the columns need only these sums):
        //   N_TS1 = A - 2T - 4cliq, N_SS1 = t(u)+t(v) - 2T - 2cliq - N_TS1,
        //   N_TI1 = D_T - 2T - 2cliq - N_TS1, cyc = C4(e) - N_TS1 - 2cliq,
        //   N_SI1 = S1(u)+S1(v) - du - dv - 2D_T - Su - Sv - N_TS1 - 2N_SS1 - 2cyc
        int64_t A, DT;
        if (a.qr_credits) {
            const int32_t q = a.mate[p];
            A = (int64_t)(a.qcred[2 * (int64_t)p] + a.qcred[2 * (int64_t)q]) - T * T;
            DT = (int64_t)(a.qcred[2 * (int64_t)p + 1] + a.qcred[2 * (int64_t)q + 1]) - T * (du + dv);
        } else {
            A = (int64_t)a.au[k];
            DT = (int64_t)a.dt[k];
        }
        const int64_t ts = A - 2 * T - 4 * cliq;
        if (a.variant != GD_VARIANT_LITERAL) cyc = c4 - ts - 2 * cliq;
        acc(S_CYC, cyc);
        const int64_t ss = (int64_t)a.tnode[u] + (int64_t)a.tnode[v] - 2 * T - 2 * cliq - ts;
        const int64_t ti = DT - 2 * T - 2 * cliq - ts;
        const int64_t si = ((int64_t)a.s1[u] + (int64_t)a.s1[v] - du - dv - 2 * DT - Su - Sv) - ts - 2 * ss - 2 * cyc;
        const int64_t ii1 = II - (cliq + ts + ti + ss + cyc + si);
        if ((Su | Sv | I | A | DT | ts | ss | ti | cyc | si | ii1 | cliq) < 0) bad = 1;
        if (a.per_edge) {
            uint64_t *o = stage + threadIdx.x * 15;
            o[0] = T;
            o[1] = Su + Sv;
            o[2] = I;
            o[3] = 0;
            o[4] = cliq;
            o[5] = T * (T - 1) / 2 - cliq + ts;
            o[6] = T * (Su + Sv) - ts + ti + ss;
            o[7] = cyc;
            o[8] = Su * (Su - 1) / 2 + Sv * (Sv - 1) / 2 - ss;
            o[9] = Su * Sv - cyc + si;
            o[10] = T * I - ti;
            o[11] = (Su + Sv) * I - si;
            o[12] = ii1;
            o[13] = (uint64_t)I * (uint64_t)(I - 1) / 2 - (uint64_t)ii1;
            o[14] = 0;
        }
      }
      if (a.per_edge) {
        __syncthreads();
        const int64_t rows = min((int64_t)blockDim.x, a.m - k0);
        uint64_t *o = a.out + k0 * 15;
        for (int64_t i = threadIdx.x; i < rows * 15; i += blockDim.x) o[i] = stage[i];
        __syncthreads();
      }
    }
    if (bad) atomicOr(a.status, ERR_NEGATIVE);
    // block reduction in 128 bits -> one 128-bit addend per sum and CTA
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    for (int i = 0; i < S_NUM + X_NUM; i++) {
        const u128 x = warp_sum_u128(loc[i]);
        if (lane == 0) red[i][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < S_NUM + X_NUM) {
        u128 s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[threadIdx.x][w];
        add_u128_wide(a.sums + 2 * threadIdx.x, s);
    }
}

// ---------------------------------------------------------------------------
// Step 4: completion (one thread), exact u128.
// ---------------------------------------------------------------------------

__device__ __forceinline__ u128 ld128(const unsigned long long *p) {
    return (u128)p[0] | ((u128)p[1] << 64);
}
__device__ __forceinline__ void st128(unsigned long long *p, u128 x) {
    p[0] = (unsigned long long)x; p[1] = (unsigned long long)(x >> 64);
}

__global__ void k_complete(const unsigned long long *sums, int64_t n, int derive_cyc,
                           unsigned long long *result, int32_t *status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    u128 s[S_NUM + X_NUM];
    for (int i = 0; i < S_NUM + X_NUM; i++) s[i] = ld128(sums + 2 * i);
    int err = 0;
    // sum cyc_e from 4-cycle credits when per-edge restricted counts were
    // not formed: sum_e N_TS1 = 2 sum T^2 - 2 sum T - 4 sum cliq, so
    // sum cyc = sum C4(e) - sum N_TS1 - 2 sum cliq.
    u128 scyc = s[S_CYC];
    if (derive_cyc) {
        u128 plus = s[S_NUM + X_C4] + 2 * s[S_T] + 2 * s[S_CLIQ];
        u128 minus = 2 * s[S_NUM + X_T2];
        if (minus > plus) err |= ERR_NEGATIVE;
        scyc = plus - minus;
    }
    const u128 N = (u128)n;
    const u128 C3 = N < 3 ? 0 : N * (N - 1) / 2 * (N - 2) / 3;
    const u128 C4 = N < 4 ? 0 : N * (N - 1) / 2 * (N - 2) / 3 * (N - 3) / 4;
    u128 f[15];
    auto exdiv = [&](u128 a, unsigned d) -> u128 { if (a % d) err |= ERR_REMAINDER; return a / d; };
    auto sub = [&](u128 a, u128 b) -> u128 { if (b > a) err |= ERR_NEGATIVE; return a - b; };
    f[0] = exdiv(s[S_T], 3);                        // Eq. triangle
    f[1] = exdiv(s[S_S], 2);                        // Eq. 2-star
    f[2] = s[S_I];                                  // Eq. g3_3
    f[3] = sub(C3, f[0] + f[1] + f[2]);             // Eq. g3_4
    const u128 f41 = exdiv(s[S_CLIQ], 6);           // Lemma 1 (each 4-clique on 6 edges)
    const u128 f44 = exdiv(scyc, 4);                // Lemma 2 (each 4-cycle on 4 edges)
    const u128 f42 = sub(s[S_TT], 6 * f41);         // Lemma 1
    const u128 f46 = sub(s[S_SUSV], 4 * f44);       // Lemma 2
    const u128 f43 = exdiv(sub(s[S_TS], 4 * f42), 2);       // Lemma 3
    const u128 f45 = exdiv(sub(s[S_SS], f43), 3);           // Lemma 4
    const u128 f47 = exdiv(sub(s[S_TI], f43), 3);           // Lemma 5
    const u128 f48 = exdiv(sub(s[S_SI], 2 * f46), 2);       // Lemma 6
    const u128 f49 = exdiv(sub(s[S_II1], 6 * f41 + 4 * f42 + 2 * f43 + 4 * f44 + 2 * f46), 2);  // Eq. g4_9
    const u128 f410 = sub(s[S_II], 2 * f49);                 // Lemma 7
    const u128 f411 = sub(C4, f41 + f42 + f43 + f44 + f45 + f46 + f47 + f48 + f49 + f410);  // Eq. g4_11
    f[4] = f41; f[5] = f42; f[6] = f43; f[7] = f44; f[8] = f45; f[9] = f46;
    f[10] = f47; f[11] = f48; f[12] = f49; f[13] = f410; f[14] = f411;
    for (int i = 0; i < 15; i++) st128(result + 2 * i, f[i]);
    if (err) atomicOr(status, err);
}

inline unsigned grid_for(int64_t items, int per_block, int max_blocks) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (unsigned)b;
}

}  // namespace

// ===========================================================================
// host launchers (all asynchronous on the graph's stream)
// ===========================================================================

cudaError_t exclusive_scan_i64(gd_graph *g, const int64_t *in, int64_t *out, int64_t len, int64_t *tmp) {
    return exclusive_scan(g, in, out, len, tmp);
}

static int sm_count(gd_graph *g) { return g->ctx->num_sms > 0 ? g->ctx->num_sms : 152; }

__global__ void k_max_degree(int32_t n, const int32_t *__restrict__ rp, int32_t *out) {
    int32_t best = 0;
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
        best = max(best, rp[u + 1] - rp[u]);
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

cudaError_t max_degree(gd_graph *g, int32_t *out_host) {
    Workspace &w = g->ws;
    cudaStream_t st = g->stream;
    cudaError_t e = cudaMemsetAsync(w.status + 3, 0, sizeof(int32_t), st);
    if (e) return e;
    if (g->n > 0) GD_LAUNCH(g, "k_max_degree", k_max_degree, grid_for(g->n, 256, sm_count(g) * 8), 256, 0, g->n, g->rp, w.status + 3);
    e = cudaMemcpyAsync(out_host, w.status + 3, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e) return e;
    e = cudaStreamSynchronize(st);
    if (e) return e;
    return cudaMemsetAsync(w.status + 3, 0, sizeof(int32_t), st);
}

cudaError_t launch_validate(gd_graph *g, int32_t *status) {
    if (g->n > 0) GD_LAUNCH(g, "k_validate", k_validate, (unsigned)(sm_count(g) * 8), 256, 0, g->n, g->nnz, g->rp, g->ci, status);
    return cudaGetLastError();
}

cudaError_t validate_csr(gd_graph *g, int32_t *bad_index, int32_t *bad_code) {
    Workspace &w = g->ws;
    cudaStream_t st = g->stream;
    int32_t init[4] = {0, 0x7fffffff, 0, 0};
    cudaError_t e = cudaMemcpyAsync(w.status, init, sizeof(init), cudaMemcpyHostToDevice, st);
    if (e) return e;
    if (g->n > 0) GD_LAUNCH(g, "k_validate", k_validate, (unsigned)(sm_count(g) * 8), 256, 0, g->n, g->nnz, g->rp, g->ci, w.status);
    int32_t h[4];
    e = cudaMemcpyAsync(h, w.status, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e) return e;
    e = cudaStreamSynchronize(st);
    if (e) return e;
    *bad_code = h[0];
    *bad_index = h[1];
    if (!h[0] && h[2] != h[3]) {   // every upper entry has its reverse, so some lower entry has none
        *bad_code = ERR_CSR;
        *bad_index = -1;
    }
    return cudaMemsetAsync(w.status, 0, 4 * sizeof(int32_t), st);
}

// Step 1 and the schedule: edge list, reverse slots, |Tri_e| per slot, wedge
// tiers.  Everything is recomputed from the CSR on every count call.
cudaError_t prepare_edges(gd_graph *g) {
    Workspace &w = g->ws;
    cudaStream_t st = g->stream;
    const int sms = sm_count(g);
    const int32_t n = g->n;
    cudaError_t e = cudaMemsetAsync(w.status, 0, 4 * sizeof(int32_t), st);
    if (e) return e;
    e = cudaMemsetAsync(w.sums, 0, sizeof(unsigned long long) * 2 * (S_NUM + X_NUM), st);
    if (e) return e;
    if (n == 0) return cudaSuccess;
    int64_t *cnt = w.scan_tmp;
    int64_t *offs = w.scan_tmp + (n + 1);
    int64_t *tmp = w.scan_tmp + 2 * (int64_t)(n + 1);
    GD_LAUNCH(g, "k_upper_count", k_upper_count, grid_for(n, 256, sms * 8), 256, 0, n, g->rp, g->ci, w.first_up, cnt);
    e = exclusive_scan(g, cnt, offs, n, tmp);
    if (e) return e;
    GD_LAUNCH(g, "k_narrow", k_narrow, grid_for(n + 1, 256, sms * 8), 256, 0, offs, w.eoff, n + 1);
    GD_LAUNCH(g, "k_edge_list", k_edge_list, (unsigned)(sms * 8), 256, 0, n, g->nnz, g->rp, g->ci, w.first_up, w.eoff,
                                                                         w.eu, w.ev, w.eslot);
    if (g->m > 0)
        GD_LAUNCH(g, "k_mate", k_mate, grid_for(g->m, 256, sms * 8), 256, 0, g->m, g->rp, g->ci, w.eu, w.ev, w.eslot, w.mate);
    return cudaGetLastError();
}

// Step 1 by per-edge intersection (literal variant and out-degree fallback)
cudaError_t run_triangles_intersect(gd_graph *g) {
    Workspace &w = g->ws;
    const int sms = sm_count(g);
    if (g->m > 0)
        GD_LAUNCH(g, "k_triangles", k_triangles, grid_for(g->m * 32, 256, sms * 16), 256, 0, g->m, g->rp, g->ci,
                  w.eu, w.ev, w.eslot, w.mate, w.tslot);
    return cudaGetLastError();
}

cudaError_t run_node_sums(gd_graph *g, bool have_nd) {
    Workspace &w = g->ws;
    const int sms = sm_count(g);
    if (g->n > 0)
        GD_LAUNCH(g, "k_node", k_node, grid_for((int64_t)g->n * 32, 256, sms * 16), 256, 0, g->n, g->rp, g->ci,
                  have_nd ? w.nd : nullptr, w.tslot, w.tnode, w.s1);
    return cudaGetLastError();
}

cudaError_t run_per_edge_sums(gd_graph *g) {
    Workspace &w = g->ws;
    const int sms = sm_count(g);
    cudaError_t e = run_node_sums(g, false);
    if (e) return e;
    if (g->m > 0)
        GD_LAUNCH(g, "k_tri_sums", k_tri_sums, grid_for(g->m * 32, 256, sms * 16), 256, 0, g->m, g->rp, g->ci, w.eu, w.ev, w.tslot,
                                                                       w.au, w.dt);
    return cudaGetLastError();
}

static const int TRI_THREADS = 256;
int32_t tribuf_warps(int sms) { return sms * 8 * (TRI_THREADS / 32); }

// Literal Step 2 (Algorithm 2's CliqueCount and CycleCount per edge).
cudaError_t run_literal(gd_graph *g) {
    Workspace &w = g->ws;
    const int sms = sm_count(g);
    if (g->m == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(w.cacc, 0, sizeof(uint64_t) * g->nnz, g->stream);
    if (e) return e;
    e = cudaMemsetAsync(w.yacc, 0, sizeof(uint64_t) * g->nnz, g->stream);
    if (e) return e;
    const int32_t warps = tribuf_warps(sms);
    const int32_t tricap = (int32_t)(w.tribuf_words / ((int64_t)warps * 3));
    const unsigned tri_blocks = (unsigned)(warps / (TRI_THREADS / 32));
    GD_LAUNCH(g, "k_literal", k_literal, tri_blocks, TRI_THREADS, 0, g->m, g->rp, g->ci, w.eu, w.ev, w.eslot,
              w.tribuf, tricap, (unsigned long long *)w.cacc, (unsigned long long *)w.yacc, w.status);
    return cudaGetLastError();
}

cudaError_t run_final(gd_graph *g, int variant, bool per_edge, bool cliq_credits, bool qr_credits,
                      uint64_t *out_dev) {
    Workspace &w = g->ws;
    const int sms = sm_count(g);
    if (g->m == 0) return cudaSuccess;
    FinalArgs a;
    a.m = g->m; a.n = g->n; a.variant = variant; a.per_edge = per_edge ? 1 : 0;
    a.need_restricted = per_edge ? 1 : 0;
    a.cliq_credits = cliq_credits ? 1 : 0;
    a.rp = g->rp; a.eu = w.eu; a.ev = w.ev; a.eslot = w.eslot; a.mate = w.mate; a.tslot = w.tslot;
    a.nd = variant == GD_VARIANT_LITERAL ? nullptr : w.nd;
    a.tnode = w.tnode; a.s1 = w.s1; a.au = w.au; a.dt = w.dt;
    a.qcred = (const unsigned long long *)w.qcred;
    a.qr_credits = qr_credits ? 1 : 0;
    a.cacc = (const unsigned long long *)w.cacc; a.yacc = (const unsigned long long *)w.yacc;
    a.y32 = variant != GD_VARIANT_LITERAL && w.yacc32 ? reinterpret_cast<const uint32_t *>(w.yacc) : nullptr;
    a.out = out_dev; a.sums = w.sums; a.status = w.status;
    GD_LAUNCH(g, "k_final", k_final, grid_for(g->m, 256, sms * 8), 256, 0, a);
    return cudaGetLastError();
}

// derive_cyc: sum cyc_e is derived from the 4-cycle credits (oriented
// variant without per-edge restricted counts).
cudaError_t run_complete(gd_graph *g, int derive_cyc) {
    GD_LAUNCH(g, "k_complete", k_complete, 1, 32, 0, g->ws.sums, g->n, derive_cyc, g->ws.result, g->ws.status);
    return cudaGetLastError();
}

}  // namespace gdi
