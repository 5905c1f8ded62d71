// gd_step2.cu -- Step 2 of Algorithm 2 (4-cliques and 4-cycles through each
// edge) and |Tri_e| per edge, organised around the degree ordering
// a precedes b  <=>  (d_a, a) < (d_b, b).
//
// Schedule (per count call, from the CSR):
//   nd[p]     degree of the neighbour in slot p (rank tests read it coalesced)
//   N+(a)     out-list of a: neighbours ranked above a, ascending ids, with the
//             CSR slot of each (a, c) edge.  Under the degree ordering every
//             out-list has at most sqrt(2|E|) entries.
//   tiers     vertices by wedge work W(u) = sum_{v in N(u), v below u} d_v.
//
// Triangles and 4-cliques ("bitmap" kernels).  For every node a, a team (a
// warp for |N+(a)| <= 64, a CTA of 256 threads up to 256, of 1024 threads up
// to 1024 -- its 128 KB bit matrix allows one CTA per SM, so all 32 warps of
// that CTA share the node --, a CTA on global scratch above)
// walks the pairs (c, x) with c in N+(a) and x in N+(c), the concatenated
// out-lists spread evenly over the team's warps; a shared-memory filter and
// hash table of N+(a) decide membership, candidates queued 32 at a time.  A
// pair whose x is in N+(a) too is the triangle {a, c, x} with a lowest,
// found exactly once, and the scan holds the CSR slots of all three edges:
//   triangle {a,c,x}:  (c,x) += 1 directly, (a,c) and (a,x) through per-c
//                      counters flushed once per node
// The same scan sets the adjacency matrix M of the subgraph induced by
// N+(a) (shared memory, one bit per pair) and records the triangle.  For an
// edge (c, x) inside N+(a), the common neighbours of c and x in M are the
// 4-cliques {a, c, x, d} with a lowest; a pass over the records credits them:
//   4-clique {a,c,x,d}: (c,x) += |M[c] & M[x]| once per inner edge,
//                       (a,c) += half the sum over the inner edges at c
// Per-edge |Tri_e| and cliq_e are the sums of the credits of both slots of
// the edge.  For the global count only sum |M[c] & M[x]| = 3 K4 is kept.
// The triangle-sum pass walks the kept records and credits each triangle's
// perimeter and degree sum to its three edges.
//
// 4-cycles.  Every 4-cycle is counted once from its highest-ranked node u
// with opposite node y: cnt[y] = number of v below u adjacent to u and y
// (wedges u-v-y with v, y below u).  Then
//   global:   4-cycles with top u = sum_y C(cnt[y], 2)
//   per edge: each wedge carries cnt[y]-1 cycles, credited to (u,v), (v,y).
// A vertex's wedges are split evenly over the warps working on it (a prefix
// of the wedge counts over N(u)); a warp walks its range 32 neighbours at a
// time, their lists spread over the lanes.  Tables by W(u):
//   tiny   : warp-private shared-memory hash (W <= 256)
//   small  : shared-memory hash per CTA (W <= half its capacity)
//   medium : one CTA per vertex, open-addressing table in global memory
//            sized to the vertex (the tables of all CTAs fit L2 together)
//   hubs   : W > max(2^k, n/8): a batch of hubs at a time, every warp of the
//            GPU taking an equal share of the batch's wedges, dense tables of
//            n counters (a few at a time, so they stay in L2).
#include <cuda_runtime.h>
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>
#include <stdint.h>

#include "gd_device.cuh"
#include "gd_internal.h"

namespace gdi {

namespace {

using namespace gdi::dev;
constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// schedule
// ---------------------------------------------------------------------------

__global__ void k_neighbor_degree(int64_t nnz, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                  int32_t *nd) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = ci[p];
        nd[p] = rp[v + 1] - rp[v];
    }
}

// Per vertex: wedge work, out-degree, tiers.  counters:
//  [C_SMALL] [C_MEDIUM] [C_MAXDP] [C_HUB] [C_CL0..C_CL3] clique buckets
// A CTA takes tiles of 256 vertices (a warp per vertex, 32 vertices per
// warp); list positions are claimed in shared memory and each list's range
// for the tile with one global atomic, so the few list counters are not
// hammered by one atomic per vertex.
constexpr int SCHED_TILE = 256;

__global__ void __launch_bounds__(256)
k_schedule(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
           const int32_t *__restrict__ nd, int64_t small_cap, int64_t hub_min, int32_t cl_max,
           int32_t *vlist, int32_t *hubs, int32_t *clist, int32_t *counters, int64_t *dplus,
           int64_t *west, int32_t *tlist) {
    // lists: 0 tiny, 1 small, 2 medium, 3 hub, 4..7 clique buckets
    __shared__ int32_t cnt[8], base[8];
    __shared__ int32_t tile_maxdp;
    __shared__ unsigned long long tile_maxw;
    __shared__ int8_t code_l[SCHED_TILE], code_b[SCHED_TILE];
    __shared__ int32_t pos_l[SCHED_TILE], pos_b[SCHED_TILE];
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    for (int64_t t0 = (int64_t)blockIdx.x * SCHED_TILE; t0 < n; t0 += (int64_t)gridDim.x * SCHED_TILE) {
        if (threadIdx.x < 8) cnt[threadIdx.x] = 0;
        if (threadIdx.x == 0) { tile_maxdp = 0; tile_maxw = 0; }
        __syncthreads();
        for (int k = 0; k < 32; k++) {
            const int t = warp * 32 + k;
            const int64_t uu = t0 + t;
            if (uu >= n) break;
            const int32_t u = (int32_t)uu;
            const int32_t bu = rp[u], du = rp[u + 1] - bu;
            int64_t est = 0;
            int32_t dp = 0;
            for (int32_t i = lane; i < du; i += WARP) {
                const int32_t v = ci[bu + i], dv = nd[bu + i];
                if (precedes(dv, v, du, u)) est += dv; else dp++;
            }
            est = warp_sum(est);
            dp = warp_sum(dp);
            if (lane == 0) {
                dplus[u] = dp;
                atomicMax(&tile_maxdp, dp);
                int l = -1;
                if (est > 0) {
                    if (est <= TINY_WEDGES) l = 0;
                    else if (est <= small_cap) l = 1;
                    else if (est <= hub_min) {
                        l = 2;
                        atomicMax(&tile_maxw, (unsigned long long)est);
                        west[u] = est;
                        atomicAdd(counters + C_MB0 + min(MB_BUCKETS - 1, 63 - __clzll(est)), 1);
                    } else {
                        l = 3;
                    }
                }
                code_l[t] = (int8_t)l;
                if (l >= 0) pos_l[t] = atomicAdd(&cnt[l], 1);
                // clique buckets by out-degree (a node needs 2 out-neighbours to
                // be the lowest node of a triangle)
                int bkt = -1;
                if (dp >= 2) {
                    bkt = (dp > cl_max || dp > CL_D2) ? 3 : dp <= CL_D0 ? 0 : dp <= CL_D1 ? 1 : 2;
                    pos_b[t] = atomicAdd(&cnt[4 + bkt], 1);
                }
                code_b[t] = (int8_t)bkt;
            }
        }
        __syncthreads();
        if (threadIdx.x < 8) {
            const int l = threadIdx.x;
            const int ctr = l == 0 ? C_TINY : l == 1 ? C_SMALL : l == 2 ? C_MEDIUM : l == 3 ? C_HUB : C_CL0 + (l - 4);
            base[l] = cnt[l] ? atomicAdd(counters + ctr, cnt[l]) : 0;
        }
        if (threadIdx.x == 0) {
            atomicMax(counters + C_MAXDP, tile_maxdp);
            if (tile_maxw) atomicMax(reinterpret_cast<unsigned long long *>(west + n), tile_maxw);
        }
        __syncthreads();
        const int t = threadIdx.x;
        if (t0 + t < n) {
            const int32_t u = (int32_t)(t0 + t);
            const int l = code_l[t];
            if (l == 0) tlist[base[0] + pos_l[t]] = u;
            else if (l == 1) vlist[base[1] + pos_l[t]] = u;
            else if (l == 2) vlist[n - 1 - (base[2] + pos_l[t])] = u;
            else if (l == 3) hubs[base[3] + pos_l[t]] = u;
            const int bk = code_b[t];
            if (bk >= 0) clist[(int64_t)bk * n + base[4 + bk] + pos_b[t]] = u;
        }
        __syncthreads();
    }
}

__global__ void k_dag_fill(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const int32_t *__restrict__ nd, const int32_t *__restrict__ dag_off,
                           int32_t *dag_col, int32_t *dag_slot, int32_t *dag_nd) {
    const int lane = lane_id();
    for (int32_t u = global_warp(); u < n; u += num_warps()) {
        const int32_t bu = rp[u], du = rp[u + 1] - bu;
        int32_t o = dag_off[u];
        for (int32_t i0 = 0; i0 < du; i0 += WARP) {
            const int32_t i = i0 + lane;
            bool up = false;
            int32_t v = 0, dv = 0;
            if (i < du) {
                v = ci[bu + i];
                dv = nd[bu + i];
                up = precedes(du, u, dv, v);
            }
            const unsigned mask = __ballot_sync(FULL, up);
            if (up) {
                const int32_t k = o + __popc(mask & ((1u << lane) - 1));
                dag_col[k] = v; dag_slot[k] = bu + i; dag_nd[k] = dv;
            }
            o += __popc(mask);
        }
    }
}

// Medium tier in decreasing order of wedge work (log2 buckets), so that the
// dynamically scheduled CTAs start the largest vertices first.
__global__ void k_medium_offsets(int32_t *counters) {
    if (threadIdx.x != 0) return;
    int32_t o = 0;
    for (int b = MB_BUCKETS - 1; b >= 0; b--) { counters[C_MOFF + b] = o; o += counters[C_MB0 + b]; }
}

__global__ void k_medium_place(int32_t n, const int32_t *__restrict__ vlist, const int64_t *__restrict__ west,
                               int32_t *counters, int32_t *mlist) {
    const int32_t nm = counters[C_MEDIUM];
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nm; i += gridDim.x * blockDim.x) {
        const int32_t u = vlist[n - 1 - i];
        const int b = min(MB_BUCKETS - 1, 63 - __clzll(west[u]));
        mlist[atomicAdd(counters + C_MOFF + b, 1)] = u;
    }
}

// ---------------------------------------------------------------------------
// triangles + 4-cliques (bitmap over N+(a))
// ---------------------------------------------------------------------------

struct CliqueArgs {
    const int32_t *clist;       // bucket list
    const int32_t *counters;
    int bucket;
    int32_t n;
    const int32_t *rp;
    const int32_t *dag_off, *dag_col, *dag_slot, *dag_nd;
    unsigned long long *cacc;   // per-slot clique credits (per-edge mode)
    uint32_t *tcred;            // per-slot triangle credits
    const uint32_t *tslot;      // |Tri| per slot (triangle-sum mode)
    unsigned long long *qcred;  // per slot: triangle-perimeter credit, then degree-sum credit (triangle-sum mode)
    unsigned long long *sums;   // u128 sums (S_CLIQ gets 6 * K4 in global mode)
    int32_t *status;            // error bits
    unsigned char *gstore;      // per-CTA work arrays of the large out-list variant
    int32_t gdmax;              // its capacity (multiple of 32, >= largest out-degree)
    size_t gstride;             // bytes per CTA
    int32_t *dyn;               // work counter of this launch (zero at launch)
    unsigned long long *pairs;  // per-team triangle records (COUNT, CREDIT)
    int32_t pair_cap;           // records per team (0: none)
    // per-edge mode: triangle records kept from the CREDIT pass for the
    // TRISUM pass, node a's in recs[toff[a], toff[a+1]) when toff[a+1] <=
    // rec_cap; tcnt[a] = records written, or -1 when a has no region
    const int64_t *toff;
    int32_t *tcnt;
    unsigned long long *recs;
    int64_t rec_cap;
};

// MODE_COUNT: |Tri| credits + number of 4-cliques (global counts)
// MODE_CREDIT: |Tri| credits + 4-clique credits on all six edges (per edge)
// MODE_TRISUM: per triangle {a,b,c} with T the final |Tri| of its edges,
//   perimeter P = T(a,b)+T(a,c)+T(b,c) and degree sum d_a+d_b+d_c credited
//   to each of its three edges; per edge e the credits add up to
//   Q(e) = A_u + A_v + T(e)^2 and R(e) = D_T + T(e)(d_u + d_v).
enum { MODE_COUNT = 0, MODE_CREDIT = 1, MODE_TRISUM = 2 };

// Open-addressing table of N+(a) (id -> position), at least twice as many
// slots as entries, and a one-bit filter over the same ids (about 32 bits
// per entry) that rejects most non-members with one shared-memory load.
__host__ __device__ constexpr int32_t clique_hash_slots(int32_t D) {
    int32_t s = 32;
    while (s < 2 * D) s <<= 1;
    return s;
}
__host__ __device__ constexpr int clique_filter_bits(int32_t D) {
    int b = 11;
    while ((1ll << b) < 32ll * D) b++;
    return b;
}
__device__ __forceinline__ uint32_t clique_hash(int32_t x, int bits) {
    return ((uint32_t)x * 0x9E3779B1u) >> (32 - bits);
}

constexpr int CQ = 64;   // candidate queue entries per warp

// Words per row of the bit matrix of an out-list of D entries.  The global
// count pass (MODE_COUNT) reads rows 128 bits at a time: the D bits rounded
// up to whole 16-byte units, plus one unit when their number is even, so
// that rows start an odd number of 16-byte units apart and the loads of
// eight lanes reading eight different rows fall on eight different bank
// groups (a stride of 32 words put every lane of a warp on one bank): R-MAT
// 22 146 -> 138 ms.  The per-edge pass keeps rows of ceil(D / 32) words
// read a word at a time: padded rows measured 0.3 ms slower there on
// Chung-Lu 1M (5.9 -> 6.2 ms).
template <int MODE>
__host__ __device__ constexpr int32_t clique_row_words(int32_t D) {
    const int32_t wd = (D + 31) >> 5, w = (wd + 3) & ~3;
    return MODE != MODE_COUNT ? wd : (w & 7) == 0 ? w + 4 : w;
}

// x added to a 64-bit counter in shared memory through 32-bit atomics on its
// words (little-endian: low word first): the low word's atomic reports its
// own wrap, which is carried into the high word, so the final value is the
// exact sum.  Hot counters take many concurrent adds, and 32-bit shared
// atomics serialise far less than 64-bit ones under contention.
__device__ __forceinline__ void smem_add_u64(unsigned long long *p, unsigned long long x) {
    uint32_t *w = reinterpret_cast<uint32_t *>(p);
    const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    const uint32_t old = atomicAdd(w, lo);
    const uint32_t up = hi + (old + lo < old ? 1u : 0u);
    if (up) atomicAdd(w + 1, up);
}

// Work arrays of one team (a warp or a CTA working on one node a), for an
// out-list of at most D entries (D a multiple of 32).  Position k is the
// k-th entry of N+(a) (ascending ids).
struct CliqueView {
    unsigned long long *qa, *ra;   // TRISUM: P and R credits of (a, c_k)
    int32_t *aslot;                // CSR slot of (a, c_k)
    uint32_t *acc;                 // TRISUM: |Tri| of (a, c_k); else triangles on (a, c_k)
    int32_t *st;                   // DAG offset of N+(c_k)
    int32_t *pre;                  // exclusive prefix of |N+(c_k)|, pre[D] = total
    int32_t *hkey;                 // hash keys (ids, -1 empty)
    uint32_t *filt;                // membership filter
    int32_t *qx, *qq;              // candidate queues (per warp: CQ entries)
    int32_t *adeg;                 // TRISUM: d(c_k)
    uint32_t *cnt;                 // CREDIT: twice the 4-cliques on (a, c_k)
    uint32_t *M;                   // COUNT/CREDIT: adjacency inside N+(a), clique_row_words<MODE>(D) words a row
    uint16_t *hpos;                // hash values (positions)
    uint16_t *qk;                  // candidate queue: list position
};

template <int MODE>
__host__ __device__ constexpr size_t team_bytes(int32_t D, int warps) {
    return (MODE == MODE_TRISUM ? (size_t)D * 16 : 0)          // qa, ra
           + (size_t)D * 12 + (size_t)(D + 32) * 4              // aslot, acc, st, pre
           + (size_t)clique_hash_slots(D) * 4                   // hkey
           + ((size_t)1 << clique_filter_bits(D)) / 8           // filt
           + (size_t)warps * CQ * 8                             // qx, qq
           + (MODE != MODE_COUNT ? (size_t)D * 4 : 0)           // adeg or cnt
           + (MODE != MODE_TRISUM ? (size_t)D * (size_t)clique_row_words<MODE>(D) * 4 : 0)   // M
           + (size_t)clique_hash_slots(D) * 2                   // hpos
           + (size_t)warps * CQ * 2;                            // qk
}

template <int MODE>
__device__ __forceinline__ CliqueView carve(unsigned char *base, int32_t D, int warps) {
    CliqueView S;
    S.qa = S.ra = nullptr;
    if (MODE == MODE_TRISUM) {
        S.qa = reinterpret_cast<unsigned long long *>(base);
        S.ra = S.qa + D;
        base += (size_t)D * 16;
    }
    int32_t *p = reinterpret_cast<int32_t *>(base);
    S.aslot = p; p += D;
    S.acc = reinterpret_cast<uint32_t *>(p); p += D;
    S.st = p; p += D;
    S.pre = p; p += D + 32;
    S.hkey = p; p += clique_hash_slots(D);
    S.filt = reinterpret_cast<uint32_t *>(p); p += (1 << clique_filter_bits(D)) / 32;
    S.qx = p; p += warps * CQ;
    S.qq = p; p += warps * CQ;
    S.adeg = p;
    S.cnt = reinterpret_cast<uint32_t *>(p);
    if (MODE != MODE_COUNT) p += D;
    S.M = reinterpret_cast<uint32_t *>(p);
    if (MODE != MODE_TRISUM) p += (size_t)D * clique_row_words<MODE>(D);
    S.hpos = reinterpret_cast<uint16_t *>(p);
    S.qk = S.hpos + clique_hash_slots(D);
    return S;
}

// Position of id x in N+(a), or -1.
__device__ __forceinline__ int32_t clique_find(const CliqueView &S, int32_t x, int bits) {
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t h = clique_hash(x, bits);
    for (uint32_t probe = 0; probe <= mask; probe++) {
        const int32_t k = S.hkey[h];
        if (k == x) return S.hpos[h];
        if (k < 0) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

// Every pair (c, x) with c in N+(a) and x in N+(c): the concatenated
// out-lists (total pre[D]) are split into 32-entry groups, each warp of the
// team taking a contiguous share of the groups; a lane finds the list of its
// entry by walking forward from the list of the previous group's last entry
// (no walk when the group lies inside one list).  Entries that pass the
// filter go to the warp's queue; 32 at a time, the lanes look them up in the
// table and call f(kc, kx, q, hm) for every pair whose x is in N+(a) too: kc,
// kx are the positions of c and x in N+(a), q the DAG entry of x in N+(c), so
// dag_slot[q] is the CSR slot of (c, x), and hm the mask of the lanes making
// the call together.  Each such pair is the triangle {a, c, x} with a lowest,
// found exactly once.
template <int TW, typename F>
__device__ __forceinline__ void scan_pairs(const CliqueArgs &a, const CliqueView &S, int32_t D, int bits, int fbits,
                                           int tw, F f) {
    const int lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    int32_t *qx = S.qx + tw * CQ, *qq = S.qq + tw * CQ;
    uint16_t *qk = S.qk + tw * CQ;
    auto drain = [&](int32_t cnt) {
        __syncwarp();
        const int32_t kx = lane < cnt ? clique_find(S, qx[lane], bits) : -1;
        const unsigned hm = __ballot_sync(FULL, kx >= 0);
        if (kx >= 0) f((int32_t)qk[lane], kx, qq[lane], hm);
        __syncwarp();
    };
    const int32_t total = S.pre[D];
    const int32_t G = (total + 31) >> 5;
    const int32_t g0 = (int32_t)(((int64_t)G * tw) / TW), g1 = (int32_t)(((int64_t)G * (tw + 1)) / TW);
    if (g0 >= g1) return;
    // list of the first entry: the last k with pre[k] <= g0 * 32
    int32_t lo = 0, hi = D - 1;
    {
        const int32_t w0 = g0 * 32;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (S.pre[mid] <= w0) lo = mid; else hi = mid - 1;
        }
    }
    int32_t kcur = lo, qn = 0;
    for (int32_t g = g0; g < g1; g++) {
        const int32_t w0 = g * 32, w = w0 + lane;
        int32_t k = kcur;
        bool cand = false;
        int32_t x = 0, q = 0;
        if (w < total) {
            if (S.pre[kcur + 1] < w0 + 32)
                while (S.pre[k + 1] <= w) k++;
            q = S.st[k] + (w - S.pre[k]);
            x = ldg(a.dag_col + q);
            const uint32_t fh = clique_hash(x, fbits);
            cand = (S.filt[fh >> 5] >> (fh & 31)) & 1u;
        }
        const unsigned m = __ballot_sync(FULL, cand);
        if (cand) {
            const int32_t p = qn + __popc(m & lt);
            qx[p] = x; qq[p] = q; qk[p] = (uint16_t)k;
        }
        qn += __popc(m);
        if (qn >= 32) {
            drain(32);
            if (lane < qn - 32) { qx[lane] = qx[32 + lane]; qq[lane] = qq[32 + lane]; qk[lane] = qk[32 + lane]; }
            qn -= 32;
            __syncwarp();
        }
        kcur = __shfl_sync(FULL, k, 31);
    }
    if (qn > 0) drain(qn);
}

// One team per node a of the bucket, the nodes taken in list order from a
// shared counter.  WARP_TEAMS: every warp of the CTA is a team with its own
// slice of shared memory (small out-lists); otherwise the whole CTA is one
// team.  DMAX == 0: work arrays in the CTA's slice of global scratch
// (out-lists above the shared-memory limit).  COUNT and CREDIT record the
// triangles found by the first scan (positions and the slot of (c, x)) in the
// team's slice of a.pairs, so the 4-clique phase walks only those; a node
// with more than a.pair_cap of them scans its lists again instead.
template <int DMAX, int THREADS, bool WARP_TEAMS, int MODE>
__global__ void __launch_bounds__(THREADS)
k_clique_bitmap(CliqueArgs a) {
    constexpr int NW = THREADS / 32;
    constexpr int TEAMS = WARP_TEAMS ? NW : 1;
    constexpr int TW = WARP_TEAMS ? 1 : NW;          // warps per team
    static_assert(DMAX > 0 || !WARP_TEAMS, "global scratch holds one team per CTA");
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int32_t wsum[NW];
    __shared__ int32_t next_idx;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const int team = WARP_TEAMS ? warp : 0;
    const int tw = WARP_TEAMS ? 0 : warp;            // warp index inside the team
    const int tt = tw * 32 + lane;                   // thread index inside the team
    const int32_t dm = DMAX > 0 ? DMAX : a.gdmax;
    unsigned char *base = DMAX > 0 ? smraw + (size_t)team * team_bytes<MODE>(DMAX, TW)
                                   : a.gstore + (size_t)blockIdx.x * a.gstride;
    const CliqueView S = carve<MODE>(base, dm, TW);
    int32_t *npair = S.pre + dm + 16;                // triangles recorded for the current node
    unsigned long long *mypairs = a.pairs + ((size_t)blockIdx.x * TEAMS + team) * (size_t)a.pair_cap;
    auto team_sync = [] { if (WARP_TEAMS) __syncwarp(); else __syncthreads(); };
    // next node index of this team (the counter hands out list positions)
    auto take = [&](int32_t mine) {
        if (WARP_TEAMS) return __shfl_sync(FULL, mine, 0);
        if (threadIdx.x == 0) next_idx = mine;
        __syncthreads();
        const int32_t v = next_idx;
        __syncthreads();
        return v;
    };

    const int32_t nv = a.counters[C_CL0 + a.bucket];
    const int32_t *list = a.clist + (int64_t)a.bucket * a.n;
    unsigned long long k4_local = 0;   // 4-cliques (COUNT)

    // warp teams claim CH consecutive list positions per atomic (one counter
    // for ~a million small nodes would serialise on it); CTA teams one
    constexpr int32_t CH = WARP_TEAMS ? 8 : 1;
    int32_t cbase = take(tt == 0 ? atomicAdd(a.dyn, CH) : 0), cnext = 0;
    int32_t idx = cbase;
    while (idx < nv) {
        if (idx == cbase) cnext = take(tt == 0 ? atomicAdd(a.dyn, CH) : 0);   // the team's next chunk
        const int32_t va = list[idx];
        const int32_t off = a.dag_off[va], D = a.dag_off[va + 1] - off;
        const int32_t Wd = (D + 31) >> 5, Ws = clique_row_words<MODE>(D);
        const int32_t hs = clique_hash_slots(D);
        const int bits = 31 - __clz(hs);
        const int fbits = clique_filter_bits(D);
        // TRISUM: records kept by the CREDIT pass replace the scan
        const int32_t ne = (MODE == MODE_TRISUM && a.tcnt != nullptr) ? a.tcnt[va] : -1;
        const bool scan = ne < 0;
        if (scan) {
            for (int32_t i = tt; i < hs; i += TW * 32) S.hkey[i] = -1;
            for (int32_t i = tt; i < (1 << fbits) / 32; i += TW * 32) S.filt[i] = 0;
        }
        if (MODE != MODE_TRISUM)
            if (MODE != MODE_COUNT)
                for (int32_t i = tt; i < D * Ws; i += TW * 32) S.M[i] = 0;
            else
                for (int32_t i = tt; i < (D * Ws) >> 2; i += TW * 32) reinterpret_cast<uint4 *>(S.M)[i] = make_uint4(0, 0, 0, 0);
        if (tt == 0) *npair = 0;
        team_sync();
        for (int32_t k = tt; k < D; k += TW * 32) {
            const int32_t c = ldg(a.dag_col + off + k);
            const int32_t s = ldg(a.dag_slot + off + k);
            S.aslot[k] = s;
            if (MODE == MODE_TRISUM) {
                S.adeg[k] = ldg(a.dag_nd + off + k);
                S.acc[k] = __ldg(a.tslot + s);
                S.qa[k] = 0;
                S.ra[k] = 0;
            } else {
                S.acc[k] = 0;
                if (MODE == MODE_CREDIT) S.cnt[k] = 0;
            }
            if (!scan) continue;
            const int32_t o = ldg(a.dag_off + c);
            S.st[k] = o;
            S.pre[k] = ldg(a.dag_off + c + 1) - o;
            // the table has at least 2D slots, so a free one is always found
            uint32_t h = clique_hash(c, bits);
            int32_t probe = 0;
            for (; probe < hs; probe++) {
                if (atomicCAS(&S.hkey[h], -1, c) == -1) { S.hpos[h] = (uint16_t)k; break; }
                h = (h + 1) & (uint32_t)(hs - 1);
            }
            if (probe == hs) atomicOr(a.status, ERR_CAPACITY);
            const uint32_t fh = clique_hash(c, fbits);
            atomicOr(&S.filt[fh >> 5], 1u << (fh & 31));
        }
        team_sync();
        // pre <- exclusive prefix of the list lengths
        if (scan) {
            int32_t carry = 0;
            for (int32_t r0 = 0; r0 < D; r0 += TW * 32) {
                const int32_t k = r0 + tt;
                const int32_t v = k < D ? S.pre[k] : 0;
                const int32_t incl = warp_incl_scan(v);
                if (TW > 1) {
                    if (lane == 31) wsum[tw] = incl;
                    __syncthreads();
                    int32_t before = 0, all = 0;
                    for (int j = 0; j < TW; j++) { const int32_t s = wsum[j]; before += j < tw ? s : 0; all += s; }
                    __syncthreads();
                    if (k < D) S.pre[k] = carry + before + incl - v;
                    carry += all;
                } else {
                    if (k < D) S.pre[k] = carry + incl - v;
                    carry += __shfl_sync(FULL, incl, 31);
                }
            }
            if (tt == 0) S.pre[D] = carry;
        }
        team_sync();

        if (MODE == MODE_TRISUM) {
            const unsigned long long da = (unsigned long long)(a.rp[va + 1] - a.rp[va]);
            auto tri_t = [&](int32_t kc, int32_t kx, int32_t s, uint32_t tcx) {
                const unsigned long long P = (unsigned long long)S.acc[kc] + S.acc[kx] + tcx;
                const unsigned long long R = da + (unsigned long long)S.adeg[kc] + (unsigned long long)S.adeg[kx];
                atomicAdd(a.qcred + 2 * (int64_t)s, P);
                atomicAdd(a.qcred + 2 * (int64_t)s + 1, R);
                smem_add_u64(&S.qa[kc], P);
                smem_add_u64(&S.qa[kx], P);
                smem_add_u64(&S.ra[kc], R);
                smem_add_u64(&S.ra[kx], R);
            };
            if (scan) {
                scan_pairs<TW>(a, S, D, bits, fbits, tw, [&](int32_t kc, int32_t kx, int32_t q, unsigned) {
                    const int32_t s = ldg(a.dag_slot + q);
                    tri_t(kc, kx, s, __ldg(a.tslot + s));
                });
            } else {
                // four records per lane at a time: their |Tri| gathers in flight together
                const unsigned long long *rec = a.recs + a.toff[va];
                constexpr int32_t ST = TW * 32;
                int32_t i = tt;
                for (; i + 3 * ST < ne; i += 4 * ST) {
                    unsigned long long v[4];
                    uint32_t t[4];
#pragma unroll
                    for (int j = 0; j < 4; j++) v[j] = rec[i + j * ST];
#pragma unroll
                    for (int j = 0; j < 4; j++) t[j] = __ldg(a.tslot + (int32_t)(v[j] >> 32));
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        tri_t((int32_t)(v[j] & 0xffffu), (int32_t)((v[j] >> 16) & 0xffffu), (int32_t)(v[j] >> 32), t[j]);
                }
                for (; i < ne; i += ST) {
                    const unsigned long long v = rec[i];
                    const int32_t s = (int32_t)(v >> 32);
                    tri_t((int32_t)(v & 0xffffu), (int32_t)((v >> 16) & 0xffffu), s, __ldg(a.tslot + s));
                }
            }
            team_sync();
            for (int32_t k = tt; k < D; k += TW * 32) {
                if (S.qa[k]) atomicAdd(a.qcred + 2 * (int64_t)S.aslot[k], S.qa[k]);
                if (S.ra[k]) atomicAdd(a.qcred + 2 * (int64_t)S.aslot[k] + 1, S.ra[k]);
            }
        } else {
            // the triangle record: node a's own region when it has one (kept
            // for the TRISUM pass), else the team's scratch slice
            unsigned long long *rec = mypairs;
            int64_t rcap = a.pair_cap;
            bool stored = false;
            if (MODE == MODE_CREDIT && a.recs != nullptr) {
                const int64_t o0 = a.toff[va], o1 = a.toff[va + 1];
                if (o1 <= a.rec_cap) { rec = a.recs + o0; rcap = o1 - o0; stored = true; }
            }
            // adjacency inside N+(a), the triangle credits, the triangle record
            // (the calling lanes hm often share c: one counter update per
            // distinct position, one record-index reservation per call)
            const unsigned lt = (1u << lane) - 1u;
            scan_pairs<TW>(a, S, D, bits, fbits, tw, [&](int32_t kc, int32_t kx, int32_t q, unsigned hm) {
                const int32_t s = ldg(a.dag_slot + q);
                atomicOr(&S.M[kc * Ws + (kx >> 5)], 1u << (kx & 31));
                atomicOr(&S.M[kx * Ws + (kc >> 5)], 1u << (kc & 31));
                atomicAdd(a.tcred + s, 1u);
                const unsigned peers = __match_any_sync(hm, kc);
                if ((peers & lt) == 0) atomicAdd(&S.acc[kc], (uint32_t)__popc(peers));
                atomicAdd(&S.acc[kx], 1u);
                const int lead = __ffs(hm) - 1;
                int32_t i = 0;
                if (lane == lead) i = atomicAdd(npair, __popc(hm));
                i = __shfl_sync(hm, i, lead) + __popc(hm & lt);
                if (i < rcap)
                    rec[i] = ((unsigned long long)(uint32_t)s << 32) | ((uint32_t)kx << 16) | (uint32_t)kc;
            });
            team_sync();
            const int32_t np = *npair;
            if (MODE == MODE_CREDIT && a.tcnt != nullptr && tt == 0) {
                // a region holds at most min(C(D,2), pairs scanned) >= np records
                if (stored && np > rcap) atomicOr(a.status, ERR_CAPACITY);
                a.tcnt[va] = stored && np <= rcap ? np : -1;
            }
            // inner edge (c, x): the 4-cliques {a, c, x, d} are the common
            // neighbours d of c and x inside N+(a)
            auto inner = [&](int32_t kc, int32_t kx, int32_t s) {
                uint32_t kq = 0;
                if (MODE != MODE_COUNT) {
                    for (int32_t w = 0; w < Wd; w++) kq += __popc(S.M[kc * Ws + w] & S.M[kx * Ws + w]);
                } else {
                    // global count: each 4-clique {a, c, x, d} once, from its
                    // triangle whose third inner node d comes after both c and
                    // x in N+(a) (the bits of positions > max(kc, kx))
                    const uint4 *rc = reinterpret_cast<const uint4 *>(S.M + kc * Ws);
                    const uint4 *rx = reinterpret_cast<const uint4 *>(S.M + kx * Ws);
                    const int32_t from = max(kc, kx) + 1, nw4 = (Wd + 3) >> 2;
                    int32_t w = from >> 7;
                    if (w < nw4) {
                        const int32_t b = from & 127, wi = b >> 5;
                        const uint32_t mb = 0xffffffffu << (b & 31);
                        const uint4 p = rc[w], q = rx[w];
                        kq += __popc(p.x & q.x & (wi == 0 ? mb : 0u)) +
                              __popc(p.y & q.y & (wi == 1 ? mb : wi < 1 ? ~0u : 0u)) +
                              __popc(p.z & q.z & (wi == 2 ? mb : wi < 2 ? ~0u : 0u)) +
                              __popc(p.w & q.w & (wi == 3 ? mb : ~0u));
                    }
                    for (w++; w < nw4; w++) {
                        const uint4 p = rc[w], q = rx[w];
                        kq += __popc(p.x & q.x) + __popc(p.y & q.y) + __popc(p.z & q.z) + __popc(p.w & q.w);
                    }
                }
                if (MODE == MODE_COUNT) {
                    k4_local += kq;
                } else if (kq) {
                    atomicAdd(a.cacc + s, (unsigned long long)kq);
                    atomicAdd(&S.cnt[kc], kq);
                    atomicAdd(&S.cnt[kx], kq);
                }
            };
            if (np <= rcap) {
                for (int32_t i = tt; i < np; i += TW * 32) {
                    const unsigned long long v = rec[i];
                    inner((int32_t)(v & 0xffffu), (int32_t)((v >> 16) & 0xffffu), (int32_t)(v >> 32));
                }
            } else if (MODE == MODE_CREDIT) {
                scan_pairs<TW>(a, S, D, bits, fbits, tw, [&](int32_t kc, int32_t kx, int32_t q, unsigned) {
                    inner(kc, kx, ldg(a.dag_slot + q));
                });
            } else {
                for (int32_t kc = tw; kc < D; kc += TW)
                    for (int32_t kx = kc + 1 + lane; kx < D; kx += WARP)
                        if ((S.M[kc * Ws + (kx >> 5)] >> (kx & 31)) & 1u) inner(kc, kx, 0);
            }
            team_sync();
            // credits of the edges (a, c_k)
            for (int32_t k = tt; k < D; k += TW * 32) {
                if (S.acc[k]) atomicAdd(a.tcred + S.aslot[k], S.acc[k]);
                if (MODE == MODE_CREDIT && S.cnt[k]) atomicAdd(a.cacc + S.aslot[k], (unsigned long long)(S.cnt[k] >> 1));
            }
        }
        team_sync();
        if (++idx == cbase + CH) { cbase = cnext; idx = cbase; }
    }
    if (MODE == MODE_COUNT) {
        __shared__ unsigned long long red[NW];
        const unsigned long long x = warp_sum(k4_local);
        if (lane == 0) red[warp] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long s = 0;
            for (int w = 0; w < NW; w++) s += red[w];
            add_u128(a.sums + 2 * S_CLIQ, 6ull * s);   // sum_e cliq_e = 6 K4
        }
    }
}

// Upper bound of the triangles whose lowest node is a: C(|N+(a)|, 2), and
// the number of pairs (c, x) a scan of N+(a) visits.
__global__ void k_tri_bound(int32_t n, const int32_t *__restrict__ dag_off, const int32_t *__restrict__ dag_col,
                            int64_t *bound) {
    const int lane = lane_id();
    for (int32_t u = global_warp(); u < n; u += num_warps()) {
        const int32_t o = dag_off[u], D = dag_off[u + 1] - o;
        int64_t x = 0;
        for (int32_t k = lane; k < D; k += WARP) {
            const int32_t c = dag_col[o + k];
            x += dag_off[c + 1] - dag_off[c];
        }
        x = warp_sum(x);
        if (lane == 0) bound[u] = D >= 2 ? min((int64_t)D * (D - 1) / 2, x) : 0;
    }
}

// |Tri_e| of both slots of every edge from the triangle credits
__global__ void k_tri_symmetrize(int64_t m, const int32_t *__restrict__ eslot, const int32_t *__restrict__ mate,
                                 const uint32_t *__restrict__ tcred, uint32_t *tslot) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = eslot[k], q = mate[p];
        const uint32_t t = tcred[p] + tcred[q];
        tslot[p] = t;
        tslot[q] = t;
    }
}

// ---------------------------------------------------------------------------
// 4-cycles
// ---------------------------------------------------------------------------

// Load-balanced walk over the wedges (u, v, y), v and y below u, for the
// neighbours of u at positions [i0, i1) taken 32 at a time by one warp.
// f(item_lane, slot_vy, y) is called for every wedge; item_lane is the lane
// that loaded v (slot of (u, v) = bu + it + item_lane).  done(it) is called
// by the whole warp after each group of 32 neighbours.
template <class F, class G>
__device__ __forceinline__ void warp_wedges(int32_t u, int32_t du, int32_t bu, int32_t i0, int32_t i1,
                                            int32_t istep, const int32_t *__restrict__ rp,
                                            const int32_t *__restrict__ ci, const int32_t *__restrict__ nd,
                                            F f, G done) {
    const int lane = lane_id();
    for (int32_t it = i0; it < i1; it += istep) {
        const int32_t i = it + lane;
        int32_t len = 0, start = 0;
        if (i < i1 && i < it + WARP) {
            const int32_t v = ci[bu + i], dv = nd[bu + i];
            if (precedes(dv, v, du, u)) { len = dv; start = rp[v]; }
        }
        const int32_t incl = warp_incl_scan(len);
        const int32_t total = __shfl_sync(FULL, incl, 31);
        const int32_t excl = incl - len;
        for (int32_t w0 = 0; w0 < total; w0 += WARP) {
            const int32_t w = w0 + lane;
            int32_t k = 0;
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                const int32_t e = __shfl_sync(FULL, excl, k + s);
                if (e <= w) k += s;
            }
            const int32_t ks = __shfl_sync(FULL, start, k);
            const int32_t ke = __shfl_sync(FULL, excl, k);
            bool ok = false;
            const bool live = w < total;
            int32_t q = 0, y = 0;
            if (live) {
                q = ks + (w - ke);
                y = ci[q];
                ok = precedes(nd[q], y, du, u);
            }
            // called by every lane: ok says whether (k, q, y) is a wedge, live
            // whether the lane lies inside this group's wedge range
            f(k, q, y, ok, live);
        }
        done(it);
    }
}

// Per-item sums inside warp_wedges: the in-range lanes of one inner
// iteration hold wedges of non-decreasing items k, each item on a contiguous
// run of lanes, so a segmented warp scan leaves the last lane of each run to
// add the run's sum to the item accumulator.  Lanes past the end of the
// group (live == false) form runs of their own and add nothing.
__device__ __forceinline__ void item_add(unsigned long long *item, int k, unsigned long long x, bool live) {
    const int lane = lane_id();
    const int kk = live ? k : -1 - lane;
    unsigned long long s = live ? x : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULL, s, o);
        const int ky = __shfl_up_sync(FULL, kk, o);
        if (lane >= o && ky == kk) s += y;
    }
    const int knext = __shfl_down_sync(FULL, kk, 1);
    const bool tail = (lane == 31) || (knext != kk);
    if (live && tail && s) atomicAdd(item + k, s);
}

// shared-memory hash (keys -1 = empty); at most cap/2 distinct keys
__device__ __forceinline__ uint32_t sm_find(const int32_t *keys, const uint32_t *vals, uint32_t capmask, int32_t y) {
    uint32_t h = hash32((uint32_t)y) & capmask;
    for (uint32_t probes = 0; probes <= capmask; probes++) {
        const int32_t k = keys[h];
        if (k == y) return vals[h];
        if (k == -1) return 0;
        h = (h + 1) & capmask;
    }
    return 0;
}

struct CycleArgs {
    int32_t n;
    const int32_t *rp, *ci, *nd;
    const int32_t *vlist, *hubs, *mlist, *tlist;
    int32_t *counters;           // counters[C_DYN] is the medium tier's work index
    uint32_t capmask;
    uint32_t *tables;            // [hub batch][n] dense counters, zero at rest
    unsigned long long *mtab;    // medium tier: per-CTA open-addressing tables, empty at rest
    int64_t mcap;                // their entries per CTA (power of two)
    const int64_t *west;         // wedges per medium vertex
    unsigned long long *yacc;    // per-slot 4-cycle credits (per-edge mode)
    uint32_t *y32;               // the same as 32-bit words (non-null when every slot's total fits)
    unsigned long long *sums;    // u128 sums: X_C4 gets sum_e C4(e) = 4 * 4-cycles (global mode)
    int32_t *status;             // error bits
    int32_t hub0, nhub;          // hub batch
    int64_t *hoff;               // [17] row offsets of the batch's hubs in the flat neighbour list
    int64_t *hlen;               // [flat] wedges contributed by each neighbour; after the
                                 // prefix, the neighbour's row (k_hub_rows)
    int64_t *hpre;               // [flat + 1] exclusive prefix of hlen (hpre[flat] = batch wedges)
};

// credit x 4-cycles to slot q
__device__ __forceinline__ void ycredit(const CycleArgs &a, int64_t q, unsigned long long x) {
    if (a.y32) atomicAdd(a.y32 + q, (uint32_t)x);
    else atomicAdd(a.yacc + q, x);
}

__device__ __forceinline__ unsigned long long c2(uint32_t c) { return (unsigned long long)c * (c - 1) / 2; }

// Wedge prefix over N(u) in shared memory: pre[i] = wedges of the
// neighbours before i (d_v for v below u, else 0), pre[du] = W(u).  All
// threads of the CTA call it; wsum holds THREADS / 32 entries.
template <int THREADS>
__device__ __forceinline__ long long wedge_prefix(const CycleArgs &a, int32_t u, int32_t bu, int32_t du,
                                                  long long *pre, long long *wsum) {
    constexpr int NW = THREADS / 32;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    long long carry = 0;
    for (int32_t b0 = 0; b0 < du; b0 += THREADS) {
        const int32_t i = b0 + threadIdx.x;
        long long len = 0;
        if (i < du) {
            const int32_t v = a.ci[bu + i], dv = a.nd[bu + i];
            if (precedes(dv, v, du, u)) len = dv;
        }
        long long incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        long long before = 0, all = 0;
        for (int j = 0; j < NW; j++) { const long long t = wsum[j]; before += j < warp ? t : 0; all += t; }
        if (i < du) pre[i] = carry + before + incl - len;
        carry += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) pre[du] = carry;
    __syncthreads();
    return carry;
}

// The wedges [w_lo, w_hi) of vertex u (flat over N(u) by the prefix pre):
// neighbours 32 at a time, their lists clipped to the range and spread over
// the lanes.  f(k, q, y, ok, live) per wedge slot as in warp_wedges;
// flush(j) after each group of 32 neighbours, j = the lane's neighbour.
template <typename F, typename G>
__device__ __forceinline__ void walk_range(const CycleArgs &a, int32_t u, int32_t bu, int32_t du,
                                           const long long *pre, long long w_lo, long long w_hi, F f, G flush) {
    if (w_lo >= w_hi) return;
    const int lane = lane_id();
    int32_t lo = 0, hi = du;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= w_lo) lo = mid; else hi = mid - 1;
    }
    for (int32_t j0 = lo; j0 < du && pre[j0] < w_hi; j0 += WARP) {
        const int32_t j = j0 + lane;
        int32_t len = 0, start = 0;
        if (j < du) {
            const long long p0 = pre[j], p1 = pre[j + 1];
            const long long s0 = max(p0, w_lo), e0 = min(p1, w_hi);
            if (e0 > s0) {
                len = (int32_t)(e0 - s0);
                start = a.rp[a.ci[bu + j]] + (int32_t)(s0 - p0);
            }
        }
        const int32_t incl = warp_incl_scan(len);
        const int32_t total = __shfl_sync(FULL, incl, 31);
        const int32_t excl = incl - len;
        for (int32_t w0 = 0; w0 < total; w0 += WARP) {
            const int32_t w = w0 + lane;
            int32_t k = 0;
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                const int32_t e = __shfl_sync(FULL, excl, k + s);
                if (e <= w) k += s;
            }
            const int32_t ks = __shfl_sync(FULL, start, k);
            const int32_t ke = __shfl_sync(FULL, excl, k);
            const bool live = w < total;
            bool ok = false;
            int32_t q = 0, y = 0;
            if (live) {
                q = ks + (w - ke);
                y = a.ci[q];
                ok = precedes(a.nd[q], y, du, u);
            }
            f(k, q, y, ok, live);
        }
        flush(j);
    }
}

// walk_range with two wedges per lane at a time (w0 + lane and w0 + 32 +
// lane), so that their table probes can be in flight together:
// f2(k0, q0, y0, ok0, live0, k1, q1, y1, ok1, live1), each half a 32-wedge
// group as in walk_range.
template <typename F2, typename G>
__device__ __forceinline__ void walk_range2(const CycleArgs &a, int32_t u, int32_t bu, int32_t du,
                                            const long long *pre, long long w_lo, long long w_hi, F2 f2, G flush) {
    if (w_lo >= w_hi) return;
    const int lane = lane_id();
    int32_t lo = 0, hi = du;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= w_lo) lo = mid; else hi = mid - 1;
    }
    for (int32_t j0 = lo; j0 < du && pre[j0] < w_hi; j0 += WARP) {
        const int32_t j = j0 + lane;
        int32_t len = 0, start = 0;
        if (j < du) {
            const long long p0 = pre[j], p1 = pre[j + 1];
            const long long s0 = max(p0, w_lo), e0 = min(p1, w_hi);
            if (e0 > s0) {
                len = (int32_t)(e0 - s0);
                start = a.rp[a.ci[bu + j]] + (int32_t)(s0 - p0);
            }
        }
        const int32_t incl = warp_incl_scan(len);
        const int32_t total = __shfl_sync(FULL, incl, 31);
        const int32_t excl = incl - len;
        for (int32_t w0 = 0; w0 < total; w0 += 2 * WARP) {
            int32_t k[2], q[2], y[2];
            bool ok[2], live[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int32_t w = w0 + h * WARP + lane;
                int32_t kk = 0;
#pragma unroll
                for (int s = 16; s >= 1; s >>= 1) {
                    const int32_t e = __shfl_sync(FULL, excl, kk + s);
                    if (e <= w) kk += s;
                }
                const int32_t ks = __shfl_sync(FULL, start, kk);
                const int32_t ke = __shfl_sync(FULL, excl, kk);
                k[h] = kk;
                live[h] = w < total;
                ok[h] = false;
                q[h] = 0;
                y[h] = 0;
                if (live[h]) {
                    q[h] = ks + (w - ke);
                    y[h] = a.ci[q[h]];
                    ok[h] = precedes(a.nd[q[h]], y[h], du, u);
                }
            }
            f2(k[0], q[0], y[0], ok[0], live[0], k[1], q[1], y[1], ok[1], live[1]);
        }
        flush(j);
    }
}

// Wedge prefix of the small tier in shared memory: vertices of larger
// degree walk their neighbours 32 at a time per warp instead.
constexpr int SMALL_PCAP = 2048;

// Tiny tier: one warp per vertex (at most TINY_WEDGES wedges), each warp
// with its own shared-memory hash of 2 * TINY_WEDGES entries; no CTA barriers.
template <bool CREDIT>
__global__ void __launch_bounds__(256)
k_cycles_tiny(CycleArgs a) {
    constexpr int NW = 8, TCAP = 2 * TINY_WEDGES;
    constexpr uint32_t TMASK = TCAP - 1;
    __shared__ int32_t keys[NW][TCAP];
    __shared__ uint32_t vals[NW][TCAP];
    __shared__ int32_t touched[NW][TINY_WEDGES];
    __shared__ int32_t ntch[NW];
    __shared__ unsigned long long item[NW][WARP];
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    int32_t *K = keys[warp];
    uint32_t *V = vals[warp];
    int32_t *tl = touched[warp];
    for (int i = lane; i < TCAP; i += WARP) { K[i] = -1; V[i] = 0; }
    if (lane == 0) ntch[warp] = 0;
    item[warp][lane] = 0;
    __syncwarp();
    const int32_t nv = a.counters[C_TINY];
    unsigned long long c4 = 0;
    for (int32_t idx = global_warp(); idx < nv; idx += num_warps()) {
        const int32_t u = a.tlist[idx];
        const int32_t bu = a.rp[u], du = a.rp[u + 1] - bu;
        warp_wedges(u, du, bu, 0, du, WARP, a.rp, a.ci, a.nd,
            [&](int k, int32_t q, int32_t y, bool ok, bool live) {
                if (!ok) return;
                uint32_t h = hash32((uint32_t)y) & TMASK;
                uint32_t old = 0;
                while (true) {
                    const int32_t kk = K[h];
                    if (kk == y) { old = atomicAdd(V + h, 1u); break; }
                    if (kk == -1) {
                        const int32_t prev = atomicCAS(K + h, -1, y);
                        if (prev == -1) { old = atomicAdd(V + h, 1u); tl[atomicAdd(&ntch[warp], 1)] = (int32_t)h; break; }
                        if (prev == y) { old = atomicAdd(V + h, 1u); break; }
                    }
                    h = (h + 1) & TMASK;
                }
                if (!CREDIT) c4 += old;
            },
            [&](int32_t) {});
        __syncwarp();
        if (CREDIT) {
            warp_wedges(u, du, bu, 0, du, WARP, a.rp, a.ci, a.nd,
                [&](int k, int32_t q, int32_t y, bool ok, bool live) {
                    const uint32_t c = ok ? sm_find(K, V, TMASK, y) : 0;
                    if (c > 1) ycredit(a, q, (unsigned long long)(c - 1));
                    item_add(item[warp], k, c > 1 ? c - 1 : 0, live);
                },
                [&](int32_t it) {
                    __syncwarp();
                    const unsigned long long s = item[warp][lane];
                    if (s) { ycredit(a, bu + it + lane, s); item[warp][lane] = 0; }
                    __syncwarp();
                });
            __syncwarp();
        }
        const int32_t nt = ntch[warp];
        for (int32_t i = lane; i < nt; i += WARP) { const int32_t h = tl[i]; K[h] = -1; V[h] = 0; }
        __syncwarp();
        if (lane == 0) ntch[warp] = 0;
        __syncwarp();
    }
    if (!CREDIT) {
        c4 = warp_sum(c4);
        if (lane == 0) add_u128(a.sums + 2 * (S_NUM + X_C4), 4 * c4);
    }
}


template <int THREADS, bool CREDIT>
__global__ void __launch_bounds__(THREADS)
k_cycles_small(CycleArgs a) {
    constexpr int NW = THREADS / 32;
    extern __shared__ __align__(16) int32_t sm[];
    __shared__ int32_t ntouched;
    __shared__ unsigned long long item[NW][WARP];
    __shared__ long long wsum[NW];
    // wedge prefix (SMALL_PCAP + 1 entries), then the hash keys, counts and touched slots
    long long *pre = reinterpret_cast<long long *>(sm);
    int32_t *keys = sm + 2 * (SMALL_PCAP + 1);
    uint32_t *vals = (uint32_t *)(keys + (a.capmask + 1));
    int32_t *touched = keys + 2 * (a.capmask + 1);
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const int32_t nv = a.counters[C_SMALL];
    for (uint32_t i = threadIdx.x; i <= a.capmask; i += THREADS) { keys[i] = -1; vals[i] = 0; }
    if (threadIdx.x == 0) ntouched = 0;
    item[warp][lane] = 0;
    unsigned long long c4 = 0;
    __syncthreads();
    for (int32_t idx = blockIdx.x; idx < nv; idx += gridDim.x) {
        const int32_t u = a.vlist[idx];
        const int32_t bu = a.rp[u], du = a.rp[u + 1] - bu;
        auto count = [&](int k, int32_t q, int32_t y, bool ok, bool live) {
            if (!ok) return;
            uint32_t h = hash32((uint32_t)y) & a.capmask;
            uint32_t old = 0;
            for (uint32_t probe = 0; probe <= a.capmask; probe++) {
                const int32_t kk = keys[h];
                if (kk == y) { old = atomicAdd(vals + h, 1u); break; }
                if (kk == -1) {
                    const int32_t prev = atomicCAS(keys + h, -1, y);
                    if (prev == -1) { old = atomicAdd(vals + h, 1u); touched[atomicAdd(&ntouched, 1)] = (int32_t)h; break; }
                    if (prev == y) { old = atomicAdd(vals + h, 1u); break; }
                }
                h = (h + 1) & a.capmask;
            }
            if (!CREDIT) c4 += old;
        };
        auto credit = [&](int k, int32_t q, int32_t y, bool ok, bool live) {
            const uint32_t c = ok ? sm_find(keys, vals, a.capmask, y) : 0;
            if (c > 1) ycredit(a, q, (unsigned long long)(c - 1));
            item_add(item[warp], k, c > 1 ? c - 1 : 0, live);
        };
        if (du <= SMALL_PCAP) {
            // every warp takes an equal range of the vertex's wedges
            const long long W = wedge_prefix<THREADS>(a, u, bu, du, pre, wsum);
            const long long w_lo = W * warp / NW, w_hi = W * (warp + 1) / NW;
            walk_range(a, u, bu, du, pre, w_lo, w_hi, count, [&](int32_t) {});
            __syncthreads();
            if (CREDIT) {
                walk_range(a, u, bu, du, pre, w_lo, w_hi, credit, [&](int32_t j) {
                    __syncwarp();
                    const unsigned long long sv = item[warp][lane];
                    if (sv) { ycredit(a, bu + j, sv); item[warp][lane] = 0; }
                    __syncwarp();
                });
                __syncthreads();
            }
        } else {
            warp_wedges(u, du, bu, warp * WARP, du, NW * WARP, a.rp, a.ci, a.nd, count, [&](int32_t) {});
            __syncthreads();
            if (CREDIT) {
                warp_wedges(u, du, bu, warp * WARP, du, NW * WARP, a.rp, a.ci, a.nd, credit,
                    [&](int32_t it) {
                        __syncwarp();
                        const unsigned long long sv = item[warp][lane];
                        if (sv) { ycredit(a, bu + it + lane, sv); item[warp][lane] = 0; }
                        __syncwarp();
                    });
                __syncthreads();
            }
        }
        const int32_t nt = ntouched;
        for (int32_t i = threadIdx.x; i < nt; i += THREADS) {
            const int32_t h = touched[i];
            keys[h] = -1; vals[h] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) ntouched = 0;
        __syncthreads();
    }
    if (!CREDIT) {
        c4 = warp_sum(c4);
        if (lane == 0) add_u128(a.sums + 2 * (S_NUM + X_C4), 4 * c4);
    }
}

// Medium tier: one vertex per CTA at a time.  Its counters live in the
// CTA's own open-addressing table in global memory, sized to the vertex: at
// least 1.5 W(u) slots (a multiple of 1024), and a vertex has at most W(u)
// distinct opposite nodes, so every insertion finds a slot and the load
// stays below 2/3 (about 0.37 on power-law graphs, where the distinct nodes
// are about half the wedges).  Tight sizing keeps the tables of all CTAs
// together small enough for L2 (measured: 1.5 W against the next power of
// two of 2 W, R-MAT 22 112 -> 95 ms, Chung-Lu 1M unchanged); the table is
// reset after each vertex.  A
// key's home slot is its 32-bit hash scaled to the table (multiply-high),
// then linear probing.  An entry is (y << 32) | count, all ones when empty.
constexpr unsigned long long MH_EMPTY = ~0ull;
constexpr unsigned long long MH_KEY = 0xffffffff00000000ull;

__device__ __forceinline__ uint32_t mh_cap(int64_t w, int64_t mcap) {
    int64_t c = (w + w / 2 + 1024) & ~1023ll;
    return (uint32_t)(c < mcap ? c : mcap);
}

__device__ __forceinline__ uint32_t mh_home(int32_t y, uint32_t cap) {
    return (uint32_t)(((unsigned long long)hash32((uint32_t)y) * cap) >> 32);
}

// cnt[y] += 1; returns the previous count (0xffffffff: table full)
__device__ __forceinline__ uint32_t mh_add(unsigned long long *t, uint32_t cap, int32_t y) {
    const unsigned long long key = (unsigned long long)(uint32_t)y << 32;
    uint32_t h = mh_home(y, cap);
    for (uint32_t probe = 0; probe < cap; probe++) {
        unsigned long long w = __ldcg(t + h);
        if (w == MH_EMPTY) {
            w = atomicCAS(t + h, MH_EMPTY, key | 1ull);
            if (w == MH_EMPTY) return 0;
        }
        if ((w & MH_KEY) == key) return (uint32_t)atomicAdd(t + h, 1ull);
        h = h + 1 < cap ? h + 1 : 0;
    }
    return 0xffffffffu;
}

__device__ __forceinline__ uint32_t mh_get(const unsigned long long *t, uint32_t cap, int32_t y) {
    const unsigned long long key = (unsigned long long)(uint32_t)y << 32;
    uint32_t h = mh_home(y, cap);
    for (uint32_t probe = 0; probe < cap; probe++) {
        const unsigned long long w = __ldcg(t + h);
        if ((w & MH_KEY) == key) return (uint32_t)w;
        if (w == MH_EMPTY) return 0;
        h = h + 1 < cap ? h + 1 : 0;
    }
    return 0;
}

// mh_add for two keys (each only if its ok): both home slots are loaded
// together and, in the common cases (the key is there, or the slot is
// empty), both atomics are issued before either result is used; any other
// case finishes through mh_add.  o0, o1: the previous counts as in mh_add.
__device__ __forceinline__ void mh_add2(unsigned long long *t, uint32_t cap, int32_t y0, bool ok0, int32_t y1,
                                        bool ok1, uint32_t &o0, uint32_t &o1) {
    const unsigned long long k0 = (unsigned long long)(uint32_t)y0 << 32, k1 = (unsigned long long)(uint32_t)y1 << 32;
    const uint32_t h0 = mh_home(y0, cap), h1 = mh_home(y1, cap);
    const unsigned long long w0 = ok0 ? __ldcg(t + h0) : 0, w1 = ok1 ? __ldcg(t + h1) : 0;
    unsigned long long r0 = 0, r1 = 0;
    int m0 = 0, m1 = 0;                       // 1: insertion tried, 2: increment issued
    if (ok0) {
        if (w0 == MH_EMPTY) { r0 = atomicCAS(t + h0, MH_EMPTY, k0 | 1ull); m0 = 1; }
        else if ((w0 & MH_KEY) == k0) { r0 = atomicAdd(t + h0, 1ull); m0 = 2; }
    }
    if (ok1) {
        if (w1 == MH_EMPTY) { r1 = atomicCAS(t + h1, MH_EMPTY, k1 | 1ull); m1 = 1; }
        else if ((w1 & MH_KEY) == k1) { r1 = atomicAdd(t + h1, 1ull); m1 = 2; }
    }
    o0 = 0;
    o1 = 0;
    if (ok0) o0 = m0 == 2 ? (uint32_t)r0 : (m0 == 1 && r0 == MH_EMPTY) ? 0u : mh_add(t, cap, y0);
    if (ok1) o1 = m1 == 2 ? (uint32_t)r1 : (m1 == 1 && r1 == MH_EMPTY) ? 0u : mh_add(t, cap, y1);
}

// mh_get for two keys, both home slots loaded together
__device__ __forceinline__ void mh_get2(const unsigned long long *t, uint32_t cap, int32_t y0, bool ok0, int32_t y1,
                                        bool ok1, uint32_t &c0, uint32_t &c1) {
    const unsigned long long k0 = (unsigned long long)(uint32_t)y0 << 32, k1 = (unsigned long long)(uint32_t)y1 << 32;
    const unsigned long long w0 = ok0 ? __ldcg(t + mh_home(y0, cap)) : MH_EMPTY;
    const unsigned long long w1 = ok1 ? __ldcg(t + mh_home(y1, cap)) : MH_EMPTY;
    c0 = (w0 & MH_KEY) == k0 && w0 != MH_EMPTY ? (uint32_t)w0 : w0 == MH_EMPTY ? 0u : mh_get(t, cap, y0);
    c1 = (w1 & MH_KEY) == k1 && w1 != MH_EMPTY ? (uint32_t)w1 : w1 == MH_EMPTY ? 0u : mh_get(t, cap, y1);
}

// Wedge prefix of the medium tier in shared memory: vertices of larger
// degree walk their neighbours 32 at a time per warp instead.
constexpr int MED_PCAP = 8192;

template <int THREADS, bool CREDIT>
__global__ void __launch_bounds__(THREADS, 2048 / THREADS)
k_cycles_medium(CycleArgs a) {
    constexpr int NW = THREADS / 32;
    __shared__ unsigned long long item[NW][WARP];
    __shared__ long long wsum[NW];
    __shared__ int32_t next;
    extern __shared__ long long pre[];          // MED_PCAP + 1 entries
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const int32_t nv = a.counters[C_MEDIUM];
    unsigned long long *tab = a.mtab + (int64_t)blockIdx.x * a.mcap;
    if (threadIdx.x == 0) next = atomicAdd(a.counters + C_DYN, 1);
    item[warp][lane] = 0;
    unsigned long long c4 = 0;
    bool full = false;
    __syncthreads();
    while (true) {
        const int32_t idx = next;
        if (idx >= nv) break;
        const int32_t u = a.mlist[idx];
        const int32_t bu = a.rp[u], du = a.rp[u + 1] - bu;
        const uint32_t cap = mh_cap(a.west[u], a.mcap);
        // count: cnt[y] += 1 (the values returned add up to C(cnt[y], 2));
        // credit: cnt[y] - 1 to (v, y) and, summed per neighbour, to (u, v)
        auto count = [&](int k, int32_t q, int32_t y, bool ok, bool live) {
            if (!ok) return;
            const uint32_t old = mh_add(tab, cap, y);
            if (old == 0xffffffffu) full = true;
            else if (!CREDIT) c4 += old;
        };
        auto credit = [&](int k, int32_t q, int32_t y, bool ok, bool live) {
            const uint32_t c = ok ? mh_get(tab, cap, y) : 0;
            if (c > 1) ycredit(a, q, (unsigned long long)(c - 1));
            item_add(item[warp], k, c > 1 ? c - 1 : 0, live);
        };
        // the same for two wedges per lane, their probes in flight together
        auto count2 = [&](int k0, int32_t q0, int32_t y0, bool ok0, bool live0,
                          int k1, int32_t q1, int32_t y1, bool ok1, bool live1) {
            uint32_t o0, o1;
            mh_add2(tab, cap, y0, ok0, y1, ok1, o0, o1);
            if ((ok0 && o0 == 0xffffffffu) || (ok1 && o1 == 0xffffffffu)) full = true;
            else if (!CREDIT) c4 += (unsigned long long)o0 + o1;
        };
        auto credit2 = [&](int k0, int32_t q0, int32_t y0, bool ok0, bool live0,
                           int k1, int32_t q1, int32_t y1, bool ok1, bool live1) {
            uint32_t c0, c1;
            mh_get2(tab, cap, y0, ok0, y1, ok1, c0, c1);
            if (c0 > 1) ycredit(a, q0, (unsigned long long)(c0 - 1));
            if (c1 > 1) ycredit(a, q1, (unsigned long long)(c1 - 1));
            item_add(item[warp], k0, c0 > 1 ? c0 - 1 : 0, live0);
            item_add(item[warp], k1, c1 > 1 ? c1 - 1 : 0, live1);
        };
        if (du <= MED_PCAP) {
            // every warp takes an equal range of the vertex's wedges
            const long long W = wedge_prefix<THREADS>(a, u, bu, du, pre, wsum);
            for (int ph = 0; ph < (CREDIT ? 2 : 1); ph++) {
                const long long w_lo = W * warp / NW, w_hi = W * (warp + 1) / NW;
                if (ph == 0) {
                    walk_range2(a, u, bu, du, pre, w_lo, w_hi, count2, [&](int32_t) {});
                } else {
                    walk_range2(a, u, bu, du, pre, w_lo, w_hi, credit2, [&](int32_t j) {
                        __syncwarp();
                        const unsigned long long sv = item[warp][lane];
                        if (sv) { ycredit(a, bu + j, sv); item[warp][lane] = 0; }
                        __syncwarp();
                    });
                }
                __syncthreads();
            }
        } else {
            warp_wedges(u, du, bu, warp * WARP, du, NW * WARP, a.rp, a.ci, a.nd, count, [&](int32_t) {});
            __syncthreads();
            if (CREDIT) {
                warp_wedges(u, du, bu, warp * WARP, du, NW * WARP, a.rp, a.ci, a.nd, credit,
                    [&](int32_t it) {
                        __syncwarp();
                        const unsigned long long sv = item[warp][lane];
                        if (sv) { ycredit(a, bu + it + lane, sv); item[warp][lane] = 0; }
                        __syncwarp();
                    });
                __syncthreads();
            }
        }
        ulonglong2 *t2 = reinterpret_cast<ulonglong2 *>(tab);
        for (uint32_t i = threadIdx.x; i < cap / 2; i += THREADS) t2[i] = make_ulonglong2(MH_EMPTY, MH_EMPTY);
        __syncthreads();
        if (threadIdx.x == 0) next = atomicAdd(a.counters + C_DYN, 1);
        __syncthreads();
    }
    if (full) atomicOr(a.status, ERR_CAPACITY);
    if (!CREDIT) {
        c4 = warp_sum(c4);
        if (lane == 0) add_u128(a.sums + 2 * (S_NUM + X_C4), 4 * c4);
    }
}

// Medium tier, vertices of at least 2^MED_CL_LOG2 wedges: a cluster of MCL
// CTAs takes one vertex at a time and shares one open-addressing table in
// global memory, so that only one table per cluster is live (a few tens of
// MB for the whole GPU, which stay in L2, where one table per CTA did not).
// The vertex's wedges are split evenly over all warps of the cluster; the
// cluster's hardware barrier separates counting, crediting and the reset
// (each CTA resets its share of the table).  The next vertex's index is
// fetched by CTA 0 and read by the others from its shared memory.
constexpr int MCL = 8;
constexpr int MED_CL_LOG2 = 16;

template <bool CREDIT>
__global__ void __cluster_dims__(MCL, 1, 1) __launch_bounds__(1024, 2)
k_cycles_medium_cl(CycleArgs a, int32_t nv_big) {
    constexpr int THREADS = 1024, NW = THREADS / 32;
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    __shared__ unsigned long long item[NW][WARP];
    __shared__ long long wsum[NW];
    __shared__ int32_t next[2];
    extern __shared__ long long pre[];          // MED_PCAP + 1 entries
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    unsigned long long *tab = a.mtab + (int64_t)(blockIdx.x / MCL) * a.mcap;
    if (rank == 0 && threadIdx.x == 0) next[0] = atomicAdd(a.counters + C_DYN2, 1);
    item[warp][lane] = 0;
    unsigned long long c4 = 0;
    bool full = false;
    const int gw = rank * NW + warp;            // warp index within the cluster
    constexpr int GW = MCL * NW;
    cl.sync();
    for (int it = 0;; it++) {
        const int32_t idx = *cl.map_shared_rank(&next[it & 1], 0);
        if (idx >= nv_big) break;
        const int32_t u = a.mlist[idx];
        const int32_t bu = a.rp[u], du = a.rp[u + 1] - bu;
        const uint32_t cap = mh_cap(a.west[u], a.mcap);
        auto count = [&](int k, int32_t q, int32_t y, bool ok, bool live) {
            if (!ok) return;
            const uint32_t old = mh_add(tab, cap, y);
            if (old == 0xffffffffu) full = true;
            else if (!CREDIT) c4 += old;
        };
        auto credit = [&](int k, int32_t q, int32_t y, bool ok, bool live) {
            const uint32_t c = ok ? mh_get(tab, cap, y) : 0;
            if (c > 1) ycredit(a, q, (unsigned long long)(c - 1));
            item_add(item[warp], k, c > 1 ? c - 1 : 0, live);
        };
        // the same for two wedges per lane, their probes in flight together
        auto count2 = [&](int k0, int32_t q0, int32_t y0, bool ok0, bool live0,
                          int k1, int32_t q1, int32_t y1, bool ok1, bool live1) {
            uint32_t o0, o1;
            mh_add2(tab, cap, y0, ok0, y1, ok1, o0, o1);
            if ((ok0 && o0 == 0xffffffffu) || (ok1 && o1 == 0xffffffffu)) full = true;
            else if (!CREDIT) c4 += (unsigned long long)o0 + o1;
        };
        auto credit2 = [&](int k0, int32_t q0, int32_t y0, bool ok0, bool live0,
                           int k1, int32_t q1, int32_t y1, bool ok1, bool live1) {
            uint32_t c0, c1;
            mh_get2(tab, cap, y0, ok0, y1, ok1, c0, c1);
            if (c0 > 1) ycredit(a, q0, (unsigned long long)(c0 - 1));
            if (c1 > 1) ycredit(a, q1, (unsigned long long)(c1 - 1));
            item_add(item[warp], k0, c0 > 1 ? c0 - 1 : 0, live0);
            item_add(item[warp], k1, c1 > 1 ? c1 - 1 : 0, live1);
        };
        if (du <= MED_PCAP) {
            const long long W = wedge_prefix<THREADS>(a, u, bu, du, pre, wsum);
            const long long w_lo = W * gw / GW, w_hi = W * (gw + 1) / GW;
            walk_range2(a, u, bu, du, pre, w_lo, w_hi, count2, [&](int32_t) {});
            cl.sync();
            if (CREDIT) {
                walk_range2(a, u, bu, du, pre, w_lo, w_hi, credit2, [&](int32_t j) {
                    __syncwarp();
                    const unsigned long long sv = item[warp][lane];
                    if (sv) { ycredit(a, bu + j, sv); item[warp][lane] = 0; }
                    __syncwarp();
                });
                cl.sync();
            }
        } else {
            warp_wedges(u, du, bu, gw * WARP, du, GW * WARP, a.rp, a.ci, a.nd, count, [&](int32_t) {});
            cl.sync();
            if (CREDIT) {
                warp_wedges(u, du, bu, gw * WARP, du, GW * WARP, a.rp, a.ci, a.nd, credit,
                    [&](int32_t i0) {
                        __syncwarp();
                        const unsigned long long sv = item[warp][lane];
                        if (sv) { ycredit(a, bu + i0 + lane, sv); item[warp][lane] = 0; }
                        __syncwarp();
                    });
                cl.sync();
            }
        }
        if (rank == 0 && threadIdx.x == 0) next[(it + 1) & 1] = atomicAdd(a.counters + C_DYN2, 1);
        ulonglong2 *t2 = reinterpret_cast<ulonglong2 *>(tab);
        const uint32_t h0 = (cap / 2) * rank / MCL, h1 = (cap / 2) * (rank + 1) / MCL;
        for (uint32_t i = h0 + threadIdx.x; i < h1; i += THREADS) t2[i] = make_ulonglong2(MH_EMPTY, MH_EMPTY);
        cl.sync();
    }
    // CTA 0's shared memory was read by the others: no CTA leaves before all
    // have read the last index
    cl.sync();
    if (full) atomicOr(a.status, ERR_CAPACITY);
    if (!CREDIT) {
        c4 = warp_sum(c4);
        if (lane == 0) add_u128(a.sums + 2 * (S_NUM + X_C4), 4 * c4);
    }
}

// Hub tier preparation, once for all hubs: hoff = exclusive prefix of the
// hubs' degrees (the hubs' rows concatenated form one flat list), hlen[j] =
// wedges of flat neighbour j (d_v if v ranks below its hub, else 0), and
// its exclusive prefix hpre (hpre[F] = all hub wedges).  A batch of hubs
// [hub0, hub0 + nhub) owns flat [hoff[hub0], hoff[hub0 + nhub]).
__global__ void k_hub_degrees(int32_t nh, const int32_t *__restrict__ hubs, const int32_t *__restrict__ rp,
                              int64_t *deg) {
    for (int32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
        const int32_t u = hubs[h];
        deg[h] = rp[u + 1] - rp[u];
    }
}

__global__ void k_hub_lengths(CycleArgs a, int32_t nh) {
    const int64_t total = a.hoff[nh];
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total; j += (int64_t)gridDim.x * blockDim.x) {
        // hub of flat entry j: the last h with hoff[h] <= j
        int32_t lo = 0, hi = nh - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (a.hoff[mid] <= j) lo = mid; else hi = mid - 1;
        }
        const int32_t u = a.hubs[lo];
        const int32_t bu = a.rp[u], du = a.rp[u + 1] - bu;
        const int32_t i = (int32_t)(j - a.hoff[lo]);
        const int32_t v = a.ci[bu + i], dv = a.nd[bu + i];
        a.hlen[j] = precedes(dv, v, du, u) ? dv : 0;
    }
}

// After the prefix, hlen holds each flat entry's row instead: the CSR start
// of the neighbour's list (low word) and the hub's index in the hub list
// (high word), so that the walks read one word per neighbour.
__global__ void k_hub_rows(CycleArgs a, int32_t nh) {
    const int64_t total = a.hoff[nh];
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total; j += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = nh - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (a.hoff[mid] <= j) lo = mid; else hi = mid - 1;
        }
        const int32_t u = a.hubs[lo];
        const int32_t v = a.ci[a.rp[u] + (int32_t)(j - a.hoff[lo])];
        a.hlen[j] = (int64_t)(uint32_t)a.rp[v] | ((int64_t)lo << 32);
    }
}

constexpr int HUB_BATCH_MAX = 16;

// G consecutive 32-wedge groups of one neighbour's list in hub u's walk,
// wedge i of this lane at ci[q0 + 32 i]: count them, or credit cnt - 1 to
// (v, y) and add it to the lane's running credit of (u, v).
template <int PH, int G>
__device__ __forceinline__ void hub_groups(const CycleArgs &a, int32_t q0, int32_t u, int32_t du, uint32_t *tab,
                                           unsigned long long &acc) {
    int32_t y[G], dy[G];
#pragma unroll
    for (int i = 0; i < G; i++) { y[i] = a.ci[q0 + i * WARP]; dy[i] = a.nd[q0 + i * WARP]; }
    if (PH == 0) {
#pragma unroll
        for (int i = 0; i < G; i++)
            if (precedes(dy[i], y[i], du, u)) atomicAdd(tab + y[i], 1u);
    } else {
        uint32_t c[G];
#pragma unroll
        for (int i = 0; i < G; i++) c[i] = precedes(dy[i], y[i], du, u) ? __ldcg(tab + y[i]) : 0;
#pragma unroll
        for (int i = 0; i < G; i++)
            if (c[i] > 1) {
                ycredit(a, q0 + i * WARP, (unsigned long long)(c[i] - 1));
                acc += c[i] - 1;
            }
    }
}

// Hub tier, phase PH (0 count, 1 credit): the batch's wedges form one flat
// space (hub rows concatenated, each neighbour contributing its list); every
// warp of the grid takes an equal range of it, finds the first neighbour of
// its range by 32-way splits of the prefix, and walks the neighbours 32 at a
// time, clipping the lists that straddle the range ends.  A 32-wedge group
// that lies in one neighbour's list (most of them: hub neighbours have long
// lists) is handled uniformly, its credits to (u, v) summed per lane until
// the walk leaves the list; a group spanning several lists maps each lane to
// its list by a search over the lanes' offsets.  Hub h counts into table h.
// (Keeping two or four groups' loads in flight was measured slower: the
// count phase is bound by the table updates in L2, not by load latency.)
template <int PH>
__global__ void __launch_bounds__(256, 8)
k_cycles_hub(CycleArgs a) {
    __shared__ unsigned long long item[8][WARP];
    __shared__ int32_t hub_u[HUB_BATCH_MAX], hub_d[HUB_BATCH_MAX], hub_b[HUB_BATCH_MAX];
    __shared__ int64_t hub_f[HUB_BATCH_MAX];
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    if (threadIdx.x < a.nhub) {
        const int32_t u = a.hubs[a.hub0 + threadIdx.x];
        hub_u[threadIdx.x] = u;
        hub_b[threadIdx.x] = a.rp[u];
        hub_d[threadIdx.x] = a.rp[u + 1] - a.rp[u];
        hub_f[threadIdx.x] = a.hoff[a.hub0 + threadIdx.x];
    }
    item[warp][lane] = 0;
    __syncthreads();
    const int64_t *hpre = a.hpre;
    const int64_t f0 = a.hoff[a.hub0], flat = a.hoff[a.hub0 + a.nhub];
    const int64_t wbase = hpre[f0], wtot = hpre[flat] - wbase;
    // every warp of the grid takes an equal share of the batch's wedges
    const int64_t gw = global_warp(), gwn = num_warps();
    const int64_t w_lo = wbase + wtot * gw / gwn;
    const int64_t w_hi = wbase + wtot * (gw + 1) / gwn;
    if (w_lo >= w_hi) return;
    // largest j in [f0, flat) with hpre[j] <= w_lo (hpre[flat] > w_lo): each
    // round probes 32 evenly spaced entries of [lo, hi] and keeps one gap
    int64_t lo = f0, hi = flat - 1;
    while (lo < hi) {
        const int64_t step = (hi - lo + WARP - 1) / WARP;
        const int64_t p = lo + (int64_t)(lane + 1) * step;
        const bool le = p <= hi && hpre[p] <= w_lo;
        const int64_t nlo = lo + (int64_t)__popc(__ballot_sync(FULL, le)) * step;
        hi = min(hi, nlo + step - 1);
        lo = nlo;
    }
    for (int64_t j0 = lo; j0 < flat && hpre[j0] < w_hi; j0 += WARP) {
        // lane l: neighbour j0 + l, its wedges clipped to [w_lo, w_hi)
        const int64_t j = j0 + lane;
        int32_t len = 0, start = 0, h = 0, slot_uv = -1;
        if (j < flat) {
            const int64_t p0 = hpre[j], p1 = hpre[j + 1];
            const int64_t s0 = max(p0, w_lo), e0 = min(p1, w_hi);
            if (e0 > s0) {
                const int64_t row = a.hlen[j];
                h = (int32_t)(row >> 32) - a.hub0;
                len = (int32_t)(e0 - s0);
                start = (int32_t)row + (int32_t)(s0 - p0);
                slot_uv = hub_b[h] + (int32_t)(j - hub_f[h]);
            }
        }
        const int32_t incl = warp_incl_scan(len);
        const int32_t total = __shfl_sync(FULL, incl, 31);
        const int32_t excl = incl - len;
        const int32_t base = start - excl;     // wedge w of lane k's list: ci[base_k + w]
        int32_t kc = 0;                        // the lane whose list holds wedge w0
        unsigned long long acc = 0;            // this lane's credits to (u, v) of lane kc
        bool held = false;
        for (int32_t w0 = 0; w0 < total;) {
            int32_t kend = __shfl_sync(FULL, incl, kc);
            while (kend <= w0 && kc < WARP - 1) {
                if (PH == 1 && held) {
                    const unsigned long long s = warp_sum(acc);
                    if (lane == 0 && s) atomicAdd(item[warp] + kc, s);
                    acc = 0;
                    held = false;
                }
                kc++;
                kend = __shfl_sync(FULL, incl, kc);
            }
            if (w0 + WARP <= kend) {
                // the group lies in lane kc's list
                const int32_t q0 = __shfl_sync(FULL, base, kc) + w0 + lane;
                const int32_t kh = __shfl_sync(FULL, h, kc);
                uint32_t *tab = a.tables + (int64_t)kh * a.n;
                hub_groups<PH, 1>(a, q0, hub_u[kh], hub_d[kh], tab, acc);
                w0 += WARP;
                held = true;
                continue;
            }
            // the group spans several lists: lane -> list by search
            const int32_t w = w0 + lane;
            int32_t k = 0;
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                const int32_t e = __shfl_sync(FULL, excl, k + s);
                if (e <= w) k += s;
            }
            const int32_t kq = __shfl_sync(FULL, base, k);
            const int32_t kh = __shfl_sync(FULL, h, k);
            const bool live = w < total;
            bool ok = false;
            int32_t q = 0, y = 0;
            if (live) {
                q = kq + w;
                y = a.ci[q];
                ok = precedes(a.nd[q], y, hub_d[kh], hub_u[kh]);
            }
            uint32_t *tab = a.tables + (int64_t)kh * a.n;
            if (PH == 0) {
                if (ok) atomicAdd(tab + y, 1u);      // result unused: a reduction
            } else {
                const uint32_t c = ok ? __ldcg(tab + y) : 0;
                if (c > 1) ycredit(a, q, (unsigned long long)(c - 1));
                item_add(item[warp], k, c > 1 ? c - 1 : 0, live);
            }
            w0 += WARP;
        }
        if (PH == 1) {
            if (held) {
                const unsigned long long s = warp_sum(acc);
                if (lane == 0 && s) atomicAdd(item[warp] + kc, s);
            }
            __syncwarp();
            const unsigned long long s = item[warp][lane];
            if (s) { ycredit(a, slot_uv, s); item[warp][lane] = 0; }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// Hub tier, global counts, pull form (heaviest hubs).  For a batch of up to
// 64 hubs u_i in decreasing rank, the 4-cycles with top node u_i and
// opposite node y number C(cnt_i[y], 2), cnt_i[y] = #{v in N(y): v below
// u_i and adjacent to it} (y below u_i).  Instead of one counter update per
// wedge, every node v carries the bits M[v] of the batch hubs above it that
// it is adjacent to, and each y sums the masks of its neighbours into
// bit-plane counters: plane a holds bit a of all 64 counters, so adding a
// mask is a ripple of ANDs and XORs.  Then
//   sum_i C(cnt_i, 2) = (sum_{a,b} 2^(a+b) |P_a & P_b & V| - sum_a 2^a |P_a & V|) / 2
// with V the hubs ranked above y.  No tables, no atomics: one read of
// N(y) and its neighbours' masks per y and batch.
// ---------------------------------------------------------------------------
constexpr int PULL_MAX = 64;          // hubs per pull batch (bits of a mask)
constexpr int PULL_WARP_DEG = 64;     // d_y >= this: a warp per y, else a thread
constexpr int PULL_TPLANES = 7;       // thread path: counters <= 63

// mark (set) or clear the masks of the lower neighbours of hubs [h0, h0 + nb)
template <bool SET>
__global__ void k_pull_mark(CycleArgs a, int32_t h0, int32_t nb, unsigned long long *mask) {
    const int64_t f0 = a.hoff[h0], f1 = a.hoff[h0 + nb];
    for (int64_t j = f0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < f1; j += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = h0, hi = h0 + nb - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (a.hoff[mid] <= j) lo = mid; else hi = mid - 1;
        }
        const int32_t u = a.hubs[lo];
        const int32_t bu = a.rp[u], du = a.rp[u + 1] - bu;
        const int32_t p = bu + (int32_t)(j - a.hoff[lo]);
        const int32_t v = a.ci[p];
        if (!SET) mask[v] = 0;
        else if (precedes(a.nd[p], v, du, u)) atomicOr(mask + v, 1ull << (lo - h0));
    }
}

// carry-save adder: a + b + c = l + 2 h, in each of the 64 bit positions
__device__ __forceinline__ void csa(unsigned long long &h, unsigned long long &l, unsigned long long a,
                                    unsigned long long b, unsigned long long c) {
    const unsigned long long u = a ^ b;
    h = (a & b) | (u & c);
    l = u ^ c;
}

// add eight masks into the lowest LA planes (Harley-Seal): the masks pass
// through carry-save adders into the ones, twos and fours planes, and only
// the eights carry ripples through the planes above; about 5.5 logic
// operations a mask where a ripple of each mask costs 2 LA.  The caller
// guarantees that no counter passes 2^LA - 1.
template <int LA, int L>
__device__ __forceinline__ void plane_add8(unsigned long long (&P)[L], const unsigned long long (&m)[8]) {
    static_assert(LA >= 4 && LA <= L, "active planes");
    unsigned long long t2a, t2b, t4a, t4b, t8;
    csa(t2a, P[0], P[0], m[0], m[1]);
    csa(t2b, P[0], P[0], m[2], m[3]);
    csa(t4a, P[1], P[1], t2a, t2b);
    csa(t2a, P[0], P[0], m[4], m[5]);
    csa(t2b, P[0], P[0], m[6], m[7]);
    csa(t4b, P[1], P[1], t2a, t2b);
    csa(t8, P[2], P[2], t4a, t4b);
#pragma unroll
    for (int b = 3; b < LA; b++) {
        const unsigned long long c = P[b] & t8;
        P[b] ^= t8;
        t8 = c;
    }
}

// sum over the hubs of V of C(cnt, 2), the counters held as L bit planes
template <int L>
__device__ __forceinline__ unsigned long long plane_pairs(const unsigned long long (&P)[L], unsigned long long V) {
    unsigned long long s1 = 0, s2 = 0;
#pragma unroll
    for (int a0 = 0; a0 < L; a0++) {
        const unsigned long long pa = P[a0] & V;
        s1 += (unsigned long long)__popcll(pa) << a0;
        s2 += (unsigned long long)__popcll(pa) << (2 * a0);
#pragma unroll
        for (int b = 0; b < L; b++)
            if (b > a0) s2 += (unsigned long long)__popcll(pa & P[b]) << (a0 + b + 1);
    }
    return (s2 - s1) >> 1;
}

// counter i out of L bit planes
template <int L>
__device__ __forceinline__ uint32_t plane_counter(const unsigned long long (&P)[L], int i) {
    uint32_t x = 0;
#pragma unroll
    for (int a0 = 0; a0 < L; a0++) x |= (uint32_t)((P[a0] >> i) & 1ull) << a0;
    return x;
}

// the hubs of the batch ranked above y: the first k (hubs in decreasing rank)
__device__ __forceinline__ unsigned long long hubs_above(int32_t dy, int32_t y, const int32_t *hd,
                                                         const int32_t *hu, int32_t nb) {
    int32_t lo = 0, hi = nb;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (precedes(dy, y, hd[mid], hu[mid])) lo = mid + 1; else hi = mid;
    }
    return lo >= 64 ? ~0ull : ((1ull << lo) - 1);
}

__device__ __forceinline__ void pull_hubs_smem(const CycleArgs &a, int32_t h0, int32_t nb, int32_t *hu, int32_t *hd) {
    if (threadIdx.x < nb) {
        const int32_t u = a.hubs[h0 + threadIdx.x];
        hu[threadIdx.x] = u;
        hd[threadIdx.x] = a.rp[u + 1] - a.rp[u];
    }
    __syncthreads();
}

// A thread per node y of degree < PULL_WARP_DEG; the neighbours' masks are
// fetched eight at a time (eight loads in flight per thread) and added by
// carry-save adders.
// TAB (per-edge credits): instead of summing C(cnt, 2), write the counters
// of at least 2 of the hubs above y into the batch's dense tables (zero at
// rest), which the credit pass reads as the push form's counts.
template <bool TAB>
__global__ void __launch_bounds__(256)
k_pull_thread(CycleArgs a, int32_t h0, int32_t nb, const unsigned long long *__restrict__ mask) {
    __shared__ int32_t hu[PULL_MAX], hd[PULL_MAX];
    pull_hubs_smem(a, h0, nb, hu, hd);
    unsigned long long c4 = 0;
    for (int32_t y = blockIdx.x * blockDim.x + threadIdx.x; y < a.n; y += gridDim.x * blockDim.x) {
        const int32_t b = __ldg(a.rp + y), e = __ldg(a.rp + y + 1), d = e - b;
        if (d < 2 || d >= PULL_WARP_DEG) continue;
        unsigned long long P[PULL_TPLANES] = {0, 0, 0, 0, 0, 0, 0};
        for (int32_t p = b; p < e; p += 8) {
            // eight masks at a time (zero past the end), their loads in flight together
            int32_t v[8];
            unsigned long long m[8];
#pragma unroll
            for (int j = 0; j < 8; j++) v[j] = p + j < e ? __ldg(a.ci + p + j) : -1;
#pragma unroll
            for (int j = 0; j < 8; j++) m[j] = v[j] >= 0 ? mask[v[j]] : 0ull;
            plane_add8<PULL_TPLANES, PULL_TPLANES>(P, m);
        }
        unsigned long long any = 0;
#pragma unroll
        for (int i = 1; i < PULL_TPLANES; i++) any |= P[i];
        if (!any) continue;                   // every counter <= 1
        const unsigned long long V = hubs_above(d, y, hd, hu, nb);
        if constexpr (TAB) {
            for (unsigned long long mm = any & V; mm; mm &= mm - 1) {
                const int i = __ffsll((long long)mm) - 1;
                a.tables[(int64_t)i * a.n + y] = plane_counter<PULL_TPLANES>(P, i);
            }
        } else {
            c4 += plane_pairs<PULL_TPLANES>(P, V);
        }
    }
    if constexpr (!TAB) {
        c4 = warp_sum(c4);
        if (lane_id() == 0 && c4) add_u128(a.sums + 2 * (S_NUM + X_C4), 4 * c4);
    }
}

// Nodes of degree >= PULL_WARP_DEG are split into chunks of at most
// PULL_CHUNK neighbours, one warp per chunk (the list of chunks is built
// once per count: the degrees do not change between batches).  A node of
// one chunk gets its C(cnt, 2) sum from the chunk's planes; a node of
// several chunks (a "heavy" node) adds each chunk's per-hub counters into
// 64 counters of its own, summed by k_pull_heavy after all chunks.
constexpr int PULL_CHUNK = 1024;
constexpr int PULL_CPLANES = 11;      // a chunk's counters are <= 1024
constexpr int PULL_LPLANES = 6;       // a lane's share of a chunk: <= 32 masks

struct PullItem { int32_t y, chunk, heavy; };

__global__ void k_pull_items(int32_t n, const int32_t *__restrict__ rp, PullItem *items, int32_t *heavy_y,
                             int32_t *counts) {
    for (int32_t y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) {
        const int32_t d = rp[y + 1] - rp[y];
        if (d < PULL_WARP_DEG) continue;
        const int32_t nch = (d + PULL_CHUNK - 1) / PULL_CHUNK;
        const int32_t pos = atomicAdd(counts, nch);
        int32_t hv = -1;
        if (nch > 1) { hv = atomicAdd(counts + 1, 1); heavy_y[hv] = y; }
        for (int32_t c = 0; c < nch; c++) items[pos + c] = PullItem{y, c, hv};
    }
}

template <bool TAB>
__global__ void __launch_bounds__(256)
k_pull_warp(CycleArgs a, int32_t h0, int32_t nb, const unsigned long long *__restrict__ mask,
            const PullItem *__restrict__ items, int32_t nitems, uint32_t *heavy_cnt) {
    __shared__ int32_t hu[PULL_MAX], hd[PULL_MAX];
    pull_hubs_smem(a, h0, nb, hu, hd);
    const int lane = lane_id();
    unsigned long long c4 = 0;
    for (int64_t it = global_warp(); it < nitems; it += num_warps()) {
        const PullItem t = items[it];
        const int32_t b0 = __ldg(a.rp + t.y), d = __ldg(a.rp + t.y + 1) - b0;
        const int32_t b = b0 + t.chunk * PULL_CHUNK, e = min(b + PULL_CHUNK, b0 + d);
        unsigned long long P[PULL_CPLANES];
#pragma unroll
        for (int i = 0; i < PULL_CPLANES; i++) P[i] = 0;
        for (int32_t p = b + lane; p < e; p += 8 * WARP) {
            // this lane's next eight masks (zero past the end), loads in flight together
            int32_t v[8];
            unsigned long long m[8];
#pragma unroll
            for (int j = 0; j < 8; j++) v[j] = p + j * WARP < e ? __ldg(a.ci + p + j * WARP) : -1;
#pragma unroll
            for (int j = 0; j < 8; j++) m[j] = v[j] >= 0 ? mask[v[j]] : 0ull;
            plane_add8<PULL_LPLANES, PULL_CPLANES>(P, m);
        }
        unsigned long long any = 0;
#pragma unroll
        for (int i = 0; i < PULL_LPLANES; i++) any |= P[i];
        if (!__any_sync(FULL, any != 0)) continue;      // no neighbour below a batch hub
        // butterfly: every lane ends with the chunk's total (<= 1024 each);
        // after level l the counters need PULL_LPLANES + l + 1 planes
#pragma unroll
        for (int l = 0; l < 5; l++) {
            const int o = 16 >> l;
            unsigned long long c = 0;
#pragma unroll
            for (int i = 0; i < PULL_CPLANES; i++) {
                if (i > PULL_LPLANES + l) break;
                const unsigned long long q = __shfl_xor_sync(FULL, P[i], o);
                const unsigned long long s = P[i] ^ q ^ c;
                c = (P[i] & q) | (c & (P[i] ^ q));
                P[i] = s;
            }
        }
        if (t.heavy < 0) {
            if constexpr (TAB) {
                // lane l: hubs l and l + 32
                const unsigned long long V = hubs_above(d, t.y, hd, hu, nb);
                const uint32_t x0 = plane_counter<PULL_CPLANES>(P, lane);
                const uint32_t x1 = plane_counter<PULL_CPLANES>(P, lane + 32);
                if (x0 > 1 && ((V >> lane) & 1ull)) a.tables[(int64_t)lane * a.n + t.y] = x0;
                if (x1 > 1 && ((V >> (lane + 32)) & 1ull)) a.tables[(int64_t)(lane + 32) * a.n + t.y] = x1;
            } else {
                if (lane == 0) c4 += plane_pairs<PULL_CPLANES>(P, hubs_above(d, t.y, hd, hu, nb));
            }
        } else {
            // lane l: counters of hubs l and l + 32 out of the planes
            uint32_t x0 = 0, x1 = 0;
#pragma unroll
            for (int i = 0; i < PULL_CPLANES; i++) {
                x0 |= (uint32_t)((P[i] >> lane) & 1ull) << i;
                x1 |= (uint32_t)((P[i] >> (lane + 32)) & 1ull) << i;
            }
            uint32_t *hc = heavy_cnt + (int64_t)t.heavy * PULL_MAX;
            if (x0) atomicAdd(hc + lane, x0);
            if (x1) atomicAdd(hc + lane + 32, x1);
        }
    }
    if constexpr (!TAB) {
        c4 = warp_sum(c4);
        if (lane == 0 && c4) add_u128(a.sums + 2 * (S_NUM + X_C4), 4 * c4);
    }
}

// heavy nodes: sum C(cnt, 2) over the hubs above y (TAB: write those of at
// least 2 into the tables), and reset the counters
template <bool TAB>
__global__ void k_pull_heavy(CycleArgs a, int32_t h0, int32_t nb, const int32_t *__restrict__ heavy_y,
                             int32_t nheavy, uint32_t *heavy_cnt) {
    __shared__ int32_t hu[PULL_MAX], hd[PULL_MAX];
    pull_hubs_smem(a, h0, nb, hu, hd);
    const int lane = lane_id();
    unsigned long long c4 = 0;
    for (int64_t k = global_warp(); k < nheavy; k += num_warps()) {
        const int32_t y = heavy_y[k];
        const int32_t d = __ldg(a.rp + y + 1) - __ldg(a.rp + y);
        const unsigned long long V = hubs_above(d, y, hd, hu, nb);
        uint32_t *hc = heavy_cnt + k * PULL_MAX;
        const uint32_t x0 = hc[lane], x1 = hc[lane + 32];
        hc[lane] = 0;
        hc[lane + 32] = 0;
        if constexpr (TAB) {
            if (x0 > 1 && ((V >> lane) & 1ull)) a.tables[(int64_t)lane * a.n + y] = x0;
            if (x1 > 1 && ((V >> (lane + 32)) & 1ull)) a.tables[(int64_t)(lane + 32) * a.n + y] = x1;
        } else {
            unsigned long long t = 0;
            if ((V >> lane) & 1ull) t += c2(x0);
            if ((V >> (lane + 32)) & 1ull) t += c2(x1);
            t = warp_sum(t);
            if (lane == 0) c4 += t;
        }
    }
    if constexpr (!TAB) {
        c4 = warp_sum(c4);
        if (lane == 0 && c4) add_u128(a.sums + 2 * (S_NUM + X_C4), 4 * c4);
    }
}

// per-hub wedge work at the hub boundaries of the flat prefix
__global__ void k_hub_work(int32_t nh, const int64_t *hoff, const int64_t *hpre, int64_t *out) {
    for (int32_t h = blockIdx.x * blockDim.x + threadIdx.x; h <= nh; h += gridDim.x * blockDim.x)
        out[h] = hpre[hoff[h]];
}

// Hub tier, last phase: clear the batch's tables.  Counting globally, a
// full scan reads every counter for the sum of C(cnt, 2) and zeroes the
// nonzero ones (a hub touches a large part of its table); with per-edge
// credits nothing is read and the tables are overwritten with zeros.
template <bool CREDIT>
__global__ void k_cycles_hub_clear(CycleArgs a) {
    unsigned long long c4 = 0;
    const int64_t total = (int64_t)a.nhub * a.n;
    const int64_t total4 = total >> 2;
    uint4 *t4 = reinterpret_cast<uint4 *>(a.tables);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total4; i += (int64_t)gridDim.x * blockDim.x) {
        if (CREDIT) {
            t4[i] = make_uint4(0, 0, 0, 0);
            continue;
        }
        const uint4 v = t4[i];
        if (v.x | v.y | v.z | v.w) {
            c4 += c2(v.x) + c2(v.y) + c2(v.z) + c2(v.w);
            t4[i] = make_uint4(0, 0, 0, 0);
        }
    }
    for (int64_t i = (total4 << 2) + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!CREDIT) c4 += c2(a.tables[i]);
        a.tables[i] = 0;
    }
    if (!CREDIT) {
        c4 = warp_sum(c4);
        if (lane_id() == 0) add_u128(a.sums + 2 * (S_NUM + X_C4), 4 * c4);
    }
}

inline unsigned grid_for(int64_t items, int per_block, int max_blocks) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (unsigned)b;
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// ===========================================================================
// host launchers
// ===========================================================================

static int sms_of(gd_graph *g) { return g->ctx->num_sms > 0 ? g->ctx->num_sms : 152; }


__global__ void k_narrow_i32(const int64_t *in, int32_t *out, int64_t len) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)in[i];
}

// nd, tiers, out-lists.  Reads the counters back (one synchronization).
cudaError_t run_schedule(gd_graph *g, int32_t *counters_host) {
    Workspace &w = g->ws;
    const int sms = sms_of(g);
    const int32_t n = g->n;
    cudaError_t e = cudaMemsetAsync(w.counters, 0, C_NUM * sizeof(int32_t), g->stream);
    if (e) return e;
    e = cudaMemsetAsync(w.west + n, 0, sizeof(int64_t), g->stream);   // largest medium W
    if (e) return e;
    if (n > 0 && g->nnz > 0) {
        GD_LAUNCH(g, "k_neighbor_degree", k_neighbor_degree, grid_for(g->nnz, 256, sms * 16), 256, 0,
                  g->nnz, g->rp, g->ci, w.nd);
        const int64_t small_cap = g->ctx->opt.smem_table_max / 2;
        // a hub's dense table costs 4n bytes: below W = n/8 wedges the
        // per-vertex open-addressing tables of the medium tier are cheaper
        const int64_t hub_min = std::max<int64_t>((int64_t)1 << g->ctx->opt.hub_wedges_log2, (int64_t)n / 8);
        GD_LAUNCH(g, "k_schedule", k_schedule, grid_for(n, SCHED_TILE, sms * 8), 256, 0,
                  n, g->rp, g->ci, w.nd, small_cap, hub_min,
                  g->ctx->opt.bitmap_max_outdeg, w.vlist, w.hubs, w.clist, w.counters, w.scan_tmp, w.west,
                  w.tlist);
        GD_LAUNCH(g, "k_medium_offsets", k_medium_offsets, 1, 32, 0, w.counters);
        GD_LAUNCH(g, "k_medium_place", k_medium_place, grid_for(n, 256, sms * 4), 256, 0, n, w.vlist, w.west,
                  w.counters, w.mlist);
        int64_t *offs = w.scan_tmp + (n + 1);
        int64_t *tmp = w.scan_tmp + 2 * (int64_t)(n + 1);
        e = exclusive_scan_i64(g, w.scan_tmp, offs, n, tmp);
        if (e) return e;
        GD_LAUNCH(g, "k_narrow", k_narrow_i32, grid_for(n + 1, 256, sms * 8), 256, 0, offs, w.dag_off, n + 1);
        GD_LAUNCH(g, "k_dag_fill", k_dag_fill, grid_for((int64_t)n * 32, 256, sms * 16), 256, 0,
                  n, g->rp, g->ci, w.nd, w.dag_off, w.dag_col, w.dag_slot, w.dag_nd);
    }
    e = cudaMemcpyAsync(counters_host, w.counters, C_NUM * sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream);
    if (e) return e;
    e = cudaMemcpyAsync(&w.medium_wmax, w.west + n, sizeof(int64_t), cudaMemcpyDeviceToHost, g->stream);
    if (e) return e;
    e = cudaStreamSynchronize(g->stream);
    if (e) return e;
    return cudaGetLastError();
}

// Triangle records per team: a warp team (out-degree <= 64) never holds more
// than C(64, 2); larger teams fall back to a second scan past 8192.
constexpr int32_t PAIR_CAP_WARP = CL_D0 * (CL_D0 - 1) / 2;
constexpr int32_t PAIR_CAP_CTA = 8192;

template <int DMAX, int THREADS, bool WARP_TEAMS, int MODE>
static cudaError_t clique_grid(gd_graph *g, int count, unsigned *grid, size_t *smem_out) {
    constexpr int TEAMS = WARP_TEAMS ? THREADS / 32 : 1;
    const size_t smem = DMAX > 0 ? (size_t)TEAMS * team_bytes<MODE>(DMAX, WARP_TEAMS ? 1 : THREADS / 32) : 0;
    auto kern = k_clique_bitmap<DMAX, THREADS, WARP_TEAMS, MODE>;
    *smem_out = smem;
    if (DMAX == 0) {
        *grid = (unsigned)g->ws.cbig_ctas;     // the global scratch holds this many CTAs
        return cudaSuccess;
    }
    cudaError_t e = allow_smem(kern, smem);
    if (e) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem);
    if (e) return e;
    *grid = grid_for((count + TEAMS - 1) / TEAMS, 1, sms_of(g) * (per_sm > 0 ? per_sm : 1));
    return cudaSuccess;
}

template <int DMAX, int THREADS, bool WARP_TEAMS>
static constexpr int32_t pair_cap_of() { return DMAX == 0 ? 0 : WARP_TEAMS ? PAIR_CAP_WARP : PAIR_CAP_CTA; }

template <int DMAX, int THREADS, bool WARP_TEAMS, int MODE>
static cudaError_t launch_clique(gd_graph *g, int bucket, int count) {
    if (count == 0) return cudaSuccess;
    Workspace &w = g->ws;
    CliqueArgs a;
    a.clist = w.clist; a.counters = w.counters; a.bucket = bucket; a.n = g->n; a.rp = g->rp;
    a.dag_off = w.dag_off; a.dag_col = w.dag_col; a.dag_slot = w.dag_slot; a.dag_nd = w.dag_nd;
    a.cacc = (unsigned long long *)w.cacc; a.tcred = w.tcred; a.tslot = w.tslot;
    a.qcred = (unsigned long long *)w.qcred;
    a.sums = w.sums; a.status = w.status;
    a.gstore = w.cbig; a.gdmax = w.cbig_dm; a.gstride = w.cbig_stride;
    a.dyn = w.counters + C_CLD0 + (MODE == MODE_TRISUM ? 4 : 0) + bucket;
    a.toff = w.toff; a.tcnt = w.recs ? w.tcnt : nullptr; a.recs = w.recs; a.rec_cap = w.recs_cap;
    if (MODE == MODE_COUNT) { a.tcnt = nullptr; a.recs = nullptr; a.rec_cap = 0; }
    constexpr int TEAMS = WARP_TEAMS ? THREADS / 32 : 1;
    unsigned grid;
    size_t smem;
    cudaError_t e = clique_grid<DMAX, THREADS, WARP_TEAMS, MODE>(g, count, &grid, &smem);
    if (e) return e;
    if (grid == 0) return cudaErrorInvalidValue;
    a.pairs = w.pairs;
    a.pair_cap = MODE == MODE_TRISUM ? 0 : pair_cap_of<DMAX, THREADS, WARP_TEAMS>();
    if ((size_t)grid * TEAMS * (size_t)a.pair_cap * 8 > w.pairs_bytes) a.pair_cap = 0;
    const char *name = MODE == MODE_TRISUM ? "k_trisum_bitmap" : "k_clique_bitmap";
    GD_LAUNCH(g, name, (k_clique_bitmap<DMAX, THREADS, WARP_TEAMS, MODE>), grid, THREADS, smem, a);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_clique_buckets(gd_graph *g, const int32_t *cnt) {
    cudaError_t e;
    if ((e = launch_clique<CL_D0, 256, true, MODE>(g, 0, cnt[C_CL0]))) return e;
    if ((e = launch_clique<CL_D1, 256, false, MODE>(g, 1, cnt[C_CL0 + 1]))) return e;
    if ((e = launch_clique<CL_D2, 1024, false, MODE>(g, 2, cnt[C_CL0 + 2]))) return e;
    return launch_clique<0, CL_BIG_THREADS, false, MODE>(g, 3, cnt[C_CL0 + 3]);
}

template <int DMAX, int THREADS, bool WARP_TEAMS>
static cudaError_t pairs_need(gd_graph *g, int count, size_t *need) {
    if (count == 0) return cudaSuccess;
    constexpr int TEAMS = WARP_TEAMS ? THREADS / 32 : 1;
    for (int mode = 0; mode < 2; mode++) {
        unsigned grid = 0;
        size_t smem;
        cudaError_t e = mode == 0 ? clique_grid<DMAX, THREADS, WARP_TEAMS, MODE_COUNT>(g, count, &grid, &smem)
                                  : clique_grid<DMAX, THREADS, WARP_TEAMS, MODE_CREDIT>(g, count, &grid, &smem);
        if (e) return e;
        const size_t b = (size_t)grid * TEAMS * (size_t)pair_cap_of<DMAX, THREADS, WARP_TEAMS>() * 8;
        if (b > *need) *need = b;
    }
    return cudaSuccess;
}

// Bytes of triangle records the clique kernels use for these bucket sizes.
cudaError_t clique_pairs_bytes(gd_graph *g, const int32_t *cnt, size_t *need) {
    *need = 0;
    cudaError_t e;
    if ((e = pairs_need<CL_D0, 256, true>(g, cnt[C_CL0], need))) return e;
    if ((e = pairs_need<CL_D1, 256, false>(g, cnt[C_CL0 + 1], need))) return e;
    return pairs_need<CL_D2, 1024, false>(g, cnt[C_CL0 + 2], need);
}

// Flat row offsets of all hubs (hub_off, nh + 1 entries); *flat receives
// hub_off[nh], the length of the hubs' concatenated rows.
cudaError_t run_hub_offsets(gd_graph *g, int32_t nh, int64_t *flat) {
    Workspace &w = g->ws;
    *flat = 0;
    if (nh == 0) return cudaSuccess;
    GD_LAUNCH(g, "k_hub_degrees", k_hub_degrees, grid_for(nh, 256, sms_of(g) * 4), 256, 0, nh, w.hubs, g->rp,
              w.scan_tmp);
    // hubs in decreasing rank (degree, then id): the heaviest come first,
    // and a batch holds hubs of similar degree
    std::vector<int32_t> ids(nh);
    std::vector<int64_t> deg(nh);
    cudaError_t e = cudaMemcpyAsync(ids.data(), w.hubs, sizeof(int32_t) * (size_t)nh, cudaMemcpyDeviceToHost, g->stream);
    if (!e) e = cudaMemcpyAsync(deg.data(), w.scan_tmp, sizeof(int64_t) * (size_t)nh, cudaMemcpyDeviceToHost, g->stream);
    if (!e) e = cudaStreamSynchronize(g->stream);
    if (e) return e;
    std::vector<int32_t> order(nh);
    for (int32_t i = 0; i < nh; i++) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        return deg[x] != deg[y] ? deg[x] > deg[y] : ids[x] > ids[y];
    });
    std::vector<int32_t> sorted(nh);
    std::vector<int64_t> sdeg(nh);
    for (int32_t i = 0; i < nh; i++) { sorted[i] = ids[order[i]]; sdeg[i] = deg[order[i]]; }
    e = cudaMemcpyAsync(w.hubs, sorted.data(), sizeof(int32_t) * (size_t)nh, cudaMemcpyHostToDevice, g->stream);
    if (!e) e = cudaMemcpyAsync(w.scan_tmp, sdeg.data(), sizeof(int64_t) * (size_t)nh, cudaMemcpyHostToDevice, g->stream);
    if (!e) e = cudaStreamSynchronize(g->stream);
    if (e) return e;
    e = exclusive_scan_i64(g, w.scan_tmp, w.hub_off, nh, w.scan_tmp + (nh + 1));
    if (e) return e;
    e = cudaMemcpyAsync(flat, w.hub_off + nh, sizeof(int64_t), cudaMemcpyDeviceToHost, g->stream);
    if (e) return e;
    return cudaStreamSynchronize(g->stream);
}

// Offsets of the per-node triangle record regions (toff, n + 1 entries);
// *total receives toff[n].
cudaError_t run_tri_bound(gd_graph *g, int64_t *total) {
    Workspace &w = g->ws;
    const int32_t n = g->n;
    *total = 0;
    if (n == 0 || g->m == 0) return cudaSuccess;     // no out-lists were built
    GD_LAUNCH(g, "k_tri_bound", k_tri_bound, grid_for((int64_t)n * 32, 256, sms_of(g) * 16), 256, 0,
              n, w.dag_off, w.dag_col, w.scan_tmp);
    cudaError_t e = exclusive_scan_i64(g, w.scan_tmp, w.toff, n, w.scan_tmp + (n + 1));
    if (e) return e;
    e = cudaMemcpyAsync(total, w.toff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, g->stream);
    if (e) return e;
    return cudaStreamSynchronize(g->stream);
}

// Upper bound of the same for a graph of n nodes (admission estimates).
size_t clique_pairs_bound(int sms, int64_t n) {
    const int64_t b0 = std::min<int64_t>((n + 7) / 8, (int64_t)sms * 8) * 8 * PAIR_CAP_WARP;
    const int64_t b1 = std::min<int64_t>(n, (int64_t)sms * 8) * PAIR_CAP_CTA;
    return (size_t)std::max(b0, b1) * 8;
}

size_t clique_big_bytes(int32_t dm) {
    const size_t c = team_bytes<MODE_CREDIT>(dm, CL_BIG_THREADS / 32), t = team_bytes<MODE_TRISUM>(dm, CL_BIG_THREADS / 32);
    const size_t k = team_bytes<MODE_COUNT>(dm, CL_BIG_THREADS / 32);
    return std::max(k, std::max(c, t));
}

// Triangles per slot and 4-cliques (credits when per_edge).  Requires the
// largest out-degree <= bitmap limit (checked by the caller).
cudaError_t run_triangles_cliques(gd_graph *g, bool per_edge, const int32_t *cnt) {
    Workspace &w = g->ws;
    const int sms = sms_of(g);
    if (g->m == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(w.tcred, 0, sizeof(uint32_t) * g->nnz, g->stream);
    if (e) return e;
    if (per_edge) {
        e = cudaMemsetAsync(w.cacc, 0, sizeof(uint64_t) * g->nnz, g->stream);
        if (e) return e;
        if ((e = launch_clique_buckets<MODE_CREDIT>(g, cnt))) return e;
    } else {
        if ((e = launch_clique_buckets<MODE_COUNT>(g, cnt))) return e;
    }
    GD_LAUNCH(g, "k_tri_symmetrize", k_tri_symmetrize, grid_for(g->m, 256, sms * 8), 256, 0,
              g->m, w.eslot, w.mate, w.tcred, w.tslot);
    return cudaGetLastError();
}

// Per-edge A_u + A_v and D_T through triangle credits (needs final |Tri|).
cudaError_t run_triangle_sums(gd_graph *g, const int32_t *cnt) {
    Workspace &w = g->ws;
    if (g->m == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(w.qcred, 0, 2 * sizeof(uint64_t) * g->nnz, g->stream);
    if (e) return e;
    return launch_clique_buckets<MODE_TRISUM>(g, cnt);
}

int32_t hub_batch(gd_graph *g) {
    // a few dense tables at a time so that they stay resident in L2 (~64 MB)
    const int64_t per = 4 * (int64_t)(g->n > 0 ? g->n : 1);
    int64_t b = (64ll << 20) / per;
    if (b < 1) b = 1;
    if (b > HUB_BATCH_MAX) b = HUB_BATCH_MAX;
    return (int32_t)b;
}

int32_t table_slots(gd_graph *g) { return hub_batch(g); }

// 4-cycles: credits (per_edge) or the 4-cycle total (global).
cudaError_t run_cycles(gd_graph *g, bool per_edge, const int32_t *cnt) {
    Workspace &w = g->ws;
    const int sms = sms_of(g);
    if (g->m == 0) return cudaSuccess;
    cudaError_t e;
    // per-slot credits in 32-bit words when they cannot pass 2^32: a slot's
    // total is at most the 4-cycles through its edge, <= (d_u - 1)(d_v - 1)
    w.yacc32 = per_edge && g->max_deg <= 65536;
    if (per_edge) {
        e = cudaMemsetAsync(w.yacc, 0, (w.yacc32 ? sizeof(uint32_t) : sizeof(uint64_t)) * g->nnz, g->stream);
        if (e) return e;
    }
    CycleArgs a;
    a.n = g->n; a.rp = g->rp; a.ci = g->ci; a.nd = w.nd;
    a.vlist = w.vlist; a.hubs = w.hubs; a.mlist = w.mlist; a.tlist = w.tlist; a.counters = w.counters;
    a.capmask = (uint32_t)(g->ctx->opt.smem_table_max - 1);
    a.tables = w.wtab; a.mtab = w.mtab; a.mcap = w.mtab_cap; a.west = w.west; a.status = w.status;
    a.yacc = (unsigned long long *)w.yacc; a.sums = w.sums;
    a.y32 = w.yacc32 ? reinterpret_cast<uint32_t *>(w.yacc) : nullptr;
    a.hub0 = 0; a.nhub = 0;
    // hubs, in batches, over one flat wedge prefix of all hubs
    const int32_t nh = cnt[C_HUB], B = std::min<int32_t>(hub_batch(g), w.wtab_ctas);   // tables allocated
    a.hoff = w.hub_off; a.hlen = w.hub_len; a.hpre = w.hub_pre;
    if (nh > 0) {
        GD_LAUNCH(g, "k_hub_lengths", k_hub_lengths, grid_for(w.hub_flat, 256, sms * 8), 256, 0, a, nh);
        e = exclusive_scan_i64(g, w.hub_len, w.hub_pre, w.hub_flat, w.hub_scan_tmp);
        if (e) return e;
        GD_LAUNCH(g, "k_hub_rows", k_hub_rows, grid_for(w.hub_flat, 256, sms * 8), 256, 0, a, nh);
    }
    int32_t first_push = 0;
    const int pull = g->ctx->opt.hub_pull;
    std::vector<int64_t> hw;
    int32_t pc[2] = {0, 0};
    PullItem *items = reinterpret_cast<PullItem *>(w.pull_items);
    const unsigned grid_f = grid_for(std::max<int64_t>(w.hub_flat, 1), 256, sms * 8);
    if (nh > 0 && w.pull_mask && pull != GD_PULL_NEVER) {
        // per-hub wedge work, and the chunks of the nodes of degree >=
        // PULL_WARP_DEG (once per count)
        hw.resize((size_t)nh + 1);
        GD_LAUNCH(g, "k_hub_work", k_hub_work, grid_for(nh + 1, 256, sms * 4), 256, 0, nh,
                  (const int64_t *)w.hub_off, (const int64_t *)w.hub_pre, w.scan_tmp);
        e = cudaMemcpyAsync(hw.data(), w.scan_tmp, sizeof(int64_t) * (size_t)(nh + 1), cudaMemcpyDeviceToHost, g->stream);
        if (!e) e = cudaMemsetAsync(w.pull_counts, 0, 2 * sizeof(int32_t), g->stream);
        if (e) return e;
        GD_LAUNCH(g, "k_pull_items", k_pull_items, grid_for(g->n, 256, sms * 8), 256, 0, g->n, g->rp, items,
                  w.pull_heavy_y, w.pull_counts);
        e = cudaMemcpyAsync(pc, w.pull_counts, sizeof(pc), cudaMemcpyDeviceToHost, g->stream);
        if (!e) e = cudaStreamSynchronize(g->stream);
        if (e) return e;
    }
    // one pull pass for hubs [h0, h0 + nb): masks set, counted, masks cleared;
    // TAB writes the per-hub counters into the batch's tables
    auto pull_batch = [&](int32_t h0, int32_t nb, bool tab) -> cudaError_t {
        const unsigned long long *mk = w.pull_mask;
        GD_LAUNCH(g, "k_pull_mark", k_pull_mark<true>, grid_f, 256, 0, a, h0, nb, w.pull_mask);
        if (tab) GD_LAUNCH(g, "k_pull_thread", k_pull_thread<true>, (unsigned)(sms * 8), 256, 0, a, h0, nb, mk);
        else GD_LAUNCH(g, "k_pull_thread", k_pull_thread<false>, (unsigned)(sms * 8), 256, 0, a, h0, nb, mk);
        if (pc[0] > 0) {
            const unsigned gr = grid_for((int64_t)pc[0] * 32, 256, sms * 8);
            if (tab) GD_LAUNCH(g, "k_pull_warp", k_pull_warp<true>, gr, 256, 0, a, h0, nb, mk, (const PullItem *)items,
                               pc[0], w.pull_heavy_cnt);
            else GD_LAUNCH(g, "k_pull_warp", k_pull_warp<false>, gr, 256, 0, a, h0, nb, mk, (const PullItem *)items,
                           pc[0], w.pull_heavy_cnt);
        }
        if (pc[1] > 0) {
            const unsigned gr = grid_for((int64_t)pc[1] * 32, 256, sms * 8);
            if (tab) GD_LAUNCH(g, "k_pull_heavy", k_pull_heavy<true>, gr, 256, 0, a, h0, nb,
                               (const int32_t *)w.pull_heavy_y, pc[1], w.pull_heavy_cnt);
            else GD_LAUNCH(g, "k_pull_heavy", k_pull_heavy<false>, gr, 256, 0, a, h0, nb,
                           (const int32_t *)w.pull_heavy_y, pc[1], w.pull_heavy_cnt);
        }
        GD_LAUNCH(g, "k_pull_clear", k_pull_mark<false>, grid_f, 256, 0, a, h0, nb, w.pull_mask);
        return cudaGetLastError();
    };
    if (!per_edge && !hw.empty()) {
        // global counts: the heaviest hubs, 64 at a time, in pull form while
        // a batch's wedges are at least half the CSR slots (a pull pass reads
        // every slot once; a push pass updates a counter per wedge and clears
        // its dense tables)
        while (first_push < nh) {
            const int32_t nb = std::min<int32_t>(PULL_MAX, nh - first_push);
            if (pull == GD_PULL_AUTO && hw[first_push + nb] - hw[first_push] < g->nnz / 2) break;
            if ((e = pull_batch(first_push, nb, false))) return e;
            first_push += nb;
        }
    }
    for (int32_t h0 = first_push; h0 < nh; h0 += B) {
        a.hub0 = h0;
        a.nhub = nh - h0 < B ? nh - h0 : B;
        // per-edge credits need the batch's counters in its tables: counted in
        // pull form when the batch's wedges are at least twice the CSR slots
        const bool tab_pull = per_edge && !hw.empty() &&
                              (pull == GD_PULL_ALWAYS || hw[h0 + a.nhub] - hw[h0] >= 2 * g->nnz);
        if (tab_pull) {
            if ((e = pull_batch(h0, a.nhub, true))) return e;
        } else {
            GD_LAUNCH(g, "k_cycles_hub_count", k_cycles_hub<0>, (unsigned)(sms * 8), 256, 0, a);
        }
        if (per_edge) GD_LAUNCH(g, "k_cycles_hub_credit", k_cycles_hub<1>, (unsigned)(sms * 8), 256, 0, a);
        if (per_edge) GD_LAUNCH(g, "k_cycles_hub_clear", k_cycles_hub_clear<true>, (unsigned)(sms * 4), 256, 0, a);
        else GD_LAUNCH(g, "k_cycles_hub_clear", k_cycles_hub_clear<false>, (unsigned)(sms * 4), 256, 0, a);
    }
    // medium tier: the largest vertices on clusters sharing one table, the
    // rest one CTA (and table) per vertex
    if (cnt[C_MEDIUM] > 0) {
        const int32_t slots = w.mtab_ctas;    // two 1024-thread CTAs fit on an SM
        const size_t smem = sizeof(long long) * (MED_PCAP + 1);
        int32_t nbig = 0;
        const int cl_log2 = g->ctx->opt.medium_cluster_log2 ? g->ctx->opt.medium_cluster_log2 : MED_CL_LOG2;
        for (int b = cl_log2; b < MB_BUCKETS; b++) nbig += cnt[C_MB0 + b];
        const int32_t ncl = std::min<int32_t>(std::min<int32_t>(slots, 2 * sms / MCL), nbig);
        if (ncl < 1) nbig = 0;
        const int32_t zero = 0;
        if ((e = cudaMemcpyAsync(w.counters + C_DYN2, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, g->stream))) return e;
        if ((e = cudaMemcpyAsync(w.counters + C_DYN, &nbig, sizeof(int32_t), cudaMemcpyHostToDevice, g->stream))) return e;
        if (nbig > 0) {
            if (per_edge) {
                if ((e = allow_smem(k_cycles_medium_cl<true>, smem))) return e;
                GD_LAUNCH(g, "k_cycles_medium", k_cycles_medium_cl<true>, (unsigned)(ncl * MCL), 1024, smem, a, nbig);
            } else {
                if ((e = allow_smem(k_cycles_medium_cl<false>, smem))) return e;
                GD_LAUNCH(g, "k_cycles_medium", k_cycles_medium_cl<false>, (unsigned)(ncl * MCL), 1024, smem, a, nbig);
            }
        }
        const int32_t rest = cnt[C_MEDIUM] - nbig;
        const unsigned grid = (unsigned)(rest < slots ? rest : slots);
        if (rest > 0) {
        if (per_edge) {
            if ((e = allow_smem(k_cycles_medium<1024, true>, smem))) return e;
            GD_LAUNCH(g, "k_cycles_medium", (k_cycles_medium<1024, true>), grid, 1024, smem, a);
        } else {
            if ((e = allow_smem(k_cycles_medium<1024, false>, smem))) return e;
            GD_LAUNCH(g, "k_cycles_medium", (k_cycles_medium<1024, false>), grid, 1024, smem, a);
        }
        }
    }
    // tiny tier
    if (cnt[C_TINY] > 0) {
        if (per_edge) GD_LAUNCH(g, "k_cycles_tiny", k_cycles_tiny<true>, grid_for((int64_t)cnt[C_TINY] * 32, 256, sms * 5), 256, 0, a);
        else GD_LAUNCH(g, "k_cycles_tiny", k_cycles_tiny<false>, grid_for((int64_t)cnt[C_TINY] * 32, 256, sms * 5), 256, 0, a);
    }
    // small tier
    if (cnt[C_SMALL] > 0) {
        const size_t smem = (size_t)(SMALL_PCAP + 1) * 8 + (size_t)(a.capmask + 1) * 8 + (size_t)((a.capmask + 1) / 2) * 4;
        if (per_edge) {
            if ((e = allow_smem(k_cycles_small<256, true>, smem))) return e;
            GD_LAUNCH(g, "k_cycles_small", (k_cycles_small<256, true>), (unsigned)(sms * 2), 256, smem, a);
        } else {
            if ((e = allow_smem(k_cycles_small<256, false>, smem))) return e;
            GD_LAUNCH(g, "k_cycles_small", (k_cycles_small<256, false>), (unsigned)(sms * 2), 256, smem, a);
        }
    }
    return cudaGetLastError();
}

}  // namespace gdi
