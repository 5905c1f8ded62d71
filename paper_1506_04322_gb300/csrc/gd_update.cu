// gd_update.cu -- exact change of the global counts when one node pair is
// toggled (an edge inserted or deleted).
//
// Only the 3- and 4-node subsets that contain both u and v change type, and
// each such subset's type with and without the edge follows from where its
// other nodes sit relative to u and v.  With A = N(u) \ {v}, B = N(v) \ {u}
// the other nodes fall into the classes of the paper's edge-centric
// decomposition (Sec. 4.1): T = A n B (Tri), Su = A \ B, Sv = B \ A (Star),
// I = the rest.  A 3-subset {u, v, w} is triangle / 2-star / 1-edge with the
// edge and 2-star / 1-edge / independent without it for w in T / S / I; a
// 4-subset {u, v, w, r} is typed by the classes of w and r and whether w and
// r are adjacent (the restricted counts N_{a,b,1} of Sec. 4.1), e.g. w, r in
// T adjacent is a 4-clique with the edge and a chordal cycle without it.
// The kernel counts, for every w in A u B, the neighbours r of w by class;
// the host turns the class sizes and the adjacent-pair counts into the
// number of subsets leaving and entering each graphlet.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "gd_device.cuh"
#include "gd_internal.h"

namespace gdi {

namespace {

using namespace gdi::dev;

// record slots: ordered adjacent pairs O[cw][cr] (cw in T,Su,Sv; cr in
// T,Su,Sv,I), class sizes |T|, |Su|, |Sv|, and whether (u, v) is an edge
enum { PR_T = 0, PR_SU = 1, PR_SV = 2, PR_I = 3 };
constexpr int PR_O = 0;           // 12 entries: 4 * cw + cr
constexpr int PR_SIZE = 12;       // 3 entries
constexpr int PR_EDGE = 15;
constexpr int PR_NUM = 16;

__device__ __forceinline__ bool in_row(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t x,
                                       int32_t y) {
    int32_t lo = rp[x], hi = rp[x + 1];
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (ci[mid] < y) lo = mid + 1; else hi = mid;
    }
    return lo < rp[x + 1] && ci[lo] == y;
}

// One warp per node w of A u B (the entries of N(u), then those of N(v)
// outside N(u)); its lanes classify the neighbours of w.
__global__ void k_pair_record(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t u, int32_t v,
                              unsigned long long *rec) {
    unsigned long long o[12];
#pragma unroll
    for (int i = 0; i < 12; i++) o[i] = 0;
    unsigned long long sz[3] = {0, 0, 0};
    const int lane = lane_id();
    const int32_t bu = rp[u], du = rp[u + 1] - bu, bv = rp[v], dv = rp[v + 1] - bv;
    for (int64_t j = global_warp(); j < (int64_t)du + dv; j += num_warps()) {
        int32_t w, cw;
        if (j < du) {
            w = ci[bu + j];
            if (w == v) continue;
            cw = in_row(rp, ci, v, w) ? PR_T : PR_SU;
        } else {
            w = ci[bv + (j - du)];
            if (w == u || in_row(rp, ci, u, w)) continue;     // u, or already seen as a member of T
            cw = PR_SV;
        }
        if (lane == 0) sz[cw]++;
        const int32_t bw = rp[w], dw = rp[w + 1] - bw;
        for (int32_t i = lane; i < dw; i += WARP) {
            const int32_t r = ci[bw + i];
            if (r == u || r == v) continue;
            const bool ra = in_row(rp, ci, u, r), rb = in_row(rp, ci, v, r);
            const int cr = ra ? (rb ? PR_T : PR_SU) : (rb ? PR_SV : PR_I);
#pragma unroll
            for (int c = 0; c < 12; c++)
                if (c == 4 * cw + cr) o[c]++;
        }
    }
#pragma unroll
    for (int c = 0; c < 12; c++) {
        const unsigned long long s = warp_sum(o[c]);
        if (lane == 0 && s) atomicAdd(rec + PR_O + c, s);
    }
#pragma unroll
    for (int c = 0; c < 3; c++)
        if (lane == 0 && sz[c]) atomicAdd(rec + PR_SIZE + c, sz[c]);
    if (blockIdx.x == 0 && threadIdx.x == 0 && in_row(rp, ci, u, v)) rec[PR_EDGE] = 1;
}

using u128 = unsigned __int128;

u128 c2(u128 x) { return x < 2 ? 0 : x * (x - 1) / 2; }

}  // namespace

}  // namespace gdi

using namespace gdi;

extern "C" {

int gd_toggle_delta(gd_graph *g, int32_t u, int32_t v, gd_u128 gain[15], gd_u128 loss[15], int *was_edge) {
    if (!g || !gain || !loss) return GD_EINVAL;
    gd_ctx *ctx = g->ctx;
    if (u < 0 || v < 0 || u >= g->n || v >= g->n || u == v) {
        ctx->err = "gd_toggle_delta: u and v must be distinct nodes of the graph";
        return GD_EINVAL;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    unsigned long long *rec = nullptr;
    int rc = GD_OK;
    if (e == cudaSuccess && (rc = scratch_alloc(ctx, (void **)&rec, sizeof(unsigned long long) * PR_NUM)) != GD_OK)
        return rc;
    unsigned long long h[PR_NUM];
    if (e == cudaSuccess) e = cudaMemsetAsync(rec, 0, sizeof(h), g->stream);
    if (e == cudaSuccess) {
        const int sms = ctx->num_sms > 0 ? ctx->num_sms : 152;
        GD_LAUNCH(g, "k_pair_record", k_pair_record, (unsigned)(sms * 4), 256, 0, g->rp, g->ci, u, v, rec);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, rec, sizeof(h), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (rec) scratch_release(ctx, rec, sizeof(unsigned long long) * PR_NUM);
    if (e != cudaSuccess) {
        ctx->err = std::string("gd_toggle_delta: ") + cudaGetErrorString(e);
        return GD_ECUDA;
    }
    // class sizes and restricted counts (unordered adjacent pairs)
    const u128 T = h[PR_SIZE + PR_T], Su = h[PR_SIZE + PR_SU], Sv = h[PR_SIZE + PR_SV];
    const bool edge = h[PR_EDGE] != 0;
    const u128 I = (u128)(g->n - 2) - T - Su - Sv;
    auto O = [&](int a, int b) { return (u128)h[PR_O + 4 * a + b]; };
    const u128 tt = O(PR_T, PR_T) / 2, tsu = O(PR_T, PR_SU), tsv = O(PR_T, PR_SV);
    const u128 susu = O(PR_SU, PR_SU) / 2, svsv = O(PR_SV, PR_SV) / 2, susv = O(PR_SU, PR_SV);
    const u128 ti = O(PR_T, PR_I), sui = O(PR_SU, PR_I), svi = O(PR_SV, PR_I);
    const u128 m_other = (u128)g->m - (edge ? 1 : 0);
    const u128 inside = tt + tsu + tsv + susu + svsv + susv, outward = ti + sui + svi;
    const u128 ii = m_other - (T * 2 + Su + Sv) - inside - outward;   // edges among I
    // (count, type with the edge, type without it), Table 1 indices
    struct Move { u128 count; int with, without; };
    const Move mv[] = {
        {T, 0, 1}, {Su + Sv, 1, 2}, {I, 2, 3},
        {tt, 4, 5},                                   // w, r in T, adjacent: 4-clique -> chordal cycle
        {c2(T) - tt, 5, 7},                           // not adjacent: chordal cycle -> 4-cycle
        {tsu + tsv, 5, 6},                            // T and Star, adjacent: chordal cycle -> tailed triangle
        {T * (Su + Sv) - tsu - tsv, 6, 9},            // not adjacent: tailed triangle -> 4-path
        {ti, 6, 8},                                   // T and I, adjacent: tailed triangle -> 3-star
        {T * I - ti, 10, 11},                         // not adjacent: triangle+1 -> 2-star+1
        {susu + svsv, 6, 10},                         // same Star, adjacent: tailed triangle -> triangle+1
        {c2(Su) + c2(Sv) - susu - svsv, 8, 11},       // not adjacent: 3-star -> 2-star+1
        {susv, 7, 9},                                 // Su, Sv adjacent: 4-cycle -> 4-path
        {Su * Sv - susv, 9, 12},                      // not adjacent: 4-path -> 2 edges
        {sui + svi, 9, 11},                           // Star and I, adjacent: 4-path -> 2-star+1
        {(Su + Sv) * I - sui - svi, 11, 13},          // not adjacent: 2-star+1 -> 1 edge+2
        {ii, 12, 13},                                 // I, I adjacent: 2 edges -> 1 edge+2
        {c2(I) - ii, 13, 14},                         // not adjacent: 1 edge+2 -> independent
    };
    u128 gn[15] = {0}, ls[15] = {0};
    for (const Move &x : mv) {
        if (edge) { ls[x.with] += x.count; gn[x.without] += x.count; }
        else { ls[x.without] += x.count; gn[x.with] += x.count; }
    }
    for (int i = 0; i < 15; i++) {
        gain[i].lo = (uint64_t)gn[i]; gain[i].hi = (uint64_t)(gn[i] >> 64);
        loss[i].lo = (uint64_t)ls[i]; loss[i].hi = (uint64_t)(ls[i] >> 64);
    }
    if (was_edge) *was_edge = edge ? 1 : 0;
    return GD_OK;
}

}  // extern "C"
