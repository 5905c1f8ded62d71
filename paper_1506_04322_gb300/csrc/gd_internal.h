// gd_internal.h -- shared between the host API (gd_api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/gd.h"

namespace gdi {

// Indices of the 13 edge-summed quantities of Algorithm 2 (Steps 1-3).
enum SumIdx {
    S_T = 0,     // sum |Tri_e|
    S_S,         // sum |Star_u| + |Star_v|
    S_I,         // sum |V| - |N(u) u N(v)|
    S_CLIQ,      // sum cliq_e  (= 6 f41)
    S_CYC,       // sum cyc_e   (= 4 f44)
    S_TT,        // sum C(T,2)
    S_SUSV,      // sum Su*Sv
    S_TS,        // sum T(Su+Sv)
    S_SS,        // sum C(Su,2)+C(Sv,2)
    S_TI,        // sum T*I
    S_SI,        // sum (Su+Sv)*I
    S_II,        // sum C(I,2)
    S_II1,       // sum |E| - du - dv + 1
    S_NUM
};

// Extra sums used only to derive sum cyc_e in the global path.
enum ExtraIdx { X_T2 = 0, X_C4 = 1, X_NUM = 2 };

// Schedule counters (device word array filled by k_schedule).
enum CounterIdx {
    C_SMALL = 0,    // vertices in the shared-memory wedge tier
    C_MEDIUM = 1,   // vertices in the per-CTA dense-table tier
    C_MAXDP = 2,    // largest out-degree under the degree ordering
    C_HUB = 3,      // hubs (whole-GPU batches)
    C_CL0 = 4,      // 4 clique buckets by out-degree: <=CL_D0, <=CL_D1, <=CL_D2, larger
    C_DYN = 8,      // dynamic work index of the medium tier
    C_TINY = 9,     // vertices in the warp-level wedge tier
    C_DYN2 = 11,    // dynamic work index of the medium tier's cluster kernel
    C_MB0 = 16,     // medium tier: vertices per log2(wedges) bucket (40 buckets)
    C_MOFF = 64,    // medium tier: placement offsets per bucket (40)
    C_CLD0 = 104,   // clique kernels: work counters (pass x bucket, 8)
    C_NUM = 112
};
constexpr int MB_BUCKETS = 40;
constexpr int TINY_WEDGES = 256;   // warp-level wedge table of 2 * TINY_WEDGES entries
constexpr int CL_D0 = 64, CL_D1 = 256, CL_D2 = 1024;
constexpr int CL_BIG_THREADS = 512;   // CTA size of the large out-list (global scratch) variant

// Device-side error bits (gdi::Status word).
enum ErrBits {
    ERR_NEGATIVE = 1,     // a restricted count came out negative: inconsistent input
    ERR_REMAINDER = 2,    // an exact division left a remainder
    ERR_CAPACITY = 4,     // a work buffer was too small (host sizing bug)
    ERR_CSR = 8,          // CSR validation failed
    ERR_TIMEOUT = 16      // a bounded wait gave up
};

// Per-graph device scratch for the wedge tables and triangle buffers.
struct Workspace {
    // edge list (canonical order: row u ascending, v > u ascending)
    int32_t *first_up = nullptr;   // [n]   first slot of row u with col > u
    int32_t *eoff = nullptr;       // [n+1] edge offset of row u
    int32_t *eu = nullptr, *ev = nullptr, *eslot = nullptr;   // [m]
    int32_t *mate = nullptr;       // [nnz] slot of the reverse direction
    uint32_t *tslot = nullptr;     // [nnz] |Tri| of the edge of each slot
    // per-edge mode
    uint64_t *tnode = nullptr;     // [n] edges inside N(x)
    uint64_t *s1 = nullptr;        // [n] sum of neighbour degrees
    uint64_t *au = nullptr, *dt = nullptr;   // [m] A_u + A_v and D_T (intersection path)
    uint64_t *qcred = nullptr;   // [2 nnz] per slot: triangle-perimeter credit, degree-sum credit
    uint64_t *cacc = nullptr;      // [nnz] 4-clique credits per slot
    uint64_t *yacc = nullptr;      // [nnz] 4-cycle credits per slot (or cyc_e for literal)
    bool yacc32 = false;           // the oriented per-edge credits are uint32 words (max degree <= 65536)
    // schedule
    int32_t *vlist = nullptr;      // [n] small tier from the front, medium tier from the back
    int32_t *hubs = nullptr;       // [n] hub tier
    int32_t *clist = nullptr;      // [4n] clique buckets by out-degree
    int32_t *counters = nullptr;   // [C_NUM]
    int32_t *nd = nullptr;         // [nnz] degree of each slot's neighbour
    int32_t *dag_off = nullptr;    // [n+1] out-lists under the degree ordering
    int32_t *dag_col = nullptr, *dag_slot = nullptr, *dag_nd = nullptr;   // [m]
    uint32_t *tcred = nullptr;     // [nnz] triangle credits per slot
    unsigned long long *pairs = nullptr;   // per-team triangle records of the clique kernels
    size_t pairs_bytes = 0;
    int64_t *toff = nullptr;               // per-edge mode: per-node triangle record offsets (n + 1)
    int32_t *tcnt = nullptr;               // records kept per node, -1 none
    unsigned long long *recs = nullptr;    // triangle records kept for the triangle-sum pass
    int64_t recs_cap = 0;                  // entries
    unsigned char *cbig = nullptr; // per-CTA scratch of the large out-list clique kernel
    size_t cbig_bytes = 0, cbig_stride = 0;
    int32_t cbig_dm = 0, cbig_ctas = 0;
    int32_t *mlist = nullptr;      // [n] medium tier sorted by decreasing wedge work
    int64_t *hub_off = nullptr, *hub_len = nullptr, *hub_pre = nullptr, *hub_scan_tmp = nullptr;
    int64_t hub_flat_cap = 0;      // capacity of hub_len / hub_pre
    unsigned long long *pull_mask = nullptr;   // [n] global counts: batch-hub bits per node (zero at rest)
    int32_t *pull_items = nullptr;         // [3 * (nnz/64 + nnz/1024 + 1)] chunks of the high-degree nodes
    int32_t *pull_heavy_y = nullptr;       // [nnz/1024 + 1] nodes of several chunks
    uint32_t *pull_heavy_cnt = nullptr;    // [64 * (nnz/1024 + 1)] their per-hub counters (zero at rest)
    int32_t *pull_counts = nullptr;        // [2] chunks, heavy nodes
    int64_t hub_flat = 0;          // the hubs' concatenated rows (this count call)
    int32_t hub_off_cap = 0;       // capacity of hub_off
    int32_t *tlist = nullptr;      // [n] tiny tier (warp per vertex)
    int64_t *west = nullptr;       // [n] wedge work of medium vertices
    // scratch
    int32_t *tribuf = nullptr;     // [warps * tricap * 3]
    int64_t tribuf_words = 0;
    uint32_t *wtab = nullptr;      // [hub batch * n] dense wedge tables (zero at rest)
    unsigned long long *mtab = nullptr;   // medium tier: per-CTA open-addressing tables (empty at rest)
    int64_t mtab_cap = 0;                 // entries per CTA (power of two)
    int32_t mtab_ctas = 0;
    int64_t medium_wmax = 0;              // largest medium-tier W of the last schedule (host copy)
    int32_t wtab_ctas = 0;
    // results
    unsigned long long *sums = nullptr;   // [2*(S_NUM+X_NUM)] u128 as lo,hi
    unsigned long long *result = nullptr; // [30] 15 x u128
    int32_t *status = nullptr;            // [4] error bits, detail
    // scan scratch
    int64_t *scan_tmp = nullptr;
    // per-edge output staging when the caller's buffer is on the host
    uint64_t *out_buf = nullptr;
    size_t out_buf_bytes = 0;
    size_t bytes = 0;
    std::vector<std::pair<void *, size_t>> blocks;   // every block above, for release
};

}  // namespace gdi


namespace gdi {
struct Service;
struct BatchGraph;      // captured CUDA graph of gd_count_batch (gd_api.cu)
void batch_graph_destroy(gd_ctx *ctx);
void serve_destroy(gd_ctx *ctx);
struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
};
}  // namespace gdi


namespace gdi {
// packed arrays of gd_count_batch_gather (grown on demand, kept for reuse)
struct GatherBufs {
    int32_t *gnp = nullptr, *eoff = nullptr, *rp = nullptr, *ci = nullptr, *misc = nullptr;
    size_t gnp_bytes = 0, eoff_bytes = 0, rp_bytes = 0, ci_bytes = 0, misc_bytes = 0;
};
}  // namespace gdi

struct gd_ctx {
    int device = 0;
    size_t budget = 0;           // 0 = unlimited
    size_t in_use = 0;           // device bytes held by this context's graphs
    gd_options opt{};
    std::string err;
    int num_sms = 0;
    cudaStream_t stream = nullptr;   // for batch calls
    std::vector<gd_graph *> graphs;
    // batch scratch (grown on demand)
    void *batch_buf = nullptr;
    size_t batch_bytes = 0;
    // caching allocator: released device blocks by size, reused by later graphs
    std::multimap<size_t, void *> pool;
    size_t pooled = 0;
    // stage timing (CUDA events around each launch while enabled)
    bool prof = false;
    std::vector<gdi::ProfRec> recs;
    std::vector<cudaEvent_t> evpool;
    int64_t launches = 0;
    // request loop (gd_serve.cu)
    gdi::Service *service = nullptr;
    // captured batch pipeline
    gdi::BatchGraph *bgraph = nullptr;
    gdi::GatherBufs gather;
    // per-edge output copied to the host in chunks on several streams at once
    static constexpr int COPY_STREAMS = 4;
    cudaStream_t copy_st[COPY_STREAMS] = {};
    cudaEvent_t copy_ev[COPY_STREAMS + 1] = {};
};

struct gd_graph {
    gd_ctx *ctx = nullptr;
    int32_t n = 0;
    int64_t nnz = 0, m = 0;
    cudaStream_t stream = nullptr;
    int32_t *rp = nullptr, *ci = nullptr;
    bool borrowed = false;
    size_t csr_bytes = 0;
    int32_t max_deg = 0;
    bool prepared = false;       // edge list (eu, ev: rows of the per-edge output) built
    gdi::Workspace ws;
};

namespace gdi {

// exclusive scan of len int64 values, out[len] = total (gd_count.cu); tmp
// needs 2 * ceil(len / 1024) + 64 entries per level
cudaError_t exclusive_scan_i64(gd_graph *g, const int64_t *in, int64_t *out, int64_t len, int64_t *tmp);

// device scratch through the context's cache and budget (gd_api.cu)
int scratch_alloc(gd_ctx *ctx, void **p, size_t bytes);
void scratch_release(gd_ctx *ctx, void *p, size_t bytes);

// launch bookkeeping (gd_api.cu): launch counter and, while profiling, an
// event pair around the launch on the graph's stream
void prof_begin(gd_ctx *c, cudaStream_t st, const char *name);
void prof_end(gd_ctx *c, cudaStream_t st);

// kernels (gd_count.cu)
cudaError_t validate_csr(gd_graph *g, int32_t *bad_index_host, int32_t *bad_code_host);
cudaError_t launch_validate(gd_graph *g, int32_t *status);   // kernel only (capturable)
cudaError_t prepare_edges(gd_graph *g);                   // edge list, reverse slots, zero sums
cudaError_t run_triangles_intersect(gd_graph *g);         // |Tri| per slot by intersection
cudaError_t run_per_edge_sums(gd_graph *g);               // t(x), S1(x), A_u, A_v, D_T
cudaError_t run_literal(gd_graph *g);                     // Algorithm 2 CliqueCount / CycleCount
cudaError_t run_final(gd_graph *g, int variant, bool per_edge, bool cliq_credits, bool qr_credits,
                      uint64_t *out_dev);
// gd_step2.cu
cudaError_t run_schedule(gd_graph *g, int32_t *counters_host);
cudaError_t run_triangles_cliques(gd_graph *g, bool per_edge, const int32_t *counters_host);
cudaError_t run_triangle_sums(gd_graph *g, const int32_t *counters_host);   // Q/R credits (needs |Tri|)
cudaError_t run_node_sums(gd_graph *g, bool have_nd);                                      // t(x), S1(x)
size_t clique_big_bytes(int32_t dm);
cudaError_t clique_pairs_bytes(gd_graph *g, const int32_t *counters_host, size_t *need);
cudaError_t run_tri_bound(gd_graph *g, int64_t *total);
cudaError_t run_hub_offsets(gd_graph *g, int32_t nh, int64_t *flat);
int64_t medium_table_limit(int64_t nnz);
size_t clique_pairs_bound(int sms, int64_t n);                                         // per CTA
cudaError_t run_cycles(gd_graph *g, bool per_edge, const int32_t *counters_host);
int32_t table_slots(gd_graph *g);
int32_t hub_batch(gd_graph *g);
cudaError_t run_complete(gd_graph *g, int derive_cyc);
cudaError_t max_degree(gd_graph *g, int32_t *out_host);
int32_t tribuf_warps(int sms);

// gd_api.cu
size_t estimate_footprint(gd_ctx *ctx, int64_t n, int64_t nnz, bool per_edge, bool host_out);

// batch (gd_batch.cu)
size_t batch_smem_bytes(int nmax);
cudaError_t launch_batch_count(gd_ctx *ctx, cudaStream_t st, int32_t num_graphs, const int32_t *gnp,
                               const int32_t *rp, const int32_t *ci, int32_t *work, unsigned long long *out,
                               int32_t *gstatus, int32_t *big_list, int32_t *big_count, int nmax);
cudaError_t launch_batch_gather(gd_ctx *ctx, cudaStream_t st, int32_t num_graphs, const int32_t *const *rps,
                                const int32_t *const *cis, const int32_t *gnp, const int32_t *eoff,
                                int32_t *rp_out, int32_t *ci_out, int32_t *gstatus);
cudaError_t launch_batch_slice(gd_ctx *ctx, cudaStream_t st, int32_t n0, int32_t n, const int32_t *rp,
                               const int32_t *ci, int32_t *lrp, int32_t *lci);

}  // namespace gdi

#define GD_LAUNCH(G, NAME, KERNEL, GRID, BLOCK, SMEM, ...)                      \
    do {                                                                        \
        gdi::prof_begin((G)->ctx, (G)->stream, NAME);                           \
        KERNEL<<<(GRID), (BLOCK), (SMEM), (G)->stream>>>(__VA_ARGS__);          \
        gdi::prof_end((G)->ctx, (G)->stream);                                   \
    } while (0)
