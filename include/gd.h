/*
 * gd.h -- exact 3- and 4-node graphlet decomposition on one GB300 (sm_103a).
 *
 * C ABI of libgd.so.  Plain pointers and sizes only.
 *
 * Paper: N. K. Ahmed, J. Neville, R. A. Rossi, N. Duffield, T. L. Willke,
 * "Graphlet Decomposition: Framework, Algorithms, and Applications" (2015),
 * arXiv:1506.04322.
 *
 * Problem (Sec. 2.1, problem statement and Definitions 1-2): for an undirected
 * simple graph G = (V, E), count the k-node subsets of V whose induced
 * subgraph is isomorphic to each graphlet of size k = 3 and k = 4 (4 and 11
 * graphlets, Table 1).  The method (Sec. 3-4, Algorithms 1-2) visits every
 * edge e = (u, v) once, finds Tri_e = N(u) n N(v) and the star sets
 * Star_u, Star_v, counts 4-cliques and 4-cycles through e directly
 * (CliqueCount, CycleCount), adds the unrestricted counts of Sec. 4.2 and
 * completes the rest with the Lemmas of Sec. 4.3 and the equations for g4_9
 * and g4_11.
 *
 * Result order (Table 1 numbering), used by every call that returns counts:
 *   index  0  1  2  3  4  5  6  7  8  9  10 11 12 13   14
 *          g31 g32 g33 g34 g41 g42 g43 g44 g45 g46 g47 g48 g49 g4_10 g4_11
 *   g31 triangle, g32 2-star, g33 3-node-1-edge, g34 3-node-independent,
 *   g41 4-clique, g42 4-chordal-cycle, g43 4-tailed-triangle, g44 4-cycle,
 *   g45 3-star, g46 4-path, g47 4-node-1-triangle, g48 4-node-2-star,
 *   g49 4-node-2-edge, g4_10 4-node-1-edge, g4_11 4-node-independent.
 *
 * Input graph format (all calls): CSR with n rows, row_ptr int32[n+1]
 * (row_ptr[0] = 0, non-decreasing), col_idx int32[nnz] with nnz = row_ptr[n]
 * = 2|E|: both directions of every edge are stored, each row strictly
 * ascending, no self-loops, every id in [0, n).  |V| = n counts isolated rows
 * (Sec. 3.2 uses |V| in the counts of g33 / g34).
 *
 * Arithmetic: exact integers only.  Global counts are unsigned 128-bit
 * (C(n,4) exceeds 2^64 for n > ~1.1e5); per-edge counts are uint64.
 *
 * Error behaviour: every call returns a gd_status.  On failure no output is
 * written (a per-edge output buffer may hold partial data) and the context's
 * last-error text (gd_last_error) says why.  GD_ECUDA means a CUDA runtime
 * error; the context should then be destroyed.
 *
 * Threading: calls on one context are not thread-safe; use one context per
 * host thread, except gd_submit / gd_poll which may be called from one
 * producer thread while the service thread runs.
 */
#ifndef GD_H
#define GD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Exact unsigned 128-bit integer: value = lo + 2^64 * hi. */
typedef struct gd_u128 { uint64_t lo, hi; } gd_u128;

typedef struct gd_ctx gd_ctx;
typedef struct gd_graph gd_graph;
typedef uint64_t gd_req;

typedef enum gd_status {
    GD_OK = 0,
    GD_EINVAL = 1,      /* bad argument, or CSR not simple/sorted/symmetric */
    GD_ENOMEM = 2,      /* host or device allocation failed, or over budget */
    GD_ECUDA = 3,       /* CUDA runtime error (see gd_last_error)           */
    GD_EAGAIN = 4,      /* gd_poll: request not finished yet               */
    GD_ETIMEDOUT = 5,   /* a bounded device-side wait gave up              */
    GD_EOVERFLOW = 6,   /* n or nnz beyond int32 ids                        */
    GD_ENOTIMPL = 7,    /* option combination not available                 */
    GD_EARITH = 8       /* an exact division left a remainder (internal)    */
} gd_status;

/* gd_create_csr flags */
enum {
    GD_DEVICE_PTRS = 1,  /* row_ptr / col_idx are device pointers            */
    GD_VALIDATE = 2,     /* accepted for clarity: the full CSR check (sorted,
                            simple, symmetric, ids in range) always runs     */
    GD_BORROW = 4        /* with GD_DEVICE_PTRS: use the caller's arrays in
                            place (caller keeps them alive and unchanged until
                            gd_destroy_graph) instead of copying them         */
};

/* gd_count_per_edge / gd_count_batch output flags */
enum { GD_OUT_DEVICE = 1 };

/* gd_count_batch flag: keep the device part of the call (validation, the
 * persistent counting launch, the result copy) as a captured CUDA graph and
 * replay it when the next call has the same pointers, sizes and graph
 * offsets.  Inputs must be device pointers (GD_DEVICE_PTRS). */
enum { GD_CAPTURE = 8 };

/* How the 4-node direct counts of Step 2 are obtained (Sec. 4.4). */
typedef enum gd_variant {
    GD_VARIANT_AUTO = 0,     /* fastest exact variant for the graph           */
    GD_VARIANT_LITERAL = 1,  /* per edge: CliqueCount scans the lists of Tri_e,
                                CycleCount scans the lists of Star_u exactly as
                                Algorithm 2 (cost sum over Star_u of degrees)  */
    GD_VARIANT_ORIENTED = 2  /* every 4-clique and 4-cycle enumerated once under
                                a degree ordering and credited to its edges;
                                cyc_e from 4-cycle counts via the restricted-
                                count identities (identical results)         */
} gd_variant;

typedef struct gd_options {
    int32_t variant;          /* gd_variant (default AUTO)                         */
    int32_t block_threads;    /* threads per CTA of the edge kernels (default 256) */
    int32_t ctas_per_sm;      /* persistent CTAs per SM (default: occupancy)       */
    int32_t smem_table_max;   /* wedge-table entries kept in shared memory per CTA
                                 (power of two in [256, 16384], default 8192);
                                 vertices with at most half as many wedges use it */
    int32_t bitmap_max_outdeg;   /* nodes with at most this many higher-ranked
                                    neighbours keep the triangle/4-clique work
                                    arrays in shared memory; nodes with more use
                                    the same kernel on global scratch
                                    (default and maximum 1024, minimum 2)       */
    int32_t hub_wedges_log2;  /* vertices with more than max(2^k, n/8) wedges are
                                 processed by the whole GPU in batches (dense
                                 tables of n counters); below, one CTA per vertex
                                 with a table sized to its wedges (default 17) */
    int32_t hub_pull;         /* global counts only: GD_PULL_AUTO (default) counts
                                 the heaviest hubs, 64 at a time, by summing per-node
                                 hub bit masks at each opposite node while a batch
                                 has at least nnz/2 wedges, the rest by counter
                                 updates; GD_PULL_NEVER, GD_PULL_ALWAYS force one
                                 form for every hub (the counts are the same)      */
    int32_t batch_threads;    /* threads per CTA of the batched kernel (one graph
                                 per CTA, its adjacency bit matrix in shared
                                 memory): 0 (default) = 256 for graphs up to 512
                                 nodes, 512 up to 1024; else 128, 256 or 512 for
                                 the 512-node kernel and 256, 512 or 1024 for
                                 the 1024-node kernel (the nearest is taken)  */
    int32_t medium_cluster_log2;  /* medium-tier vertices with at least 2^k wedges
                                     are counted by clusters of 8 CTAs sharing one
                                     table (0: default 16; above 40: never)      */
    int32_t reserved[3];
} gd_options;

enum { GD_PULL_AUTO = 0, GD_PULL_NEVER = 1, GD_PULL_ALWAYS = 2 };

/* Fill *opt with the defaults. */
void gd_default_options(gd_options *opt);

/* Replace a context's options (same checks as gd_init); the next count call
 * uses them.  *opt receives nothing; gd_get_options reads them back. */
int gd_set_options(gd_ctx *ctx, const gd_options *opt);
int gd_get_options(const gd_ctx *ctx, gd_options *opt);

/* Create a context on CUDA device `device`.  hbm_budget_bytes = 0: no limit;
 * otherwise graphs whose device footprint would exceed the budget are refused
 * with GD_ENOMEM.  opt may be NULL (defaults).  *ctx receives the handle. */
int gd_init(gd_ctx **ctx, int device, size_t hbm_budget_bytes, const gd_options *opt);

/* Destroy a context and every graph still attached to it. */
void gd_destroy(gd_ctx *ctx);

/* Text of the last error on this context ("" if none).  Valid until the next
 * call on the context. */
const char *gd_last_error(gd_ctx *ctx);

/* Upload (or adopt, with GD_DEVICE_PTRS|GD_BORROW) a CSR graph.  n rows,
 * nnz = row_ptr[n] entries.  cuda_stream (a cudaStream_t, may be NULL for the
 * legacy default stream) is the stream every later call on this graph uses.
 * The CSR is always checked on the device (row bounds, strictly ascending
 * rows, ids in range, no self-loops, every edge stored in both directions);
 * a violation returns GD_EINVAL naming the first bad row.  The check costs
 * one binary search per stored entry.  *out receives the handle. */
int gd_create_csr(gd_ctx *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr,
                  const int32_t *col_idx, int flags, void *cuda_stream, gd_graph **out);

/* n and |E| of a graph. */
int gd_graph_info(const gd_graph *g, int32_t *n, int64_t *m);

/* Bytes of device memory the graph holds now (CSR + per-graph work arrays). */
int gd_graph_footprint(const gd_graph *g, size_t *bytes);

/* Release a graph (device memory included). */
void gd_destroy_graph(gd_graph *g);

/* Global counts of all 15 graphlets of size 3 and 4 (Algorithm 2 result).
 * out: host array of 15 gd_u128.  Synchronous. */
int gd_count_global(gd_graph *g, gd_u128 out[15]);

/* Per-edge counts: for every edge e = (u, v), u < v, in CSR order (row u
 * ascending, then v ascending), the number of induced 3- and 4-node subsets
 * that contain u and v and are isomorphic to each graphlet (Corollaries 1-14
 * evaluated per edge).  out: uint64[|E|][15] row-major, host memory, or
 * device memory if out_flags has GD_OUT_DEVICE.  Columns g34 and g4_11 are 0
 * by definition (those graphlets have no edge).  global_out (host, nullable)
 * receives the global counts too.  Synchronous. */
int gd_count_per_edge(gd_graph *g, uint64_t *out, int out_flags, gd_u128 global_out[15]);

/* Batch of independent graphs packed in one CSR: graph i owns node ids
 * graph_node_ptr[i] .. graph_node_ptr[i+1]-1, and its edges stay inside that
 * range.  row_ptr has graph_node_ptr[num_graphs]+1 entries, col_idx holds
 * global node ids.  out: uint64[num_graphs][15] per-graph global counts
 * (host memory, or device memory with GD_OUT_DEVICE in flags).  Every
 * graph's counts fit uint64 when it has at most 65,535 nodes; a larger
 * graph in the batch is refused with GD_EOVERFLOW.  flags: GD_DEVICE_PTRS
 * (inputs on the device), GD_VALIDATE, GD_OUT_DEVICE.  Runs on the context's
 * stream.  Synchronous. */
int gd_count_batch(gd_ctx *ctx, int32_t num_graphs, const int32_t *graph_node_ptr,
                   const int32_t *row_ptr, const int32_t *col_idx, int flags,
                   uint64_t *out);

/* The counts of gd_count_batch for graphs that sit in device memory as
 * separate CSRs (the collections of small graphs of Sec. 6, e.g. requests
 * uploaded one by one): graph i has num_nodes[i] nodes and num_slots[i]
 * stored entries, its row_ptr at row_ptrs[i] and its col_idx (local ids
 * 0..n_i-1) at col_idxs[i].  row_ptrs and col_idxs are DEVICE arrays of
 * num_graphs DEVICE pointers; num_nodes and num_slots are HOST arrays (the
 * packed offsets are formed from them without a device round trip).  One
 * gather kernel packs the graphs into one CSR (row offsets shifted by each
 * graph's slot offset, ids by its node offset) held by the context; then the
 * validation and the persistent counting launch of gd_count_batch run on it.
 * out: DEVICE, num_graphs x 15 uint64.  flags: GD_CAPTURE records the gather,
 * the validation and the count as one CUDA graph, replayed while the
 * pointers and sizes stay the same (graphs of at most 1024 nodes).  Errors as
 * gd_count_batch, plus GD_EINVAL when a graph's row_ptr does not start at 0
 * or does not end at its slot count.  Runs on the context's stream;
 * synchronous.  The caller keeps every array alive during the call. */
int gd_count_batch_gather(gd_ctx *ctx, int32_t num_graphs, const int32_t *const *row_ptrs,
                          const int32_t *const *col_idxs, const int32_t *num_nodes,
                          const int64_t *num_slots, int flags, uint64_t *out);

/* ------------------------------------------------------------------------
 * Measurement and memory hooks (no counterpart in the paper).
 * ------------------------------------------------------------------------ */

/* Per-kernel device time collected between gd_profile_begin and
 * gd_profile_end: CUDA events recorded on each graph's stream around every
 * kernel launch of this context.  name: kernel name; ms_total: summed device
 * time; launches: number of launches. */
typedef struct gd_stage_stat {
    char name[40];
    double ms_total;
    int64_t launches;
} gd_stage_stat;

/* Start collecting (discards what was collected before). */
int gd_profile_begin(gd_ctx *ctx);

/* Stop, wait for the recorded events, and aggregate per kernel name into
 * out[0 .. min(*num_out, max_out)).  *num_out receives the number of distinct
 * kernels.  out may be NULL to query the count. */
int gd_profile_end(gd_ctx *ctx, gd_stage_stat *out, int32_t max_out, int32_t *num_out);

/* Number of kernels this context has launched since gd_init. */
int64_t gd_kernel_launches(const gd_ctx *ctx);

/* Device blocks of destroyed graphs stay cached in the context for reuse by
 * later graphs of the same shape (they count against the budget; a budget
 * refusal first releases them).  This call returns them to CUDA now. */
int gd_pool_release(gd_ctx *ctx);

/* ------------------------------------------------------------------------
 * Autotuning (the paper's "auto-optimizer", Sec. 5.2, chooses data
 * structures by graph density; here: the kernel cut-overs).
 * ------------------------------------------------------------------------ */

typedef struct gd_tune_result {
    gd_options best;           /* fastest options found (now the context's)  */
    double best_ms;            /* device time of one count with them        */
    double default_ms;         /* device time with the options before tuning */
    int32_t trials;            /* option sets timed                          */
    int32_t reserved;
} gd_tune_result;

/* Time counts of g (per_edge != 0: gd_count_per_edge, else gd_count_global)
 * under up to max_trials option sets -- shared-memory wedge table size,
 * bitmap out-degree limit, hub wedge threshold, then the medium tier's
 * cluster cut-over -- with CUDA events on the
 * graph's stream, and make the fastest the context's options.  The counts
 * are identical under every option set; only the time differs. */
int gd_autotune(gd_graph *g, int per_edge, int32_t max_trials, gd_tune_result *res);

/* The same for the batched path (Sec. 6 collections): time gd_count_batch on
 * this batch (arguments as gd_count_batch; out receives its counts) under
 * every batch_threads value (host wall time of the synchronous call, best of
 * two), and keep the fastest in the context's options; res->best.batch_threads
 * is the choice.  Counts are identical under every value. */
int gd_autotune_batch(gd_ctx *ctx, int32_t num_graphs, const int32_t *graph_node_ptr, const int32_t *row_ptr,
                      const int32_t *col_idx, int flags, uint64_t *out, gd_tune_result *res);

/* ------------------------------------------------------------------------
 * Serving: a request loop with continuous batching (no counterpart in the
 * paper; the counts of every request are those of gd_count_global).
 * ------------------------------------------------------------------------ */

/* One counting request.  row_ptr / col_idx are HOST memory in the CSR format
 * above; gd_submit copies them, so the caller may free them on return. */
typedef struct gd_request_desc {
    int32_t n;                 /* rows                                       */
    int64_t nnz;               /* row_ptr[n]                                 */
    const int32_t *row_ptr;
    const int32_t *col_idx;
    int32_t mode;              /* 0: the 15 global counts (the only mode)    */
    int32_t reserved;
} gd_request_desc;

/* Timing of a finished request, in milliseconds since the service started. */
typedef struct gd_req_stats {
    double submit_ms;          /* gd_submit returned                         */
    double start_ms;           /* a worker took it                           */
    double end_ms;             /* its counts were ready                      */
    size_t footprint;          /* device bytes reserved for it from admission
                                  (CSR upload) to the end of its count        */
    int32_t slot;              /* worker that ran it                         */
    int32_t batched;           /* 1 if it ran inside a batched launch        */
} gd_req_stats;

/* A request that does not fit the budget may be passed by later requests
 * that do, for at most this long after it was first passed at the head of
 * the queue; then no other request is admitted until it fits. */
#define GD_SERVE_MAX_BYPASS_MS 50.0

/* Start the service of a context: a stager thread and `slots` worker
 * threads, each worker with its own CUDA stream and device-block cache, so
 * their requests overlap on the GPU.  hbm_budget_bytes (0: the context's
 * budget; 0 there too: 45% of the device memory free at this call, the
 * workers' block caches being kept within budget / slots each) bounds the
 * sum of the estimated footprints of the admitted requests
 * (gd_footprint_estimate); a request larger than it is refused by
 * gd_submit with GD_ENOMEM.  The stager admits a
 * request when it fits, reserving its footprint and uploading its CSR to the
 * device, where it stays until the request's counts are done; workers count
 * admitted requests straight from their device CSRs.  gd_submit starts a
 * service with 4 slots if none is running. */
int gd_serve_start(gd_ctx *ctx, int32_t slots, size_t hbm_budget_bytes);

/* Queue a request; *id identifies it.  Non-blocking.  GD_ENOMEM: the request
 * alone exceeds the budget; GD_EINVAL: malformed descriptor (the full CSR
 * check runs on the device later and is reported by gd_poll). */
int gd_submit(gd_ctx *ctx, const gd_request_desc *desc, gd_req *id);

/* GD_EAGAIN while the request is queued or running.  Once it is done: its
 * status (GD_OK, or the error of its count) is returned, out (nullable) gets
 * the 15 counts, st (nullable) its timing, and the request is released. */
int gd_poll(gd_ctx *ctx, gd_req id, gd_u128 out[15], gd_req_stats *st);

/* Block until the request is done (timeout_ms < 0: no limit); GD_ETIMEDOUT
 * if the limit passes first.  Does not release it (call gd_poll). */
int gd_wait(gd_ctx *ctx, gd_req id, int32_t timeout_ms);

/* Queue length, requests running, bytes admitted, and how many launches were
 * batched / single-graph so far. */
int gd_serve_stats(gd_ctx *ctx, int64_t *queued, int64_t *running, size_t *inflight_bytes,
                   int64_t *batched_launches, int64_t *single_launches);

/* Finish the queued requests, stop the workers, release the service. */
int gd_serve_stop(gd_ctx *ctx);

/* Estimated device bytes of one count of a graph with n rows and nnz slots
 * (the admission footprint): CSR copy plus every work array;
 * per_edge adds the per-edge arrays and the staged output. */
int gd_footprint_estimate(gd_ctx *ctx, int32_t n, int64_t nnz, int per_edge, size_t *bytes);

/* ------------------------------------------------------------------------
 * Local update of the counts when one edge is inserted or deleted (the
 * paper's closing remarks on dynamic graphs; only the subsets that contain
 * both end nodes change).
 * ------------------------------------------------------------------------ */

/* Toggle the pair {u, v} of g (delete it if it is an edge, insert it if not)
 * and report, per graphlet (Table 1 order), how many 3-/4-node subsets enter
 * it (gain) and leave it (loss): the counts of the toggled graph are
 * count + gain - loss, exactly.  Work is proportional to the neighbourhoods
 * of u and v and their neighbours' lists (no full recount).  The graph
 * itself is not modified; *was_edge (nullable) says which way the toggle
 * went.  GD_EINVAL if u == v or either is out of range. */
int gd_toggle_delta(gd_graph *g, int32_t u, int32_t v, gd_u128 gain[15], gd_u128 loss[15], int *was_edge);

/* ------------------------------------------------------------------------
 * Ranking by graphlet counts (Sec. 6 and Fig. 6: the edges and nodes with
 * the most triangles, 4-cliques, stars, ... surfaced for analysis).
 * ------------------------------------------------------------------------ */

/* The k largest of values[i * stride], 0 <= i < count (uint64): indices to
 * idx_out (int64) and values to val_out (nullable), both host arrays of k
 * entries, ordered by value descending and, among equal values, by index
 * ascending, so the answer is unique.  values is device memory when flags
 * has GD_DEVICE_PTRS, else host memory (copied in).  Work runs on
 * cuda_stream (NULL: legacy default stream); scratch comes from the
 * context's cache and budget.  0 <= k <= count, stride >= 1.
 * For the edges with the most 4-cliques: values = per-edge matrix + 4,
 * stride 15, count = m (row i is the i-th edge of gd_count_per_edge). */
int gd_topk(gd_ctx *ctx, const uint64_t *values, int64_t count, int64_t stride, int flags, int64_t k,
            int64_t *idx_out, uint64_t *val_out, void *cuda_stream);

/* For every node v, the sum over the edges e incident to v of
 * per_edge[e * 15 + column] (per_edge: the m x 15 matrix gd_count_per_edge
 * wrote for this graph; device memory with GD_DEVICE_PTRS in flags, else
 * host).  Column 0 gives twice the number of triangles at v; column 4 three
 * times the 4-cliques at v.  node_out: n uint64, device memory with
 * GD_OUT_DEVICE in out_flags, else host.  The graph must have been counted
 * per edge (GD_EINVAL otherwise). */
int gd_node_sums(gd_graph *g, const uint64_t *per_edge, int flags, int column, uint64_t *node_out,
                 int out_flags);

/* ------------------------------------------------------------------------
 * Graphlet frequency features (Sec. 6: graph classification with graphlet
 * features; Table 1 sizes k = 2, 3, 4).
 * ------------------------------------------------------------------------ */

/* The 17 normalised frequencies of a graph with n nodes, m edges and the
 * 15 exact counts of gd_count_global:
 *   out[0] = m / C(n,2), out[1] = (C(n,2) - m) / C(n,2)      (k = 2)
 *   out[2..5]  = g31..g34 / C(n,3)
 *   out[6..16] = g41..g4_11 / C(n,4)
 * Each value is the exact rational rounded once to the nearest double, ties
 * to even; a size with no subsets (C(n,k) = 0) gives 0.  Host only.
 * GD_EINVAL for n < 0, m < 0 or m > C(n,2). */
int gd_gfd(int64_t n, int64_t m, const gd_u128 counts[15], double out[17]);

/* The same for the num_graphs graphs of a batch on the GPU: graph_node_ptr
 * and row_ptr as given to gd_count_batch, counts the num_graphs x 15 uint64
 * it wrote, out num_graphs x 17 doubles.  All DEVICE pointers (flags must
 * have GD_DEVICE_PTRS); runs on cuda_stream and waits for it. */
int gd_gfd_batch(gd_ctx *ctx, int32_t num_graphs, const int32_t *graph_node_ptr, const int32_t *row_ptr,
                 const uint64_t *counts, int flags, double *out, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Counting without allocating (no counterpart in the paper).
 *
 * For callers that must not allocate device memory: code running next to a
 * latency-critical pipeline (cudaMalloc/cudaFree may synchronize the device
 * and stall the other streams), plug-ins whose host framework owns every
 * device byte through its own allocator, and processes under a fixed device
 * memory quota.  The scratch is one static array inside libgd's device image
 * (GD_STATIC_SCRATCH_BYTES on every GPU where that image is loaded, held
 * until the process exits); nothing is allocated per call.  The CUDA runtime
 * loads device code lazily by default, so the first call on a device (its
 * set-up step below) may load the image and reserve the array: make that
 * call early, outside any latency-critical section.
 * ------------------------------------------------------------------------ */
#define GD_STATIC_MAX_N 32768              /* largest n accepted            */
#define GD_STATIC_MAX_NNZ 262144           /* largest nnz (= 2|E|) accepted */
#define GD_STATIC_SCRATCH_BYTES 5505024    /* 5.25 MiB of static scratch    */

/* The 15 global counts of gd_count_global (same order, exact), for a graph
 * with n <= GD_STATIC_MAX_N and nnz <= GD_STATIC_MAX_NNZ.  row_ptr, col_idx
 * and out (15 gd_u128) are DEVICE pointers owned by the caller; the kernel
 * runs on cuda_stream (NULL: legacy default stream) on the current device and
 * the call waits for it.  Returns GD_EOVERFLOW for larger graphs (nothing is
 * launched), GD_EINVAL for a malformed CSR (same checks as gd_create_csr),
 * GD_ECUDA on a CUDA error.
 * The first call on each device looks up the scratch address
 * (cudaGetSymbolAddress) with that device current: make it before any stream
 * capture on that device.  All calls on a device share the one scratch
 * array, which keeps the last call's contents (each call clears what must
 * start at zero): calls whose kernels overlap on the GPU race and must be
 * serialized by the caller. */
int gd_count_global_static(int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                           gd_u128 *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* GD_H */
