// gd_api.cu -- the C ABI of libgd (declared in include/gd.h): contexts,
// graphs, device memory, validation and the count calls.  Every step of the
// counting runs in the kernels of gd_count.cu / gd_batch.cu; this file only
// allocates, orders launches and reports errors.
#include <cuda_runtime.h>

#include <chrono>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "gd_internal.h"

using namespace gdi;

namespace {

int fail(gd_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

int cuda_fail(gd_ctx *ctx, cudaError_t e, const char *where) {
    return fail(ctx, GD_ECUDA, "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

#define GD_CK(ctx, call)                                              \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);    \
    } while (0)

size_t round_block(size_t bytes) { return (bytes + 255) & ~(size_t)255; }

// Release every cached block of the context's pool.
void trim_pool(gd_ctx *ctx) {
    for (auto &kv : ctx->pool) cudaFree(kv.second);
    ctx->in_use -= std::min(ctx->in_use, ctx->pooled);
    ctx->pool.clear();
    ctx->pooled = 0;
}

// Device allocation accounted against the context budget.  Blocks released
// by destroyed graphs are cached in the context and reused for the same
// rounded size (a later graph of the same shape allocates nothing).
int ctx_alloc(gd_ctx *ctx, void **p, size_t bytes) {
    bytes = round_block(bytes ? bytes : 16);
    auto it = ctx->pool.find(bytes);
    if (it != ctx->pool.end()) {
        *p = it->second;
        ctx->pool.erase(it);
        ctx->pooled -= bytes;        // stays in in_use: moves from cached to live
        return GD_OK;
    }
    if (ctx->budget && ctx->in_use + bytes > ctx->budget) trim_pool(ctx);
    if (ctx->budget && ctx->in_use + bytes > ctx->budget)
        return fail(ctx, GD_ENOMEM, "device budget exceeded: need %zu more bytes, %zu of %zu in use",
                    bytes, ctx->in_use, ctx->budget);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess && !ctx->pool.empty()) {
        cudaGetLastError();
        trim_pool(ctx);
        e = cudaMalloc(p, bytes);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(ctx, GD_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    ctx->in_use += bytes;
    return GD_OK;
}

void ctx_release(gd_ctx *ctx, void *p, size_t bytes) {
    if (!p) return;
    ctx->pool.emplace(round_block(bytes ? bytes : 16), p);
    ctx->pooled += round_block(bytes ? bytes : 16);
}

int dalloc(gd_graph *g, void **p, size_t bytes) {
    int rc = ctx_alloc(g->ctx, p, bytes);
    if (rc == GD_OK) {
        g->ws.bytes += round_block(bytes ? bytes : 16);
        g->ws.blocks.emplace_back(*p, round_block(bytes ? bytes : 16));
    }
    return rc;
}

template <typename T>
int dalloc_n(gd_graph *g, T **p, int64_t count) {
    return dalloc(g, (void **)p, sizeof(T) * (size_t)std::max<int64_t>(count, 1));
}

void free_workspace(gd_graph *g) {
    Workspace &w = g->ws;
    if (g->ctx)
        for (auto &b : w.blocks) ctx_release(g->ctx, b.first, b.second);
    w = Workspace();
}

// Give one block of this graph back to the context pool.
void release_block(gd_graph *g, void *p) {
    auto &bl = g->ws.blocks;
    for (size_t i = 0; i < bl.size(); i++)
        if (bl[i].first == p) {
            ctx_release(g->ctx, p, bl[i].second);
            g->ws.bytes -= bl[i].second;
            bl.erase(bl.begin() + i);
            return;
        }
}

int32_t tricap_for(gd_graph *g, int variant) {
    int64_t cap = g->max_deg;
    if (variant != GD_VARIANT_LITERAL) {
        // |Tri+(a,b)| <= out-degree of b <= sqrt(2|E|) under the degree order
        int64_t s = (int64_t)std::ceil(std::sqrt((double)g->nnz)) + 1;
        cap = std::min(cap, s);
    }
    return (int32_t)std::max<int64_t>(cap, 1);
}

// Every work array of a graph, as (pointer, bytes): one list serves both the
// allocation and the footprint estimate used for admission.
struct AllocSpec {
    void **ptr;
    size_t bytes;
};

template <typename T>
AllocSpec spec(T **p, int64_t count) {
    return AllocSpec{(void **)p, sizeof(T) * (size_t)std::max<int64_t>(count, 1)};
}

// part 0: arrays of every count call; part 1: dense wedge tables; part 2:
// per-edge mode arrays
void workspace_specs(Workspace &w, int64_t n, int64_t m, int64_t nnz, int32_t slots, int part,
                     std::vector<AllocSpec> &out) {
    if (part == 0) {
        out.push_back(spec(&w.first_up, n));
        out.push_back(spec(&w.eoff, n + 1));
        out.push_back(spec(&w.eu, m));
        out.push_back(spec(&w.ev, m));
        out.push_back(spec(&w.eslot, m));
        out.push_back(spec(&w.mate, nnz));
        out.push_back(spec(&w.tslot, nnz));
        out.push_back(spec(&w.tcred, nnz));
        out.push_back(spec(&w.nd, nnz));
        out.push_back(spec(&w.vlist, n));
        out.push_back(spec(&w.hubs, n));
        out.push_back(spec(&w.clist, 4 * n));
        out.push_back(spec(&w.counters, (int64_t)C_NUM));
        out.push_back(spec(&w.dag_off, n + 1));
        out.push_back(spec(&w.dag_col, m));
        out.push_back(spec(&w.dag_slot, m));
        out.push_back(spec(&w.dag_nd, m));
        out.push_back(spec(&w.sums, 2 * (int64_t)(S_NUM + X_NUM)));
        out.push_back(spec(&w.result, 30));
        out.push_back(spec(&w.scan_tmp, 3 * (n + 1) + 4096));
        out.push_back(spec(&w.cacc, nnz));
        out.push_back(spec(&w.yacc, nnz));
        out.push_back(spec(&w.mlist, n));
        out.push_back(spec(&w.west, n + 1));
        out.push_back(spec(&w.tlist, n));
    } else if (part == 1) {
        out.push_back(spec(&w.wtab, (int64_t)slots * n));
    } else {
        out.push_back(spec(&w.tnode, n));
        out.push_back(spec(&w.s1, n));
        out.push_back(spec(&w.au, m));
        out.push_back(spec(&w.dt, m));
        out.push_back(spec(&w.qcred, 2 * nnz));     // (Q, R) credit pair per slot
        out.push_back(spec(&w.toff, n + 1));
        out.push_back(spec(&w.tcnt, n));
    }
}

int alloc_specs(gd_graph *g, const std::vector<AllocSpec> &sp) {
    for (const AllocSpec &a : sp) {
        int rc = dalloc(g, a.ptr, a.bytes);
        if (rc) return rc;
    }
    return GD_OK;
}

// Allocate everything a count call needs (kept across calls; contents are
// recomputed by every call).
int ensure_workspace(gd_graph *g, bool per_edge) {
    Workspace &w = g->ws;
    const int64_t n = g->n, m = g->m, nnz = g->nnz;
    int rc;
    if (!w.status) {
        if ((rc = dalloc_n(g, &w.status, 4))) return rc;
        GD_CK(g->ctx, cudaMemsetAsync(w.status, 0, 4 * sizeof(int32_t), g->stream));
    }
    std::vector<AllocSpec> sp;
    if (!w.first_up) {
        workspace_specs(w, n, m, nnz, 0, 0, sp);
        if ((rc = alloc_specs(g, sp))) return rc;
        sp.clear();
    }
    if (!w.wtab && n > 0) {
        w.wtab_ctas = table_slots(g);
        workspace_specs(w, n, m, nnz, w.wtab_ctas, 1, sp);
        if ((rc = alloc_specs(g, sp))) return rc;
        sp.clear();
        GD_CK(g->ctx, cudaMemsetAsync(w.wtab, 0, sizeof(uint32_t) * (size_t)w.wtab_ctas * n, g->stream));
    }
    if (per_edge && !w.tnode) {
        workspace_specs(w, n, m, nnz, 0, 2, sp);
        if ((rc = alloc_specs(g, sp))) return rc;
    }
    return GD_OK;
}

}  // namespace

namespace gdi {

// Device bytes the medium tier's tables may take for a graph of nnz slots
// (64 per slot, at least 64 MB): fewer CTAs share the tier beyond that.
int64_t medium_table_limit(int64_t nnz) { return std::max<int64_t>(int64_t(64) << 20, 64 * nnz); }

// Device bytes a graph of n rows and nnz slots holds after one count call
// (CSR copy included); per_edge adds the per-edge arrays and the staging of
// a host-side output matrix.
size_t estimate_footprint(gd_ctx *ctx, int64_t n, int64_t nnz, bool per_edge, bool host_out) {
    Workspace w;
    gd_graph g;
    g.ctx = ctx; g.n = (int32_t)n; g.nnz = nnz; g.m = nnz / 2;
    std::vector<AllocSpec> sp;
    workspace_specs(w, n, nnz / 2, nnz, 0, 0, sp);
    if (n > 0) workspace_specs(w, n, nnz / 2, nnz, table_slots(&g), 1, sp);
    if (per_edge) workspace_specs(w, n, nnz / 2, nnz, 0, 2, sp);
    size_t b = round_block(sizeof(int32_t) * (size_t)(n + 1 + nnz)) + round_block(16);   // CSR + status
    for (const AllocSpec &a : sp) b += round_block(a.bytes);
    if (per_edge && host_out) b += round_block(sizeof(uint64_t) * 15 * (size_t)(nnz / 2));
    if (n > 0) b += round_block(clique_pairs_bound(ctx ? ctx->num_sms : 152, n));
    if (n > 0) {
        // medium-tier tables: W(u) <= min(2^hub, nnz) entries, two per SM,
        // within the per-graph limit
        const int64_t hub = std::max<int64_t>(int64_t(1) << (ctx ? ctx->opt.hub_wedges_log2 : 17), n / 8);
        int64_t cap = 1024;
        while (cap < 2 * std::min<int64_t>(hub, nnz)) cap <<= 1;
        const int64_t ctas = std::min<int64_t>(2 * (ctx ? ctx->num_sms : 152), n);
        b += round_block((size_t)std::min<int64_t>(8 * cap * ctas, std::max<int64_t>(8 * cap, medium_table_limit(nnz))));
    }
    if (per_edge) b += round_block(sizeof(unsigned long long) * 2 * (size_t)nnz);   // triangle records (typical)
    if (n > 0) {
        // pull form of the hub tier: node masks, chunks, heavy-node counters
        const size_t items = (size_t)(nnz / 64 + nnz / 1024 + 1), heavy = (size_t)(nnz / 1024 + 1);
        b += round_block(8 * (size_t)n) + round_block(12 * items) + round_block(4 * heavy) +
             round_block(256 * heavy) + round_block(8);
    }
    g.ws = Workspace();
    return b;
}

// Scratch through the context's cache and budget (for calls outside a
// graph's workspace).
int scratch_alloc(gd_ctx *ctx, void **p, size_t bytes) { return ctx_alloc(ctx, p, bytes); }
void scratch_release(gd_ctx *ctx, void *p, size_t bytes) { ctx_release(ctx, p, bytes); }

}  // namespace gdi

namespace {

// Per-CTA scratch of the large out-list clique kernel (out-lists above the
// shared-memory limit), sized from the largest out-degree.
int ensure_clique_scratch(gd_graph *g, const int32_t *cnt) {
    Workspace &w = g->ws;
    const int32_t dm = ((cnt[C_MAXDP] + 31) / 32) * 32;
    const int32_t ctas = std::min<int32_t>(cnt[C_CL0 + 3], g->ctx->num_sms);
    const size_t stride = (clique_big_bytes(dm) + 255) & ~(size_t)255;
    const size_t need = stride * (size_t)ctas;
    if (w.cbig && w.cbig_bytes >= need && w.cbig_dm >= dm) {
        w.cbig_ctas = ctas;
        return GD_OK;
    }
    if (w.cbig) { release_block(g, w.cbig); w.cbig = nullptr; }
    int rc = dalloc(g, (void **)&w.cbig, need);
    if (rc) return rc;
    w.cbig_bytes = need; w.cbig_stride = stride; w.cbig_dm = dm; w.cbig_ctas = ctas;
    return GD_OK;
}

// Per-team triangle records of the clique kernels, sized for this graph's
// bucket counts.
int ensure_pairs(gd_graph *g, const int32_t *cnt) {
    Workspace &w = g->ws;
    size_t need = 0;
    GD_CK(g->ctx, clique_pairs_bytes(g, cnt, &need));
    if (w.pairs && w.pairs_bytes >= need) return GD_OK;
    if (w.pairs) { release_block(g, w.pairs); w.pairs = nullptr; w.pairs_bytes = 0; }
    if (need == 0) return GD_OK;
    int rc = dalloc(g, (void **)&w.pairs, need);
    if (rc) return rc;
    w.pairs_bytes = need;
    return GD_OK;
}

// Triangle records kept from the 4-clique pass for the triangle-sum pass
// (per-edge mode): up to `total` entries, capped at 16 bytes per CSR slot
// plus 1 GB; nodes past the cap scan again.  A failed allocation only
// disables the records.
int ensure_records(gd_graph *g, int64_t total) {
    Workspace &w = g->ws;
    const int64_t cap = std::min<int64_t>(total, 2 * g->nnz + (int64_t(1) << 27));
    if (w.recs && w.recs_cap >= cap) return GD_OK;
    if (w.recs) { release_block(g, w.recs); w.recs = nullptr; w.recs_cap = 0; }
    if (cap <= 0) return GD_OK;
    if (dalloc(g, (void **)&w.recs, sizeof(unsigned long long) * (size_t)cap) != GD_OK) {
        w.recs = nullptr;
        g->ctx->err.clear();
        return GD_OK;
    }
    w.recs_cap = cap;
    return GD_OK;
}

// Per-CTA tables of the medium tier: a power of two >= 2 W entries for the
// largest medium vertex (a vertex uses the first 1.5 W + 1024 or fewer), one per CTA (two per SM, fewer when there are fewer
// vertices or the tables would pass medium_table_limit), all entries empty
// (all ones).
int ensure_medium_scratch(gd_graph *g, const int32_t *cnt) {
    Workspace &w = g->ws;
    int64_t cap = 1024;
    while (cap < 2 * w.medium_wmax) cap <<= 1;
    int64_t ctas = std::min<int64_t>(2 * g->ctx->num_sms, cnt[C_MEDIUM]);
    const int64_t limit = medium_table_limit(g->nnz);
    while (ctas > 1 && ctas * cap * 8 > limit) ctas--;
    if (w.mtab && w.mtab_cap >= cap && w.mtab_ctas >= ctas) return GD_OK;
    if (w.mtab) { release_block(g, w.mtab); w.mtab = nullptr; w.mtab_cap = 0; w.mtab_ctas = 0; }
    int rc = dalloc(g, (void **)&w.mtab, sizeof(unsigned long long) * (size_t)(ctas * cap));
    if (rc) return rc;
    GD_CK(g->ctx, cudaMemsetAsync(w.mtab, 0xff, sizeof(unsigned long long) * (size_t)(ctas * cap), g->stream));
    w.mtab_cap = cap;
    w.mtab_ctas = (int32_t)ctas;
    return GD_OK;
}

// Flat neighbour lists of the hubs: row offsets (from the hub list), then
// lengths, prefix and scan scratch sized to the hubs' concatenated rows.
int ensure_hub_scratch(gd_graph *g, const int32_t *cnt) {
    Workspace &w = g->ws;
    const int32_t nh = cnt[C_HUB];
    int rc;
    if (!w.pull_mask) {
        // hub masks of the pull form; zero at rest, cleared here once and by
        // every pull batch after use
        // a node of degree >= 64 takes at least 64 slots: at most nnz / 64 of
        // them, with at most nnz / 1024 further chunks; a node of several
        // chunks has degree > 1024
        const int64_t items = g->nnz / 64 + g->nnz / 1024 + 1, heavy = g->nnz / 1024 + 1;
        if ((rc = dalloc_n(g, &w.pull_mask, (int64_t)g->n))) return rc;
        if ((rc = dalloc_n(g, &w.pull_items, 3 * items))) return rc;
        if ((rc = dalloc_n(g, &w.pull_heavy_y, heavy))) return rc;
        if ((rc = dalloc_n(g, &w.pull_heavy_cnt, 64 * heavy))) return rc;
        if ((rc = dalloc_n(g, &w.pull_counts, 2))) return rc;
        GD_CK(g->ctx, cudaMemsetAsync(w.pull_mask, 0, sizeof(unsigned long long) * (size_t)g->n, g->stream));
        GD_CK(g->ctx, cudaMemsetAsync(w.pull_heavy_cnt, 0, sizeof(uint32_t) * 64 * (size_t)heavy, g->stream));
    }
    if (!w.hub_off || w.hub_off_cap < nh + 1) {
        if (w.hub_off) { release_block(g, w.hub_off); w.hub_off = nullptr; }
        if ((rc = dalloc_n(g, &w.hub_off, (int64_t)nh + 1))) return rc;
        w.hub_off_cap = nh + 1;
    }
    int64_t flat = 0;
    GD_CK(g->ctx, run_hub_offsets(g, nh, &flat));
    w.hub_flat = flat;
    if (w.hub_len && w.hub_flat_cap >= flat) return GD_OK;
    if (w.hub_len) {
        release_block(g, w.hub_len); release_block(g, w.hub_pre); release_block(g, w.hub_scan_tmp);
        w.hub_len = w.hub_pre = w.hub_scan_tmp = nullptr;
    }
    if ((rc = dalloc_n(g, &w.hub_len, flat))) return rc;
    if ((rc = dalloc_n(g, &w.hub_pre, flat + 1))) return rc;
    if ((rc = dalloc_n(g, &w.hub_scan_tmp, 2 * (flat / 2048 + 1) + 4096))) return rc;
    w.hub_flat_cap = flat;
    return GD_OK;
}

// Candidate buffers of the literal kernel.
int ensure_tribuf(gd_graph *g, int variant) {
    Workspace &w = g->ws;
    const int64_t need = (int64_t)tribuf_warps(g->ctx->num_sms) * tricap_for(g, variant) * 3;
    if (w.tribuf_words >= need) return GD_OK;
    if (w.tribuf) { release_block(g, w.tribuf); w.tribuf = nullptr; w.tribuf_words = 0; }
    int rc = dalloc_n(g, &w.tribuf, need);
    if (rc) return rc;
    w.tribuf_words = need;
    return GD_OK;
}

int resolve_variant(gd_graph *g) {
    int v = g->ctx->opt.variant;
    if (v == GD_VARIANT_LITERAL) return GD_VARIANT_LITERAL;
    return GD_VARIANT_ORIENTED;
}

int check_status(gd_graph *g, const int32_t *st) {
    if (st[0] == 0) return GD_OK;
    if (st[0] & ERR_CAPACITY) return fail(g->ctx, GD_EARITH, "internal: a work buffer was too small");
    if (st[0] & ERR_TIMEOUT) return fail(g->ctx, GD_ETIMEDOUT, "a bounded device wait gave up");
    return fail(g->ctx, GD_EARITH, "inconsistent counts (status bits 0x%x): the graph is not a simple "
                "undirected CSR, or an internal error", st[0]);
}

int read_results(gd_graph *g, gd_u128 *out) {
    unsigned long long res[30];
    int32_t st[4];
    GD_CK(g->ctx, cudaMemcpyAsync(res, g->ws.result, sizeof(res), cudaMemcpyDeviceToHost, g->stream));
    GD_CK(g->ctx, cudaMemcpyAsync(st, g->ws.status, sizeof(st), cudaMemcpyDeviceToHost, g->stream));
    GD_CK(g->ctx, cudaStreamSynchronize(g->stream));
    int rc = check_status(g, st);
    if (rc) return rc;
    if (out)
        for (int i = 0; i < 15; i++) { out[i].lo = res[2 * i]; out[i].hi = res[2 * i + 1]; }
    return GD_OK;
}

cudaEvent_t take_event(gd_ctx *c) {
    if (!c->evpool.empty()) {
        cudaEvent_t e = c->evpool.back();
        c->evpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace

namespace gdi {

void prof_begin(gd_ctx *c, cudaStream_t st, const char *name) {
    c->launches++;
    if (!c->prof) return;
    ProfRec r;
    r.name = name;
    r.a = take_event(c);
    r.b = take_event(c);
    cudaEventRecord(r.a, st);
    c->recs.push_back(r);
}

void prof_end(gd_ctx *c, cudaStream_t st) {
    if (!c->prof || c->recs.empty()) return;
    cudaEventRecord(c->recs.back().b, st);
}

struct BatchGraph {
    int32_t G = 0, N = 0;
    int64_t nnz = 0;
    const void *gnp = nullptr, *rp = nullptr, *ci = nullptr;
    const void *rps = nullptr, *cis = nullptr, *eoff = nullptr;   // gather step (gd_count_batch_gather)
    std::vector<int32_t> eoff_host;
    void *out = nullptr;
    std::vector<int32_t> gnp_host;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int32_t *d_misc = nullptr, *d_big = nullptr;
    size_t misc_bytes = 0, big_bytes = 0;
    int32_t *h_status = nullptr;      // pinned
};

void batch_graph_destroy(gd_ctx *ctx) {
    BatchGraph *b = ctx->bgraph;
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->d_misc) ctx_release(ctx, b->d_misc, b->misc_bytes);
    if (b->d_big) ctx_release(ctx, b->d_big, b->big_bytes);
    if (b->h_status) cudaFreeHost(b->h_status);
    delete b;
    ctx->bgraph = nullptr;
}

}  // namespace gdi

extern "C" {

void gd_default_options(gd_options *opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->variant = GD_VARIANT_AUTO;
    opt->block_threads = 256;
    opt->ctas_per_sm = 0;
    opt->smem_table_max = 8192;
    opt->bitmap_max_outdeg = gdi::CL_D2;
    opt->hub_wedges_log2 = 17;
}

static int check_options(gd_options *o) {
    const int t = o->smem_table_max;
    if (t < 256 || t > 16384 || (t & (t - 1))) return GD_EINVAL;
    if (o->variant < 0 || o->variant > 2) return GD_EINVAL;
    if (o->bitmap_max_outdeg == 0) o->bitmap_max_outdeg = gdi::CL_D2;
    if (o->hub_wedges_log2 == 0) o->hub_wedges_log2 = 17;
    if (o->bitmap_max_outdeg < 2 || o->bitmap_max_outdeg > gdi::CL_D2 || o->hub_wedges_log2 < 4 ||
        o->hub_wedges_log2 > 40) return GD_EINVAL;
    if (o->hub_pull < GD_PULL_AUTO || o->hub_pull > GD_PULL_ALWAYS) return GD_EINVAL;
    if (o->batch_threads < 0 || o->batch_threads > 1024) return GD_EINVAL;
    if (o->medium_cluster_log2 < 0 || o->medium_cluster_log2 > 64) return GD_EINVAL;
    return GD_OK;
}

int gd_set_options(gd_ctx *ctx, const gd_options *opt) {
    if (!ctx || !opt) return GD_EINVAL;
    gd_options o = *opt;
    int rc = check_options(&o);
    if (rc) return fail(ctx, rc, "invalid options");
    ctx->opt = o;
    return GD_OK;
}

int gd_get_options(const gd_ctx *ctx, gd_options *opt) {
    if (!ctx || !opt) return GD_EINVAL;
    *opt = ctx->opt;
    return GD_OK;
}

int gd_init(gd_ctx **ctx_out, int device, size_t hbm_budget_bytes, const gd_options *opt) {
    if (!ctx_out) return GD_EINVAL;
    *ctx_out = nullptr;
    gd_ctx *ctx = new (std::nothrow) gd_ctx();
    if (!ctx) return GD_ENOMEM;
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    gd_default_options(&ctx->opt);
    if (opt) {
        ctx->opt = *opt;
        if (check_options(&ctx->opt)) {
            delete ctx;
            return GD_EINVAL;
        }
    }
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return GD_ECUDA;
    }
    *ctx_out = ctx;
    return GD_OK;
}

void gd_destroy(gd_ctx *ctx) {
    if (!ctx) return;
    gdi::serve_destroy(ctx);
    cudaSetDevice(ctx->device);
    gdi::batch_graph_destroy(ctx);
    std::vector<gd_graph *> gs = ctx->graphs;
    for (gd_graph *g : gs) gd_destroy_graph(g);
    if (ctx->batch_buf) cudaFree(ctx->batch_buf);
    {
        gdi::GatherBufs &gb = ctx->gather;
        if (gb.gnp) ctx_release(ctx, gb.gnp, gb.gnp_bytes);
        if (gb.eoff) ctx_release(ctx, gb.eoff, gb.eoff_bytes);
        if (gb.rp) ctx_release(ctx, gb.rp, gb.rp_bytes);
        if (gb.ci) ctx_release(ctx, gb.ci, gb.ci_bytes);
        if (gb.misc) ctx_release(ctx, gb.misc, gb.misc_bytes);
        gb = gdi::GatherBufs();
    }
    trim_pool(ctx);
    for (auto &r : ctx->recs) { ctx->evpool.push_back(r.a); ctx->evpool.push_back(r.b); }
    for (cudaEvent_t ev : ctx->evpool) cudaEventDestroy(ev);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    for (int i = 0; i < gd_ctx::COPY_STREAMS; i++)
        if (ctx->copy_st[i]) cudaStreamDestroy(ctx->copy_st[i]);
    for (int i = 0; i <= gd_ctx::COPY_STREAMS; i++)
        if (ctx->copy_ev[i]) cudaEventDestroy(ctx->copy_ev[i]);
    delete ctx;
}

const char *gd_last_error(gd_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

// row_ptr[u] <= row_ptr[u + 1] for every row, checked a chunk at a time
// without early exits (so the compiler vectorises the comparisons); the first
// decreasing row goes to *bad_row.
static bool rows_nondecreasing(const int32_t *rp, int32_t n, int32_t *bad_row) {
    constexpr int32_t CH = 4096;
    for (int32_t u0 = 0; u0 < n; u0 += CH) {
        const int32_t u1 = n - u0 < CH ? n : u0 + CH;
        int dec = 0;
        for (int32_t u = u0; u < u1; u++) dec |= rp[u + 1] < rp[u];
        if (dec) {
            for (int32_t u = u0; u < u1; u++)
                if (rp[u + 1] < rp[u]) { *bad_row = u; return false; }
        }
    }
    return true;
}

int gd_create_csr(gd_ctx *ctx, int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx,
                  int flags, void *cuda_stream, gd_graph **out) {
    if (!ctx || !out) return GD_EINVAL;
    *out = nullptr;
    ctx->err.clear();
    if (n < 0 || nnz < 0) return fail(ctx, GD_EINVAL, "negative n or nnz");
    if (n == INT32_MAX) return fail(ctx, GD_EOVERFLOW, "n must be below INT32_MAX");
    if (nnz > INT32_MAX) return fail(ctx, GD_EOVERFLOW, "nnz %lld exceeds int32 slot ids", (long long)nnz);
    if (nnz % 2) return fail(ctx, GD_EINVAL, "nnz is odd: an undirected CSR stores both directions");
    if (!row_ptr || (nnz > 0 && !col_idx)) return fail(ctx, GD_EINVAL, "null CSR array");
    const bool dev = (flags & GD_DEVICE_PTRS) != 0;
    if ((flags & GD_BORROW) && !dev) return fail(ctx, GD_EINVAL, "GD_BORROW needs GD_DEVICE_PTRS");
    GD_CK(ctx, cudaSetDevice(ctx->device));
    if (!dev) {
        // O(1) checks of row_ptr on the host; the O(n) one runs below, while
        // the upload is in flight
        if (row_ptr[0] != 0) return fail(ctx, GD_EINVAL, "row_ptr[0] = %d, expected 0", row_ptr[0]);
        if ((int64_t)row_ptr[n] != nnz) return fail(ctx, GD_EINVAL, "row_ptr[n] = %d != nnz", row_ptr[n]);
    }
    gd_graph *g = new (std::nothrow) gd_graph();
    if (!g) return fail(ctx, GD_ENOMEM, "host allocation failed");
    g->ctx = ctx;
    g->n = n;
    g->nnz = nnz;
    g->m = nnz / 2;
    g->stream = (cudaStream_t)cuda_stream;
    ctx->graphs.push_back(g);
    int rc = GD_OK;
    if (dev && (flags & GD_BORROW)) {
        g->rp = const_cast<int32_t *>(row_ptr);
        g->ci = const_cast<int32_t *>(col_idx);
        g->borrowed = true;
    } else {
        size_t bytes = sizeof(int32_t) * ((size_t)n + 1 + (size_t)nnz);
        int arc = ctx_alloc(ctx, (void **)&g->rp, bytes);
        if (arc) {
            std::string msg = ctx->err;
            g->rp = nullptr;
            gd_destroy_graph(g);
            ctx->err = msg;
            return arc;
        }
        g->csr_bytes = bytes;
        g->ci = g->rp + (n + 1);
        cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        cudaError_t e = cudaMemcpyAsync(g->rp, row_ptr, sizeof(int32_t) * ((size_t)n + 1), kind, g->stream);
        if (e == cudaSuccess && nnz > 0)
            e = cudaMemcpyAsync(g->ci, col_idx, sizeof(int32_t) * (size_t)nnz, kind, g->stream);
        if (e != cudaSuccess) {
            rc = cuda_fail(ctx, e, "CSR upload");
            gd_destroy_graph(g);
            return rc;
        }
        int32_t bad_row = -1;
        if (!dev && !rows_nondecreasing(row_ptr, n, &bad_row)) {
            cudaStreamSynchronize(g->stream);     // the upload targets blocks about to be released
            gd_destroy_graph(g);
            return fail(ctx, GD_EINVAL, "row_ptr decreases at row %d", bad_row);
        }
    }
    if ((rc = dalloc_n(g, &g->ws.status, 4))) { gd_destroy_graph(g); return rc; }
    cudaError_t e = cudaMemsetAsync(g->ws.status, 0, 4 * sizeof(int32_t), g->stream);
    if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "status init"); gd_destroy_graph(g); return rc; }
    if (dev) {
        // row_ptr checks on the device copy: rp[0]==0 and rp[n]==nnz
        int32_t ends[2] = {0, 0};
        e = cudaMemcpyAsync(&ends[0], g->rp, sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], g->rp + n, sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "row_ptr read"); gd_destroy_graph(g); return rc; }
        if (ends[0] != 0 || (int64_t)ends[1] != nnz) {
            gd_destroy_graph(g);
            return fail(ctx, GD_EINVAL, "row_ptr[0]=%d, row_ptr[n]=%d, nnz=%lld", ends[0], ends[1], (long long)nnz);
        }
    }
    {   // the full check always runs: no kernel reads through an unchecked id
        int32_t bad_index = -1, bad_code = 0;
        e = validate_csr(g, &bad_index, &bad_code);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "validate"); gd_destroy_graph(g); return rc; }
        if (bad_code) {
            gd_destroy_graph(g);
            if (bad_index < 0)
                return fail(ctx, GD_EINVAL, "invalid CSR: some entry below the diagonal has no reverse entry "
                            "(every edge must be stored in both directions)");
            return fail(ctx, GD_EINVAL, "invalid CSR at row %d: rows must be strictly ascending, ids in [0,n), "
                        "no self-loops, and every edge stored in both directions", bad_index);
        }
    }
    e = max_degree(g, &g->max_deg);
    if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "max degree"); gd_destroy_graph(g); return rc; }
    *out = g;
    return GD_OK;
}

int gd_graph_info(const gd_graph *g, int32_t *n, int64_t *m) {
    if (!g) return GD_EINVAL;
    if (n) *n = g->n;
    if (m) *m = g->m;
    return GD_OK;
}

int gd_graph_footprint(const gd_graph *g, size_t *bytes) {
    if (!g || !bytes) return GD_EINVAL;
    *bytes = g->csr_bytes + g->ws.bytes;
    return GD_OK;
}

void gd_destroy_graph(gd_graph *g) {
    if (!g) return;
    gd_ctx *ctx = g->ctx;
    if (ctx) cudaSetDevice(ctx->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    free_workspace(g);
    if (!g->borrowed && g->rp && ctx) ctx_release(ctx, g->rp, g->csr_bytes);
    if (ctx) {
        auto &v = ctx->graphs;
        v.erase(std::remove(v.begin(), v.end(), g), v.end());
    }
    delete g;
}

// The whole single-graph path (rows a1-a8); per_edge writes the 15 columns
// to out_dev.
static int count_path(gd_graph *g, bool per_edge, uint64_t *out_dev) {
    gd_ctx *ctx = g->ctx;
    const int variant = resolve_variant(g);
    int rc = ensure_workspace(g, per_edge);
    if (rc) return rc;
    GD_CK(ctx, prepare_edges(g));
    g->prepared = true;                  // edge list (row order of the per-edge output) in place
    if (variant == GD_VARIANT_LITERAL) {
        if ((rc = ensure_tribuf(g, variant))) return rc;
        GD_CK(ctx, run_triangles_intersect(g));
        if (per_edge) GD_CK(ctx, run_per_edge_sums(g));
        GD_CK(ctx, run_literal(g));
        GD_CK(ctx, run_final(g, variant, per_edge, false, false, out_dev));
        GD_CK(ctx, run_complete(g, 0));
        return GD_OK;
    }
    int32_t cnt[C_NUM];
    GD_CK(ctx, run_schedule(g, cnt));
    if (cnt[C_CL0 + 3] > 0 && (rc = ensure_clique_scratch(g, cnt))) return rc;
    if (cnt[C_HUB] > 0 && (rc = ensure_hub_scratch(g, cnt))) return rc;
    if (cnt[C_MEDIUM] > 0 && (rc = ensure_medium_scratch(g, cnt))) return rc;
    if ((rc = ensure_pairs(g, cnt))) return rc;
    if (per_edge) {
        int64_t total = 0;
        GD_CK(ctx, run_tri_bound(g, &total));
        if ((rc = ensure_records(g, total))) return rc;
    }
    GD_CK(ctx, run_triangles_cliques(g, per_edge, cnt));
    bool cliq_credits = per_edge, qr_credits = false;
    if (per_edge) {
        GD_CK(ctx, run_node_sums(g, true));
        GD_CK(ctx, run_triangle_sums(g, cnt));
        qr_credits = true;
    }
    GD_CK(ctx, run_cycles(g, per_edge, cnt));
    GD_CK(ctx, run_final(g, variant, per_edge, cliq_credits, qr_credits, out_dev));
    GD_CK(ctx, run_complete(g, per_edge ? 0 : 1));
    return GD_OK;
}

int gd_count_global(gd_graph *g, gd_u128 out[15]) {
    if (!g || !out) return GD_EINVAL;
    gd_ctx *ctx = g->ctx;
    ctx->err.clear();
    GD_CK(ctx, cudaSetDevice(ctx->device));
    int rc = count_path(g, false, nullptr);
    if (rc) return rc;
    return read_results(g, out);
}

int gd_count_per_edge(gd_graph *g, uint64_t *out, int out_flags, gd_u128 global_out[15]) {
    if (!g || (!out && g->m > 0)) return GD_EINVAL;
    gd_ctx *ctx = g->ctx;
    ctx->err.clear();
    GD_CK(ctx, cudaSetDevice(ctx->device));
    uint64_t *dst = out;
    const bool dev_out = (out_flags & GD_OUT_DEVICE) != 0;
    const size_t out_bytes = sizeof(uint64_t) * 15 * (size_t)g->m;
    int rc;
    if (!dev_out) {
        if (!g->ws.out_buf || g->ws.out_buf_bytes < out_bytes) {
            if (g->ws.out_buf) { release_block(g, g->ws.out_buf); g->ws.out_buf = nullptr; }
            if ((rc = dalloc(g, (void **)&g->ws.out_buf, out_bytes))) return rc;
            g->ws.out_buf_bytes = out_bytes;
        }
        dst = g->ws.out_buf;
    }
    rc = count_path(g, true, dst);
    if (rc) return rc;
    if (!dev_out && g->m > 0) {
        // the matrix back to the host in chunks on several streams at once
        // (more copy engines at work than one stream's copy gets); the
        // graph's stream waits for all of them before the results are read
        constexpr int K = gd_ctx::COPY_STREAMS;
        if (!ctx->copy_st[0]) {
            for (int i = 0; i < K; i++)
                GD_CK(ctx, cudaStreamCreateWithFlags(&ctx->copy_st[i], cudaStreamNonBlocking));
            for (int i = 0; i <= K; i++) GD_CK(ctx, cudaEventCreateWithFlags(&ctx->copy_ev[i], cudaEventDisableTiming));
        }
        GD_CK(ctx, cudaEventRecord(ctx->copy_ev[K], g->stream));
        const size_t rows = (size_t)g->m, per = (rows + K - 1) / K;
        for (int i = 0; i < K; i++) {
            const size_t r0 = std::min(rows, per * (size_t)i), r1 = std::min(rows, per * (size_t)(i + 1));
            GD_CK(ctx, cudaStreamWaitEvent(ctx->copy_st[i], ctx->copy_ev[K], 0));
            if (r1 > r0)
                GD_CK(ctx, cudaMemcpyAsync(out + r0 * 15, dst + r0 * 15, sizeof(uint64_t) * 15 * (r1 - r0),
                                           cudaMemcpyDeviceToHost, ctx->copy_st[i]));
            GD_CK(ctx, cudaEventRecord(ctx->copy_ev[i], ctx->copy_st[i]));
            GD_CK(ctx, cudaStreamWaitEvent(g->stream, ctx->copy_ev[i], 0));
        }
    }
    return read_results(g, global_out);
}

// Scoped device blocks from the context pool (released on scope exit).
struct PoolBlocks {
    gd_ctx *ctx;
    std::vector<std::pair<void *, size_t>> bl;
    explicit PoolBlocks(gd_ctx *c) : ctx(c) {}
    int get(void **p, size_t bytes) {
        int rc = ctx_alloc(ctx, p, bytes);
        if (rc == GD_OK) bl.emplace_back(*p, bytes);
        return rc;
    }
    ~PoolBlocks() { for (auto &b : bl) ctx_release(ctx, b.first, b.second); }
};

// The device part of a batch call as a captured CUDA graph: (gather the
// per-graph CSRs into the packed arrays,) zero the work words, validate the
// packed union, count (one persistent launch), copy the status words to
// pinned host memory.  Replayed while the call is the same.
static int count_batch_captured(gd_ctx *ctx, int32_t G, const std::vector<int32_t> &gnp, int32_t N, int64_t nnz,
                                int32_t nmax_graph, const int32_t *d_gnp, const int32_t *d_rp, const int32_t *d_ci,
                                uint64_t *d_out, const int32_t *const *rps = nullptr,
                                const int32_t *const *cis = nullptr, const int32_t *d_eoff = nullptr,
                                const std::vector<int32_t> *eoff = nullptr) {
    cudaStream_t st = ctx->stream;
    BatchGraph *b = ctx->bgraph;
    const bool same = b && b->G == G && b->N == N && b->nnz == nnz && b->gnp == d_gnp && b->rp == d_rp &&
                      b->ci == d_ci && b->out == d_out && b->gnp_host == gnp && b->rps == (const void *)rps &&
                      b->cis == (const void *)cis && b->eoff == d_eoff && (!eoff || b->eoff_host == *eoff);
    if (!same) {
        batch_graph_destroy(ctx);
        b = new (std::nothrow) BatchGraph();
        if (!b) return fail(ctx, GD_ENOMEM, "host allocation failed");
        ctx->bgraph = b;
        b->G = G; b->N = N; b->nnz = nnz; b->gnp = d_gnp; b->rp = d_rp; b->ci = d_ci; b->out = d_out;
        b->gnp_host = gnp;
        b->rps = rps; b->cis = cis; b->eoff = d_eoff;
        if (eoff) b->eoff_host = *eoff;
        b->misc_bytes = 64 * sizeof(int32_t);
        b->big_bytes = sizeof(int32_t) * (size_t)G;
        int rc;
        if ((rc = ctx_alloc(ctx, (void **)&b->d_misc, b->misc_bytes))) { batch_graph_destroy(ctx); return rc; }
        if ((rc = ctx_alloc(ctx, (void **)&b->d_big, b->big_bytes))) { batch_graph_destroy(ctx); return rc; }
        GD_CK(ctx, cudaHostAlloc((void **)&b->h_status, 64 * sizeof(int32_t), cudaHostAllocDefault));
        gd_graph tmp;
        tmp.ctx = ctx; tmp.stream = st; tmp.n = N; tmp.nnz = nnz; tmp.m = nnz / 2;
        tmp.rp = const_cast<int32_t *>(d_rp); tmp.ci = const_cast<int32_t *>(d_ci);
        const bool prof = ctx->prof;
        ctx->prof = false;      // no event records inside the capture
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_misc, 0, b->misc_bytes, st);
        if (e == cudaSuccess && rps)
            e = launch_batch_gather(ctx, st, G, rps, cis, d_gnp, d_eoff, const_cast<int32_t *>(d_rp),
                                    const_cast<int32_t *>(d_ci), b->d_misc + 16);
        if (e == cudaSuccess) e = launch_validate(&tmp, b->d_misc + 8);
        if (e == cudaSuccess)
            e = launch_batch_count(ctx, st, G, d_gnp, d_rp, d_ci, b->d_misc, (unsigned long long *)d_out,
                                   b->d_misc + 1, b->d_big, b->d_misc + 2, nmax_graph <= 512 ? 512 : 1024);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->h_status, b->d_misc, 20 * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(st, &graph);
        ctx->prof = prof;
        tmp.ws = Workspace();
        if (e == cudaSuccess) e = e2;
        if (e != cudaSuccess) { if (graph) cudaGraphDestroy(graph); batch_graph_destroy(ctx); return cuda_fail(ctx, e, "batch capture"); }
        b->graph = graph;
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (e != cudaSuccess) { batch_graph_destroy(ctx); return cuda_fail(ctx, e, "batch graph instantiate"); }
    }
    GD_CK(ctx, cudaGraphLaunch(b->exec, st));
    GD_CK(ctx, cudaStreamSynchronize(st));
    const int32_t *h = b->h_status;
    if (rps && h[16])
        return fail(ctx, GD_EINVAL, "a graph's row_ptr does not start at 0 or does not end at its slot count");
    if (h[8] || h[10] != h[11])
        return fail(ctx, GD_EINVAL, "invalid batch CSR: rows must be strictly ascending, ids in range, "
                    "no self-loops, every edge stored in both directions");
    if (h[1] & 1) return fail(ctx, GD_EINVAL, "an edge of the batch leaves its graph's node range");
    if (h[1]) return fail(ctx, GD_EARITH, "inconsistent batch counts (status 0x%x)", h[1]);
    return GD_OK;
}

// Validate and count a packed batch already on the device (the union CSR
// d_rp / d_ci with graph offsets d_gnp; host copy gnp), rows of 15 counts to
// d_out; graphs above the shared-memory limit go through the single-graph
// path on a relabelled copy.
static int count_packed(gd_ctx *ctx, int32_t num_graphs, const std::vector<int32_t> &gnp, int32_t N, int64_t nnz,
                        int32_t nmax_graph, const int32_t *d_gnp, const int32_t *d_rp, const int32_t *d_ci,
                        unsigned long long *d_out, PoolBlocks &pb) {
    cudaStream_t st = ctx->stream;
    int rc;
    int32_t *d_misc;    // [0] work index, [1] status, [2] big count, [3..6] validate status
    int32_t *d_big;
    if ((rc = pb.get((void **)&d_misc, 64 * sizeof(int32_t)))) return rc;
    if ((rc = pb.get((void **)&d_big, sizeof(int32_t) * (size_t)num_graphs))) return rc;
    // validate the packed union (rows sorted, ids in range, no self-loops, symmetric)
    {
        gd_graph tmp;
        tmp.ctx = ctx; tmp.stream = st; tmp.n = N; tmp.nnz = nnz; tmp.m = nnz / 2;
        tmp.rp = const_cast<int32_t *>(d_rp); tmp.ci = const_cast<int32_t *>(d_ci);
        tmp.ws.status = d_misc + 8;
        int32_t bad_index = -1, bad_code = 0;
        GD_CK(ctx, validate_csr(&tmp, &bad_index, &bad_code));
        tmp.ws = Workspace();
        if (bad_code)
            return fail(ctx, GD_EINVAL, "invalid batch CSR at row %d: rows must be strictly ascending, ids in range, "
                        "no self-loops, every edge stored in both directions", bad_index);
    }
    GD_CK(ctx, cudaMemsetAsync(d_misc, 0, 8 * sizeof(int32_t), st));
    const int nmax = nmax_graph <= 512 ? 512 : 1024;
    GD_CK(ctx, launch_batch_count(ctx, st, num_graphs, d_gnp, d_rp, d_ci, d_misc, d_out, d_misc + 1, d_big,
                                  d_misc + 2, nmax));
    int32_t misc[3];
    GD_CK(ctx, cudaMemcpyAsync(misc, d_misc, sizeof(misc), cudaMemcpyDeviceToHost, st));
    GD_CK(ctx, cudaStreamSynchronize(st));
    if (misc[1] & 1) return fail(ctx, GD_EINVAL, "an edge of the batch leaves its graph's node range");
    if (misc[1]) return fail(ctx, GD_EARITH, "inconsistent batch counts (status 0x%x)", misc[1]);
    // graphs above the shared-memory limit: the single-graph path on a relabelled copy
    if (misc[2] > 0) {
        std::vector<int32_t> big((size_t)misc[2]);
        GD_CK(ctx, cudaMemcpyAsync(big.data(), d_big, sizeof(int32_t) * big.size(), cudaMemcpyDeviceToHost, st));
        GD_CK(ctx, cudaStreamSynchronize(st));
        for (int32_t gi : big) {
            const int32_t n0 = gnp[gi], n = gnp[gi + 1] - gnp[gi];
            int32_t ends[2];
            GD_CK(ctx, cudaMemcpyAsync(ends, d_rp + n0, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            GD_CK(ctx, cudaMemcpyAsync(ends + 1, d_rp + n0 + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            GD_CK(ctx, cudaStreamSynchronize(st));
            const int64_t ne = ends[1] - ends[0];
            PoolBlocks lb(ctx);
            int32_t *lrp, *lci;
            if ((rc = lb.get((void **)&lrp, sizeof(int32_t) * ((size_t)n + 1)))) return rc;
            if ((rc = lb.get((void **)&lci, sizeof(int32_t) * (size_t)std::max<int64_t>(ne, 1)))) return rc;
            GD_CK(ctx, launch_batch_slice(ctx, st, n0, n, d_rp, d_ci, lrp, lci));
            gd_graph *sub = nullptr;
            if ((rc = gd_create_csr(ctx, n, ne, lrp, lci, GD_DEVICE_PTRS | GD_BORROW, st, &sub))) return rc;
            gd_u128 r[15];
            rc = gd_count_global(sub, r);
            gd_destroy_graph(sub);
            if (rc) return rc;
            uint64_t row[15];
            for (int k = 0; k < 15; k++) {
                if (r[k].hi) return fail(ctx, GD_EOVERFLOW, "graph %d: a count exceeds uint64", gi);
                row[k] = r[k].lo;
            }
            GD_CK(ctx, cudaMemcpyAsync(d_out + (size_t)gi * 15, row, sizeof(row), cudaMemcpyHostToDevice, st));
            GD_CK(ctx, cudaStreamSynchronize(st));
        }
    }
    return GD_OK;
}

int gd_count_batch(gd_ctx *ctx, int32_t num_graphs, const int32_t *graph_node_ptr, const int32_t *row_ptr,
                   const int32_t *col_idx, int flags, uint64_t *out) {
    if (!ctx) return GD_EINVAL;
    ctx->err.clear();
    if (num_graphs < 0 || !graph_node_ptr || !row_ptr || !out)
        return fail(ctx, GD_EINVAL, "gd_count_batch: null pointer or negative graph count");
    GD_CK(ctx, cudaSetDevice(ctx->device));
    if (num_graphs == 0) return GD_OK;
    const bool dev = (flags & GD_DEVICE_PTRS) != 0;
    const bool dev_out = (flags & GD_OUT_DEVICE) != 0;
    cudaStream_t st = ctx->stream;
    // graph offsets on the host (they decide the kernel variant and the fallback)
    std::vector<int32_t> gnp((size_t)num_graphs + 1);
    if (dev) {
        GD_CK(ctx, cudaMemcpyAsync(gnp.data(), graph_node_ptr, sizeof(int32_t) * gnp.size(), cudaMemcpyDeviceToHost, st));
        GD_CK(ctx, cudaStreamSynchronize(st));
    } else {
        memcpy(gnp.data(), graph_node_ptr, sizeof(int32_t) * gnp.size());
    }
    if (gnp[0] != 0) return fail(ctx, GD_EINVAL, "graph_node_ptr[0] must be 0");
    int32_t nmax_graph = 0;
    for (int32_t i = 0; i < num_graphs; i++) {
        if (gnp[i + 1] < gnp[i]) return fail(ctx, GD_EINVAL, "graph_node_ptr decreases at graph %d", i);
        nmax_graph = std::max(nmax_graph, gnp[i + 1] - gnp[i]);
    }
    if (nmax_graph > 65535)
        return fail(ctx, GD_EOVERFLOW, "a graph of the batch has %d nodes; per-graph uint64 counts need <= 65535",
                    nmax_graph);
    const int32_t N = gnp[num_graphs];
    int32_t nnz32 = 0;
    if (dev) {
        GD_CK(ctx, cudaMemcpyAsync(&nnz32, row_ptr + N, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        GD_CK(ctx, cudaStreamSynchronize(st));
    } else {
        nnz32 = row_ptr[N];
        if (row_ptr[0] != 0) return fail(ctx, GD_EINVAL, "row_ptr[0] must be 0");
        for (int32_t u = 0; u < N; u++)
            if (row_ptr[u + 1] < row_ptr[u]) return fail(ctx, GD_EINVAL, "row_ptr decreases at row %d", u);
    }
    const int64_t nnz = nnz32;
    if (nnz < 0 || (nnz & 1)) return fail(ctx, GD_EINVAL, "row_ptr[N] must be a non-negative even count");
    if (nnz > 0 && !col_idx) return fail(ctx, GD_EINVAL, "null col_idx");
    if ((flags & GD_CAPTURE) && dev && dev_out && nmax_graph <= 1024)
        return count_batch_captured(ctx, num_graphs, gnp, N, nnz, nmax_graph, graph_node_ptr, row_ptr, col_idx, out);
    PoolBlocks pb(ctx);
    int rc;
    const int32_t *d_gnp = graph_node_ptr, *d_rp = row_ptr, *d_ci = col_idx;
    if (!dev) {
        int32_t *a, *b, *c;
        if ((rc = pb.get((void **)&a, sizeof(int32_t) * gnp.size()))) return rc;
        if ((rc = pb.get((void **)&b, sizeof(int32_t) * ((size_t)N + 1)))) return rc;
        if ((rc = pb.get((void **)&c, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1)))) return rc;
        GD_CK(ctx, cudaMemcpyAsync(a, gnp.data(), sizeof(int32_t) * gnp.size(), cudaMemcpyHostToDevice, st));
        GD_CK(ctx, cudaMemcpyAsync(b, row_ptr, sizeof(int32_t) * ((size_t)N + 1), cudaMemcpyHostToDevice, st));
        if (nnz > 0) GD_CK(ctx, cudaMemcpyAsync(c, col_idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, st));
        d_gnp = a; d_rp = b; d_ci = c;
    }
    unsigned long long *d_out = (unsigned long long *)out;
    if (!dev_out) {
        if ((rc = pb.get((void **)&d_out, sizeof(uint64_t) * 15 * (size_t)num_graphs))) return rc;
    }
    if ((rc = count_packed(ctx, num_graphs, gnp, N, nnz, nmax_graph, d_gnp, d_rp, d_ci, d_out, pb))) return rc;
    if (!dev_out) {
        GD_CK(ctx, cudaMemcpyAsync(out, d_out, sizeof(uint64_t) * 15 * (size_t)num_graphs, cudaMemcpyDeviceToHost, st));
    }
    GD_CK(ctx, cudaStreamSynchronize(st));
    return GD_OK;
}

int gd_count_batch_gather(gd_ctx *ctx, int32_t num_graphs, const int32_t *const *row_ptrs,
                          const int32_t *const *col_idxs, const int32_t *num_nodes, const int64_t *num_slots,
                          int flags, uint64_t *out) {
    if (!ctx) return GD_EINVAL;
    ctx->err.clear();
    if (num_graphs < 0 || (num_graphs > 0 && (!row_ptrs || !col_idxs || !num_nodes || !num_slots || !out)))
        return fail(ctx, GD_EINVAL, "gd_count_batch_gather: null pointer or negative graph count");
    GD_CK(ctx, cudaSetDevice(ctx->device));
    if (num_graphs == 0) return GD_OK;
    cudaStream_t st = ctx->stream;
    // node and slot offsets of the packed batch, from the host sizes
    std::vector<int32_t> gnp((size_t)num_graphs + 1), eoff((size_t)num_graphs + 1);
    int64_t N = 0, E = 0;
    int32_t nmax_graph = 0;
    for (int32_t i = 0; i < num_graphs; i++) {
        const int32_t n = num_nodes[i];
        const int64_t e = num_slots[i];
        if (n < 0 || e < 0 || (e & 1))
            return fail(ctx, GD_EINVAL, "graph %d: negative size or odd slot count", i);
        gnp[i] = (int32_t)N;
        eoff[i] = (int32_t)E;
        N += n;
        E += e;
        if (N > INT32_MAX - 1 || E > INT32_MAX)
            return fail(ctx, GD_EOVERFLOW, "the packed batch exceeds int32 node or slot indices");
        nmax_graph = std::max(nmax_graph, n);
    }
    gnp[num_graphs] = (int32_t)N;
    eoff[num_graphs] = (int32_t)E;
    if (nmax_graph > 65535)
        return fail(ctx, GD_EOVERFLOW, "a graph of the batch has %d nodes; per-graph uint64 counts need <= 65535",
                    nmax_graph);
    // packed arrays, kept by the context for the next call of the same shape
    GatherBufs &gb = ctx->gather;
    int rc;
    auto grow = [&](void **p, size_t &cap, size_t need) -> int {
        if (*p && cap >= need) return GD_OK;
        if (*p) { ctx_release(ctx, *p, cap); *p = nullptr; cap = 0; }
        int r = ctx_alloc(ctx, p, need);
        if (r == GD_OK) cap = need;
        return r;
    };
    if ((rc = grow((void **)&gb.gnp, gb.gnp_bytes, sizeof(int32_t) * gnp.size()))) return rc;
    if ((rc = grow((void **)&gb.eoff, gb.eoff_bytes, sizeof(int32_t) * eoff.size()))) return rc;
    if ((rc = grow((void **)&gb.rp, gb.rp_bytes, sizeof(int32_t) * (size_t)(N + 1)))) return rc;
    if ((rc = grow((void **)&gb.ci, gb.ci_bytes, sizeof(int32_t) * (size_t)std::max<int64_t>(E, 1)))) return rc;
    if ((rc = grow((void **)&gb.misc, gb.misc_bytes, 64 * sizeof(int32_t)))) return rc;
    GD_CK(ctx, cudaMemcpyAsync(gb.gnp, gnp.data(), sizeof(int32_t) * gnp.size(), cudaMemcpyHostToDevice, st));
    GD_CK(ctx, cudaMemcpyAsync(gb.eoff, eoff.data(), sizeof(int32_t) * eoff.size(), cudaMemcpyHostToDevice, st));
    if ((flags & GD_CAPTURE) && nmax_graph <= 1024)
        return count_batch_captured(ctx, num_graphs, gnp, (int32_t)N, E, nmax_graph, gb.gnp, gb.rp, gb.ci, out,
                                    row_ptrs, col_idxs, gb.eoff, &eoff);
    GD_CK(ctx, cudaMemsetAsync(gb.misc, 0, sizeof(int32_t), st));
    GD_CK(ctx, launch_batch_gather(ctx, st, num_graphs, row_ptrs, col_idxs, gb.gnp, gb.eoff, gb.rp, gb.ci, gb.misc));
    int32_t gstat = 0;
    GD_CK(ctx, cudaMemcpyAsync(&gstat, gb.misc, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GD_CK(ctx, cudaStreamSynchronize(st));
    if (gstat) return fail(ctx, GD_EINVAL, "a graph's row_ptr does not start at 0 or does not end at its slot count");
    PoolBlocks pb(ctx);
    if ((rc = count_packed(ctx, num_graphs, gnp, (int32_t)N, E, nmax_graph, gb.gnp, gb.rp, gb.ci,
                           (unsigned long long *)out, pb))) return rc;
    GD_CK(ctx, cudaStreamSynchronize(st));
    return GD_OK;
}

int gd_autotune(gd_graph *g, int per_edge, int32_t max_trials, gd_tune_result *res) {
    if (!g || !res) return GD_EINVAL;
    gd_ctx *ctx = g->ctx;
    ctx->err.clear();
    GD_CK(ctx, cudaSetDevice(ctx->device));
    const gd_options start = ctx->opt;
    uint64_t *out = nullptr;
    int rc;
    if (per_edge) {
        const size_t bytes = sizeof(uint64_t) * 15 * (size_t)g->m;
        if (!g->ws.out_buf || g->ws.out_buf_bytes < bytes) {
            if (g->ws.out_buf) { release_block(g, g->ws.out_buf); g->ws.out_buf = nullptr; }
            if ((rc = dalloc(g, (void **)&g->ws.out_buf, bytes))) return rc;
            g->ws.out_buf_bytes = bytes;
        }
        out = g->ws.out_buf;
    }
    cudaEvent_t e0, e1;
    GD_CK(ctx, cudaEventCreate(&e0));
    GD_CK(ctx, cudaEventCreate(&e1));
    auto time_once = [&](double *ms) -> int {
        // two runs: the first settles allocations and caches, the second is timed
        for (int r = 0; r < 2; r++) {
            GD_CK(ctx, cudaEventRecord(e0, g->stream));
            int rc2 = count_path(g, per_edge != 0, out);
            if (rc2) return rc2;
            GD_CK(ctx, cudaEventRecord(e1, g->stream));
            if ((rc2 = read_results(g, nullptr))) return rc2;
            float f = 0.f;
            GD_CK(ctx, cudaEventElapsedTime(&f, e0, e1));
            *ms = f;
        }
        return GD_OK;
    };
    double best_ms = 0;
    if ((rc = time_once(&best_ms))) { ctx->opt = start; return rc; }
    res->default_ms = best_ms;
    gd_options best = start;
    int32_t trials = 1;
    const int32_t smem_c[] = {4096, 8192, 16384};
    const int32_t bitmap_c[] = {256, 1024};
    const int32_t hub_c[] = {14, 16, 18, 20};
    for (int32_t sm : smem_c)
        for (int32_t bm : bitmap_c)
            for (int32_t hb : hub_c) {
                if (trials >= max_trials) break;
                gd_options o = start;
                o.smem_table_max = sm; o.bitmap_max_outdeg = bm; o.hub_wedges_log2 = hb;
                if (o.smem_table_max == start.smem_table_max && o.bitmap_max_outdeg == start.bitmap_max_outdeg &&
                    o.hub_wedges_log2 == start.hub_wedges_log2) continue;
                ctx->opt = o;
                double ms = 0;
                if ((rc = time_once(&ms))) { ctx->opt = start; cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
                trials++;
                if (ms < best_ms) { best_ms = ms; best = o; }
            }
    // the medium tier's cluster cut-over, on the best set so far
    for (int32_t mc : {15, 17, 41}) {
        if (trials >= max_trials) break;
        gd_options o = best;
        o.medium_cluster_log2 = mc;
        ctx->opt = o;
        double ms = 0;
        if ((rc = time_once(&ms))) { ctx->opt = start; cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
        trials++;
        if (ms < best_ms) { best_ms = ms; best = o; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->opt = best;
    res->best = best;
    res->best_ms = best_ms;
    res->trials = trials;
    return GD_OK;
}

int gd_autotune_batch(gd_ctx *ctx, int32_t num_graphs, const int32_t *graph_node_ptr, const int32_t *row_ptr,
                      const int32_t *col_idx, int flags, uint64_t *out, gd_tune_result *res) {
    if (!ctx || !res) return GD_EINVAL;
    memset(res, 0, sizeof(*res));
    const gd_options start = ctx->opt;
    using clk = std::chrono::steady_clock;
    auto time_once = [&](double *ms) -> int {
        double best = 1e30;
        for (int r = 0; r < 2; r++) {
            const auto t0 = clk::now();
            int rc = gd_count_batch(ctx, num_graphs, graph_node_ptr, row_ptr, col_idx, flags & ~GD_CAPTURE, out);
            if (rc) return rc;
            best = std::min(best, std::chrono::duration<double, std::milli>(clk::now() - t0).count());
        }
        *ms = best;
        return GD_OK;
    };
    double best_ms = 0;
    int rc = time_once(&best_ms);
    if (rc) { ctx->opt = start; return rc; }
    res->default_ms = best_ms;
    gd_options best = start;
    int32_t trials = 1;
    for (int32_t t : {128, 256, 512, 1024}) {
        if (t == start.batch_threads) continue;
        gd_options o = start;
        o.batch_threads = t;
        ctx->opt = o;
        double ms = 0;
        if ((rc = time_once(&ms))) { ctx->opt = start; return rc; }
        trials++;
        if (ms < best_ms) { best_ms = ms; best = o; }
    }
    ctx->opt = best;
    res->best = best;
    res->best_ms = best_ms;
    res->trials = trials;
    return GD_OK;
}

int gd_profile_begin(gd_ctx *ctx) {
    if (!ctx) return GD_EINVAL;
    for (auto &r : ctx->recs) { ctx->evpool.push_back(r.a); ctx->evpool.push_back(r.b); }
    ctx->recs.clear();
    ctx->prof = true;
    return GD_OK;
}

int gd_profile_end(gd_ctx *ctx, gd_stage_stat *out, int32_t max_out, int32_t *num_out) {
    if (!ctx) return GD_EINVAL;
    ctx->prof = false;
    std::vector<gd_stage_stat> agg;
    int rc = GD_OK;
    for (auto &r : ctx->recs) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "profile event"); break; }
        size_t i = 0;
        while (i < agg.size() && strncmp(agg[i].name, r.name, sizeof(agg[i].name)) != 0) i++;
        if (i == agg.size()) {
            gd_stage_stat st;
            memset(&st, 0, sizeof(st));
            snprintf(st.name, sizeof(st.name), "%s", r.name);
            agg.push_back(st);
        }
        agg[i].ms_total += ms;
        agg[i].launches += 1;
    }
    for (auto &r : ctx->recs) { ctx->evpool.push_back(r.a); ctx->evpool.push_back(r.b); }
    ctx->recs.clear();
    if (num_out) *num_out = (int32_t)agg.size();
    if (out)
        for (size_t i = 0; i < agg.size() && (int32_t)i < max_out; i++) out[i] = agg[i];
    return rc;
}

int64_t gd_kernel_launches(const gd_ctx *ctx) { return ctx ? ctx->launches : -1; }

int gd_footprint_estimate(gd_ctx *ctx, int32_t n, int64_t nnz, int per_edge, size_t *bytes) {
    if (!ctx || !bytes || n < 0 || nnz < 0) return GD_EINVAL;
    *bytes = estimate_footprint(ctx, n, nnz, per_edge != 0, per_edge != 0);
    return GD_OK;
}

int gd_pool_release(gd_ctx *ctx) {
    if (!ctx) return GD_EINVAL;
    cudaSetDevice(ctx->device);
    trim_pool(ctx);
    return GD_OK;
}

}  // extern "C"
