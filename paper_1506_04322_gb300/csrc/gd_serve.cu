// gd_serve.cu -- the request loop: counting requests of mixed graph sizes are
// submitted as they arrive (gd_submit), admitted by device-memory footprint,
// run concurrently on the GPU, and collected with gd_poll.  Host code only.
//
// A service owns `slots` worker threads.  Each worker has its own libgd
// context (its own CUDA stream, its own block cache), so the requests it runs
// overlap on the device with the other workers' requests.  A worker takes the
// oldest queued request whose estimated footprint fits in what the budget has
// left; a small request (a graph that fits the batched kernel) takes every
// other queued small request that fits with it and runs them as one batched
// launch (continuous batching: requests that arrived while the GPU was busy
// ride along in the next launch).  A request larger than the whole budget is
// refused at submission with GD_ENOMEM.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gd_internal.h"

namespace gdi {

namespace {

constexpr int32_t SMALL_N = 1024;          // batched-kernel node limit
constexpr int32_t BATCH_MAX_GRAPHS = 4096;

struct Request {
    gd_req id = 0;
    int32_t n = 0;
    int64_t nnz = 0;
    std::vector<int32_t> rp, ci;
    size_t footprint = 0;
    int state = 0;            // 0 queued, 1 running, 2 done
    int status = GD_OK;
    gd_u128 result[15];
    double t_submit = 0, t_start = 0, t_end = 0;
    int32_t slot = -1, batched = 0;
};

}  // namespace

struct Service {
    gd_ctx *parent = nullptr;
    int32_t slots = 0;
    size_t budget = 0;         // 0: no limit
    size_t inflight = 0;
    std::vector<gd_ctx *> sub;
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<gd_req, Request *> all;
    gd_req next_id = 1;
    bool stop = false;
    std::chrono::steady_clock::time_point t0;
    // totals
    int64_t launches_batched = 0, launches_single = 0;

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    bool fits(size_t fp) const { return budget == 0 || inflight + fp <= budget; }
};

namespace {

// Take work for one worker: the oldest fitting request, plus fitting small
// requests to batch with it.  Called with the lock held.
bool pick(Service *s, std::vector<Request *> &out) {
    out.clear();
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        Request *r = *it;
        if (!s->fits(r->footprint)) continue;
        out.push_back(r);
        s->inflight += r->footprint;
        s->queue.erase(it);
        break;
    }
    if (out.empty()) return false;
    if (out[0]->n <= SMALL_N) {
        for (auto it = s->queue.begin(); it != s->queue.end() && (int32_t)out.size() < BATCH_MAX_GRAPHS;) {
            Request *r = *it;
            if (r->n <= SMALL_N && s->fits(r->footprint)) {
                s->inflight += r->footprint;
                out.push_back(r);
                it = s->queue.erase(it);
            } else {
                ++it;
            }
        }
    }
    return true;
}

void run_single(gd_ctx *ctx, Request *r) {
    gd_graph *g = nullptr;
    int rc = gd_create_csr(ctx, r->n, r->nnz, r->rp.data(), r->ci.empty() ? r->rp.data() : r->ci.data(), 0,
                           ctx->stream, &g);
    if (rc == GD_OK) rc = gd_count_global(g, r->result);
    gd_destroy_graph(g);
    r->status = rc;
}

void run_batch(gd_ctx *ctx, std::vector<Request *> &rs) {
    const int32_t G = (int32_t)rs.size();
    std::vector<int32_t> gnp((size_t)G + 1, 0);
    int64_t N = 0, E = 0;
    for (int32_t i = 0; i < G; i++) { N += rs[i]->n; E += rs[i]->nnz; }
    std::vector<int32_t> rp((size_t)N + 1), ci((size_t)std::max<int64_t>(E, 1));
    int64_t no = 0, eo = 0;
    for (int32_t i = 0; i < G; i++) {
        Request *r = rs[i];
        gnp[i] = (int32_t)no;
        for (int32_t u = 0; u < r->n; u++) rp[no + u] = (int32_t)(eo + r->rp[u]);
        for (int64_t p = 0; p < r->nnz; p++) ci[eo + p] = (int32_t)(no + r->ci[p]);
        no += r->n;
        eo += r->nnz;
    }
    gnp[G] = (int32_t)no;
    rp[no] = (int32_t)eo;
    std::vector<uint64_t> out((size_t)G * 15);
    int rc = gd_count_batch(ctx, G, gnp.data(), rp.data(), ci.data(), 0, out.data());
    if (rc != GD_OK && G > 1) {
        // one bad request must not fail the others: count them one by one
        for (Request *r : rs) run_single(ctx, r);
        return;
    }
    for (int32_t i = 0; i < G; i++) {
        rs[i]->status = rc;
        for (int k = 0; k < 15; k++) { rs[i]->result[k].lo = out[(size_t)i * 15 + k]; rs[i]->result[k].hi = 0; }
    }
}

void worker_main(Service *s, int32_t k) {
    gd_ctx *ctx = s->sub[k];
    cudaSetDevice(ctx->device);
    std::vector<Request *> work;
    while (true) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            // the requests of the previous round may be gone (polled and freed):
            // only what pick() hands out in this round is run
            work.clear();
            s->cv_work.wait(lk, [&] { return s->stop || pick(s, work); });
            if (s->stop && work.empty()) break;      // stop requested and nothing picked
            const double t = s->now_ms();
            for (Request *r : work) { r->state = 1; r->t_start = t; r->slot = k; r->batched = work.size() > 1 || r->n <= SMALL_N; }
        }
        if (work.size() == 1 && work[0]->n > SMALL_N) {
            run_single(ctx, work[0]);
        } else {
            run_batch(ctx, work);
        }
        // keep the worker's block cache within its share of the budget
        if (s->budget && ctx->pooled > s->budget / (size_t)s->slots) gd_pool_release(ctx);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            const double t = s->now_ms();
            for (Request *r : work) {
                r->state = 2;
                r->t_end = t;
                s->inflight -= r->footprint;
            }
            if (work.size() > 1 || (work.size() == 1 && work[0]->n <= SMALL_N)) s->launches_batched++;
            else s->launches_single++;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

}  // namespace

void serve_destroy(gd_ctx *ctx) {
    Service *s = ctx->service;
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    for (gd_ctx *c : s->sub) gd_destroy(c);
    for (auto &kv : s->all) delete kv.second;
    delete s;
    ctx->service = nullptr;
}

}  // namespace gdi

using namespace gdi;

extern "C" {

int gd_serve_start(gd_ctx *ctx, int32_t slots, size_t hbm_budget_bytes) {
    if (!ctx || slots < 1 || slots > 64) return GD_EINVAL;
    if (ctx->service) return GD_OK;
    Service *s = new (std::nothrow) Service();
    if (!s) return GD_ENOMEM;
    s->parent = ctx;
    s->slots = slots;
    s->budget = hbm_budget_bytes ? hbm_budget_bytes : ctx->budget;
    s->t0 = std::chrono::steady_clock::now();
    for (int32_t k = 0; k < slots; k++) {
        gd_ctx *c = nullptr;
        int rc = gd_init(&c, ctx->device, 0, &ctx->opt);
        if (rc) {
            for (gd_ctx *x : s->sub) gd_destroy(x);
            delete s;
            return rc;
        }
        s->sub.push_back(c);
    }
    ctx->service = s;
    for (int32_t k = 0; k < slots; k++) s->workers.emplace_back(worker_main, s, k);
    return GD_OK;
}

int gd_submit(gd_ctx *ctx, const gd_request_desc *desc, gd_req *id) {
    if (!ctx || !desc || !id) return GD_EINVAL;
    if (!ctx->service) {
        int rc = gd_serve_start(ctx, 4, 0);
        if (rc) return rc;
    }
    Service *s = ctx->service;
    if (desc->n < 0 || desc->nnz < 0 || !desc->row_ptr || (desc->nnz > 0 && !desc->col_idx)) return GD_EINVAL;
    if (desc->nnz > INT32_MAX) return GD_EOVERFLOW;
    if (desc->mode != 0) return GD_ENOTIMPL;
    if (desc->row_ptr[0] != 0 || (int64_t)desc->row_ptr[desc->n] != desc->nnz) return GD_EINVAL;
    Request *r = new (std::nothrow) Request();
    if (!r) return GD_ENOMEM;
    r->n = desc->n;
    r->nnz = desc->nnz;
    r->rp.assign(desc->row_ptr, desc->row_ptr + (size_t)desc->n + 1);
    if (desc->nnz > 0) r->ci.assign(desc->col_idx, desc->col_idx + desc->nnz);
    r->footprint = r->n <= SMALL_N
        ? sizeof(int32_t) * (size_t)(r->n + 1 + r->nnz) + 512
        : estimate_footprint(ctx, r->n, r->nnz, false, false);
    if (s->budget && r->footprint > s->budget) {
        delete r;
        return GD_ENOMEM;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->id = s->next_id++;
        r->t_submit = s->now_ms();
        s->all[r->id] = r;
        s->queue.push_back(r);
        *id = r->id;
    }
    s->cv_work.notify_one();
    return GD_OK;
}

int gd_poll(gd_ctx *ctx, gd_req id, gd_u128 out[15], gd_req_stats *st) {
    if (!ctx || !ctx->service) return GD_EINVAL;
    Service *s = ctx->service;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return GD_EINVAL;
    Request *r = it->second;
    if (r->state != 2) return GD_EAGAIN;
    if (out) memcpy(out, r->result, sizeof(r->result));
    if (st) {
        st->submit_ms = r->t_submit;
        st->start_ms = r->t_start;
        st->end_ms = r->t_end;
        st->footprint = r->footprint;
        st->slot = r->slot;
        st->batched = r->batched;
    }
    const int status = r->status;
    s->all.erase(it);
    delete r;
    return status;
}

int gd_wait(gd_ctx *ctx, gd_req id, int32_t timeout_ms) {
    if (!ctx || !ctx->service) return GD_EINVAL;
    Service *s = ctx->service;
    std::unique_lock<std::mutex> lk(s->mu);
    auto done = [&] {
        auto it = s->all.find(id);
        return it == s->all.end() || it->second->state == 2;
    };
    if (timeout_ms < 0) s->cv_done.wait(lk, done);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) return GD_ETIMEDOUT;
    return s->all.count(id) ? GD_OK : GD_EINVAL;
}

int gd_serve_stats(gd_ctx *ctx, int64_t *queued, int64_t *running, size_t *inflight_bytes,
                   int64_t *batched_launches, int64_t *single_launches) {
    if (!ctx || !ctx->service) return GD_EINVAL;
    Service *s = ctx->service;
    std::lock_guard<std::mutex> lk(s->mu);
    int64_t run = 0;
    for (auto &kv : s->all) run += kv.second->state == 1;
    if (queued) *queued = (int64_t)s->queue.size();
    if (running) *running = run;
    if (inflight_bytes) *inflight_bytes = s->inflight;
    if (batched_launches) *batched_launches = s->launches_batched;
    if (single_launches) *single_launches = s->launches_single;
    return GD_OK;
}

int gd_serve_stop(gd_ctx *ctx) {
    if (!ctx) return GD_EINVAL;
    serve_destroy(ctx);
    return GD_OK;
}

}  // extern "C"
