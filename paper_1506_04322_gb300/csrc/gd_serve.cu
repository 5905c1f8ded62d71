// gd_serve.cu -- the request loop: counting requests of mixed graph sizes are
// submitted as they arrive (gd_submit), admitted by device-memory footprint,
// kept resident on the device, run concurrently on the GPU, and collected
// with gd_poll.  Host code only.
//
// A service owns a stager thread and `slots` worker threads.  The stager
// admits requests in arrival order as the budget allows: it reserves a
// request's estimated footprint and uploads its CSR to the device on its own
// stream, so the CSR stays resident from admission until the counts are
// done.  A request that does not fit yet may be passed by later ones that
// do, but once it has waited GD_SERVE_MAX_BYPASS_MS at the head of the
// queue, nothing else is admitted until it fits (no starvation).  Each
// worker has its own libgd context (its own CUDA stream, its own block
// cache), so the requests it runs overlap on the device with the other
// workers' requests.  A worker takes the oldest admitted request; a small one
// (a graph that fits the batched kernel) takes every other admitted small
// request with it and counts them in one batched launch straight from their
// device CSRs (continuous batching: requests that arrived while the GPU was
// busy ride along in the next launch).  A request larger than the whole
// budget is refused at submission with GD_ENOMEM.
#include <cuda_runtime.h>

#include <algorithm>
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
    std::vector<int32_t> rp, ci;          // host copy until the upload at admission
    int32_t *d_rp = nullptr, *d_ci = nullptr;   // device CSR, admission to completion
    size_t footprint = 0;
    int state = 0;            // 0 queued, 3 admitted (resident), 1 running, 2 done
    int status = GD_OK;
    gd_u128 result[15];
    double t_submit = 0, t_start = 0, t_end = 0;
    double t_passed = -1;     // first time it was passed over at the head of the queue
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
    std::condition_variable cv_work, cv_done, cv_admit;
    std::deque<Request *> queue;       // submitted, waiting for admission
    std::deque<Request *> admitted;    // footprint reserved, CSR on the device
    std::thread stager;
    cudaStream_t stage_stream = nullptr;
    double max_bypass_ms = GD_SERVE_MAX_BYPASS_MS;
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

// Admission (stager, lock held): the oldest queued request if it fits; else
// a later one that fits, unless the oldest has waited max_bypass_ms since it
// was first passed over -- then nothing until it fits.
Request *admit(Service *s) {
    if (s->queue.empty()) return nullptr;
    Request *head = s->queue.front();
    if (s->fits(head->footprint)) {
        s->queue.pop_front();
        s->inflight += head->footprint;
        return head;
    }
    const double t = s->now_ms();
    if (head->t_passed < 0) head->t_passed = t;
    if (t - head->t_passed >= s->max_bypass_ms) return nullptr;
    for (auto it = s->queue.begin() + 1; it != s->queue.end(); ++it) {
        Request *r = *it;
        if (!s->fits(r->footprint)) continue;
        s->queue.erase(it);
        s->inflight += r->footprint;
        return r;
    }
    return nullptr;
}

// Upload an admitted request's CSR on the stager's stream (stream-ordered
// allocation: no device-wide synchronization while workers count).
int stage(Service *s, Request *r) {
    cudaStream_t st = s->stage_stream;
    const size_t rb = sizeof(int32_t) * ((size_t)r->n + 1), cb = sizeof(int32_t) * (size_t)std::max<int64_t>(r->nnz, 1);
    cudaError_t e = cudaMallocAsync((void **)&r->d_rp, rb, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&r->d_ci, cb, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->d_rp, r->rp.data(), rb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && r->nnz > 0)
        e = cudaMemcpyAsync(r->d_ci, r->ci.data(), sizeof(int32_t) * (size_t)r->nnz, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? GD_ENOMEM : GD_ECUDA;
    std::vector<int32_t>().swap(r->rp);      // the device copy is the request's CSR now
    std::vector<int32_t>().swap(r->ci);
    return GD_OK;
}

void release_csr(Request *r, cudaStream_t st) {
    if (r->d_rp) cudaFreeAsync(r->d_rp, st);
    if (r->d_ci) cudaFreeAsync(r->d_ci, st);
    r->d_rp = r->d_ci = nullptr;
}

void stager_main(Service *s) {
    cudaSetDevice(s->parent->device);
    while (true) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_admit.wait(lk, [&] { return s->stop || (r = admit(s)) != nullptr; });
            if (s->stop && !r) break;
        }
        const int rc = stage(s, r);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (rc == GD_OK) {
                r->state = 3;
                s->admitted.push_back(r);
            } else {
                release_csr(r, s->stage_stream);
                r->status = rc;
                r->state = 2;
                r->t_start = r->t_end = s->now_ms();
                s->inflight -= r->footprint;
            }
        }
        if (rc == GD_OK) s->cv_work.notify_one();
        else s->cv_done.notify_all();
    }
}

// Work for one worker (lock held): the oldest admitted request, plus every
// other admitted small request when it is small.
bool pick(Service *s, std::vector<Request *> &out) {
    out.clear();
    if (s->admitted.empty()) return false;
    out.push_back(s->admitted.front());
    s->admitted.pop_front();
    if (out[0]->n <= SMALL_N) {
        for (auto it = s->admitted.begin(); it != s->admitted.end() && (int32_t)out.size() < BATCH_MAX_GRAPHS;) {
            if ((*it)->n <= SMALL_N) {
                out.push_back(*it);
                it = s->admitted.erase(it);
            } else {
                ++it;
            }
        }
    }
    return true;
}

void run_single(gd_ctx *ctx, Request *r) {
    gd_graph *g = nullptr;
    int rc = gd_create_csr(ctx, r->n, r->nnz, r->d_rp, r->d_ci, GD_DEVICE_PTRS | GD_BORROW, ctx->stream, &g);
    if (rc == GD_OK) rc = gd_count_global(g, r->result);
    gd_destroy_graph(g);
    r->status = rc;
}

// Worker buffers of the batched launch: the requests' device pointers and the
// counts.
struct BatchBufs {
    const int32_t **d_ptrs = nullptr;    // [2 * BATCH_MAX_GRAPHS]
    uint64_t *d_out = nullptr;           // [BATCH_MAX_GRAPHS * 15]
};

void run_batch(gd_ctx *ctx, BatchBufs &bb, std::vector<Request *> &rs) {
    const int32_t G = (int32_t)rs.size();
    std::vector<const int32_t *> ptrs((size_t)2 * G);
    std::vector<int32_t> nn((size_t)G);
    std::vector<int64_t> ns((size_t)G);
    for (int32_t i = 0; i < G; i++) {
        ptrs[i] = rs[i]->d_rp;
        ptrs[G + i] = rs[i]->d_ci;
        nn[i] = rs[i]->n;
        ns[i] = rs[i]->nnz;
    }
    std::vector<uint64_t> out((size_t)G * 15);
    cudaError_t e = cudaMemcpyAsync(bb.d_ptrs, ptrs.data(), sizeof(const int32_t *) * ptrs.size(),
                                    cudaMemcpyHostToDevice, ctx->stream);
    int rc = e == cudaSuccess ? GD_OK : GD_ECUDA;
    if (rc == GD_OK)
        rc = gd_count_batch_gather(ctx, G, bb.d_ptrs, bb.d_ptrs + G, nn.data(), ns.data(), 0, bb.d_out);
    if (rc == GD_OK) {
        e = cudaMemcpyAsync(out.data(), bb.d_out, sizeof(uint64_t) * out.size(), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = GD_ECUDA;
    }
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
    BatchBufs bb;
    const bool bufs_ok =
        cudaMalloc((void **)&bb.d_ptrs, sizeof(const int32_t *) * 2 * BATCH_MAX_GRAPHS) == cudaSuccess &&
        cudaMalloc((void **)&bb.d_out, sizeof(uint64_t) * 15 * BATCH_MAX_GRAPHS) == cudaSuccess;
    std::vector<Request *> work;
    while (true) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            // the requests of the previous round may be gone (polled and freed):
            // only what pick() hands out in this round is run
            work.clear();
            s->cv_work.wait(lk, [&] { return s->stop || pick(s, work); });
            if (s->stop) {
                for (Request *r : work) s->admitted.push_front(r);   // released at shutdown
                break;
            }
            const double t = s->now_ms();
            for (Request *r : work) { r->state = 1; r->t_start = t; r->slot = k; r->batched = work.size() > 1 || r->n <= SMALL_N; }
        }
        if (work.size() == 1 && work[0]->n > SMALL_N) {
            run_single(ctx, work[0]);
        } else if (bufs_ok) {
            run_batch(ctx, bb, work);
        } else {
            for (Request *r : work) run_single(ctx, r);
        }
        for (Request *r : work) release_csr(r, ctx->stream);
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
        s->cv_admit.notify_all();
        s->cv_work.notify_all();
    }
    cudaStreamSynchronize(ctx->stream);
    if (bb.d_ptrs) cudaFree(bb.d_ptrs);
    if (bb.d_out) cudaFree(bb.d_out);
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
    s->cv_admit.notify_all();
    if (s->stager.joinable()) s->stager.join();
    for (auto &t : s->workers) t.join();
    cudaSetDevice(ctx->device);
    for (auto &kv : s->all) release_csr(kv.second, s->stage_stream);
    if (s->stage_stream) {
        cudaStreamSynchronize(s->stage_stream);
        cudaStreamDestroy(s->stage_stream);
    }
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
    if (!s->budget) {
        // no budget given: 45% of the device memory free now, so that the
        // admitted footprints and the workers' block caches (each kept
        // within budget / slots) stay below what the device has
        size_t free_b = 0, total_b = 0;
        if (cudaSetDevice(ctx->device) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            delete s;
            return GD_ECUDA;
        }
        s->budget = free_b / 20 * 9;
    }
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
    if (cudaSetDevice(ctx->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->stage_stream, cudaStreamNonBlocking) != cudaSuccess) {
        for (gd_ctx *x : s->sub) gd_destroy(x);
        delete s;
        return GD_ECUDA;
    }
    ctx->service = s;
    s->stager = std::thread(stager_main, s);
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
    s->cv_admit.notify_one();
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
    if (queued) *queued = (int64_t)(s->queue.size() + s->admitted.size());
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
