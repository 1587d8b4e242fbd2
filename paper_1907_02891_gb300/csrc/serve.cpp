// Request scheduler ("serving"): continuous batching of map requests.
//
// Requests (one radiance map and n spectra each) are queued by
// lp_serve_submit and started by a scheduler thread as soon as a stream slot
// is free and the request's device footprint (its workspace) fits the
// context's HBM budget next to the requests already running.  Each slot owns
// a CUDA stream and a workspace, so requests admitted while others are on the
// GPU run concurrently with them.  Completion is observed with CUDA events;
// latency = completion - submission (host clock).  Spectra and plans are
// the context's device-resident caches, shared by all requests.  With a log
// file set (lp_serve_log), every finished request appends one JSON line.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cstdio>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/lp.h"
#include "lp_runtime.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    const float* L;
    int h, w, ldl, ldo;
    lp_outmode mode;
    std::vector<const lp_spectrum*> spectra;
    std::vector<float*> out;
    MapDims dims;
    size_t footprint;
    Clock::time_point submitted;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    uint64_t ticket = 0;
    size_t footprint = 0;
    std::vector<const lp_spectrum*> spectra;  // references held by the running request
    Clock::time_point submitted, started;
    int h = 0, w = 0, n = 0, mode = 0, prec = 0;  // for the request log
};

struct Result {
    lp_status status;
    double latency_ms;
    double queue_ms;
};

}  // namespace

struct ServeState {
    lp_ctx* ctx = nullptr;
    std::vector<Slot> slots;
    std::deque<Request> queue;
    std::map<uint64_t, Result> done;
    std::mutex mu;
    std::condition_variable cv_work;  // scheduler: new request or stop
    std::condition_variable cv_done;  // pollers: a request finished
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    size_t reserved = 0;   // footprint of running requests
    size_t capacity = 0;   // bytes the running requests may hold together
    size_t max_queue = 1 << 16;
    // counters
    uint64_t n_done = 0, n_failed = 0;
    // per-request log (JSON lines), times in ms from t0
    FILE* log = nullptr;
    Clock::time_point t0 = Clock::now();
};

static double ms_since(Clock::time_point t0, Clock::time_point t)
{
    return std::chrono::duration<double, std::milli>(t - t0).count();
}



static void finish_slot(ServeState* S, Slot& sl, lp_status st)
{
    const auto now = Clock::now();
    for (const lp_spectrum* sp : sl.spectra) lp_spectrum_unref(S->ctx, sp);
    sl.spectra.clear();
    Result r;
    r.status = st;
    r.latency_ms = std::chrono::duration<double, std::milli>(now - sl.submitted).count();
    r.queue_ms = std::chrono::duration<double, std::milli>(sl.started - sl.submitted).count();
    S->done[sl.ticket] = r;
    if (S->log) {
        // completion is seen by the scheduler's event poll (every 20 us while requests run)
        std::fprintf(S->log,
                     "{\"ticket\": %llu, \"status\": %d, \"h\": %d, \"w\": %d, \"n_psf\": %d, \"mode\": %d, "
                     "\"precision\": %d, \"workspace_bytes\": %zu, \"output_mpix\": %.6f, \"submit_ms\": %.4f, "
                     "\"start_ms\": %.4f, \"end_ms\": %.4f, \"queue_ms\": %.4f, \"latency_ms\": %.4f}\n",
                     (unsigned long long)sl.ticket, (int)st, sl.h, sl.w, sl.n, sl.mode, sl.prec, sl.footprint,
                     (double)sl.h * sl.w * sl.n / 1e6, ms_since(S->t0, sl.submitted), ms_since(S->t0, sl.started),
                     ms_since(S->t0, now), r.queue_ms, r.latency_ms);
    }
    S->reserved -= sl.footprint;
    sl.busy = false;
    sl.footprint = 0;
    if (st == LP_OK) S->n_done++;
    else S->n_failed++;
}

static void scheduler_loop(ServeState* S)
{
    cudaSetDevice(S->ctx->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool progressed = false;
        // 1. completions
        for (auto& sl : S->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaSuccess) {
                finish_slot(S, sl, LP_OK);
                progressed = true;
            } else if (q != cudaErrorNotReady) {
                finish_slot(S, sl, LP_ERR_CUDA);
                progressed = true;
            }
        }
        if (progressed) S->cv_done.notify_all();
        // 2. admission: FIFO, by free slot and HBM footprint
        while (!S->queue.empty()) {
            Request& rq = S->queue.front();
            Slot* free_slot = nullptr;
            for (auto& sl : S->slots)
                if (!sl.busy) {
                    free_slot = &sl;
                    break;
                }
            if (!free_slot) break;
            const bool alone = S->reserved == 0;
            if (!alone && S->reserved + rq.footprint > S->capacity) break;  // wait for memory
            Slot& sl = *free_slot;
            void* ws = nullptr;
            lp_status st = lp_get_workspace(S->ctx, sl.stream, rq.footprint, &ws);
            // failure injection (host side): this request fails as a launch would
            if (st == LP_OK && (S->ctx->test_hook.fetch_and(~LP_TEST_SERVE_FAIL) & LP_TEST_SERVE_FAIL))
                st = lp_fail(LP_ERR_CUDA, "injected launch failure (LP_TEST_SERVE_FAIL)");
            if (st == LP_OK)
                st = lp_launch_map(S->ctx, rq.L, rq.h, rq.w, rq.ldl, rq.spectra.data(), (int)rq.spectra.size(),
                                   rq.out.data(), rq.ldo, rq.dims, ws, sl.stream);
            sl.ticket = rq.ticket;
            sl.spectra = rq.spectra;
            sl.submitted = rq.submitted;
            sl.started = Clock::now();
            sl.footprint = rq.footprint;
            sl.h = rq.h;
            sl.w = rq.w;
            sl.n = (int)rq.spectra.size();
            sl.mode = (int)rq.mode;
            sl.prec = (int)rq.spectra[0]->prec;
            sl.busy = true;
            S->reserved += rq.footprint;
            if (st == LP_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) st = LP_ERR_CUDA;
            if (st != LP_OK) {
                finish_slot(S, sl, st);
                S->cv_done.notify_all();
            }
            S->queue.pop_front();
            progressed = true;
        }
        bool any_busy = false;
        for (auto& sl : S->slots) any_busy = any_busy || sl.busy;
        if (S->stop && S->queue.empty() && !any_busy) break;
        if (!progressed) {
            // in flight: poll completions every 20 us; idle: sleep until work
            if (any_busy)
                S->cv_work.wait_for(lk, std::chrono::microseconds(20));
            else
                S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
        }
    }
}

extern "C" lp_status lp_serve_start(lp_ctx* ctx, int n_slots)
{
    if (!ctx) return lp_fail(LP_ERR_INVALID, "lp_serve_start: NULL context");
    if (n_slots < 1 || n_slots > 64) return lp_fail(LP_ERR_INVALID, "lp_serve_start: n_slots %d not in [1, 64]", n_slots);
    if (ctx->serve) return lp_fail(LP_ERR_BUSY, "lp_serve_start: already serving");
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return lp_fail(LP_ERR_CUDA, "lp_serve_start: cudaSetDevice failed");
    auto S = new ServeState();
    S->ctx = ctx;
    S->slots.resize(n_slots);
    for (auto& sl : S->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            for (auto& x : S->slots) {
                if (x.stream) cudaStreamDestroy(x.stream);
                if (x.done) cudaEventDestroy(x.done);
            }
            delete S;
            if (prev >= 0) cudaSetDevice(prev);
            return lp_fail(LP_ERR_CUDA, "lp_serve_start: stream/event creation failed");
        }
    }
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    {
        std::lock_guard<std::mutex> g(ctx->mem_mu);
        if (ctx->budget) S->capacity = ctx->budget > ctx->used ? ctx->budget - ctx->used : 0;
        else S->capacity = free_b / 10 * 9;
    }
    ctx->serve = S;
    S->worker = std::thread(scheduler_loop, S);
    if (prev >= 0) cudaSetDevice(prev);
    return LP_OK;
}

extern "C" lp_status lp_serve_submit(lp_ctx* ctx, const float* L, int h, int w, int ldl,
                                     const lp_spectrum* const* spectra, int n, float* const* out,
                                     int ldo, lp_outmode mode, uint64_t* ticket)
{
    if (ticket) *ticket = 0;
    if (!ctx || !ticket) return lp_fail(LP_ERR_INVALID, "lp_serve_submit: NULL argument");
    ServeState* S = ctx->serve;
    if (!S) return lp_fail(LP_ERR_BUSY, "lp_serve_submit: serving not started");
    if (!spectra || n < 1 || !spectra[0]) return lp_fail(LP_ERR_INVALID, "lp_serve_submit: need spectra");
    MapDims d;
    lp_status st = lp_validate_map(ctx, L, h, w, ldl, spectra, n, out, ldo, mode, spectra[0]->prec, &d);
    if (st != LP_OK) return st;
    for (int k = 0; k < n; ++k)
        if (!out[k]) return lp_fail(LP_ERR_INVALID, "lp_serve_submit: out[%d] is NULL", k);
    Request rq;
    rq.L = L;
    rq.h = h;
    rq.w = w;
    rq.ldl = ldl;
    rq.ldo = ldo;
    rq.mode = mode;
    rq.spectra.assign(spectra, spectra + n);
    rq.out.assign(out, out + n);
    rq.dims = d;
    rq.footprint = lp_workspace_bytes(d, n);
    rq.submitted = Clock::now();
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->stop) return lp_fail(LP_ERR_BUSY, "lp_serve_submit: serving is stopping");
        if (S->queue.size() >= S->max_queue) return lp_fail(LP_ERR_BUSY, "lp_serve_submit: queue full");
        if (rq.footprint > S->capacity)
            return lp_fail(LP_ERR_OOM, "lp_serve_submit: request needs %zu bytes, serving capacity is %zu",
                           rq.footprint, S->capacity);
        rq.ticket = S->next_ticket++;
        *ticket = rq.ticket;
        for (const lp_spectrum* sp : rq.spectra) lp_spectrum_ref(ctx, sp);
        S->queue.push_back(std::move(rq));
    }
    S->cv_work.notify_one();
    return LP_OK;
}

extern "C" lp_status lp_serve_poll(lp_ctx* ctx, uint64_t ticket, int timeout_ms, double* latency_ms)
{
    if (!ctx) return lp_fail(LP_ERR_INVALID, "lp_serve_poll: NULL context");
    ServeState* S = ctx->serve;
    if (!S) return lp_fail(LP_ERR_BUSY, "lp_serve_poll: serving not started");
    std::unique_lock<std::mutex> lk(S->mu);
    if (ticket == 0 || ticket >= S->next_ticket) return lp_fail(LP_ERR_INVALID, "lp_serve_poll: unknown ticket");
    auto ready = [&] { return S->done.count(ticket) != 0; };
    if (timeout_ms < 0) S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return lp_fail(LP_ERR_TIMEOUT, "lp_serve_poll: ticket %llu not finished", (unsigned long long)ticket);
    auto it = S->done.find(ticket);
    const Result r = it->second;
    S->done.erase(it);
    if (latency_ms) *latency_ms = r.latency_ms;
    if (r.status != LP_OK) return lp_fail(r.status, "lp_serve_poll: request %llu failed", (unsigned long long)ticket);
    return LP_OK;
}

extern "C" lp_status lp_serve_stats(lp_ctx* ctx, uint64_t* completed, uint64_t* failed, int* queued,
                                    int* running)
{
    if (!ctx || !ctx->serve) return lp_fail(LP_ERR_BUSY, "lp_serve_stats: serving not started");
    ServeState* S = ctx->serve;
    std::lock_guard<std::mutex> g(S->mu);
    if (completed) *completed = S->n_done;
    if (failed) *failed = S->n_failed;
    if (queued) *queued = (int)S->queue.size();
    if (running) {
        int r = 0;
        for (auto& sl : S->slots) r += sl.busy ? 1 : 0;
        *running = r;
    }
    return LP_OK;
}

extern "C" lp_status lp_serve_cancel(lp_ctx* ctx, uint64_t ticket)
{
    if (!ctx) return lp_fail(LP_ERR_INVALID, "lp_serve_cancel: NULL context");
    ServeState* S = ctx->serve;
    if (!S) return lp_fail(LP_ERR_BUSY, "lp_serve_cancel: serving not started");
    std::vector<const lp_spectrum*> refs;
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (ticket == 0 || ticket >= S->next_ticket)
            return lp_fail(LP_ERR_INVALID, "lp_serve_cancel: unknown ticket");
        auto it = S->queue.begin();
        while (it != S->queue.end() && it->ticket != ticket) ++it;
        if (it == S->queue.end())
            return lp_fail(LP_ERR_BUSY, "lp_serve_cancel: request %llu is running or finished",
                           (unsigned long long)ticket);
        refs.swap(it->spectra);
        S->queue.erase(it);
        Result r;
        r.status = LP_ERR_CANCELLED;
        r.latency_ms = 0.0;
        r.queue_ms = 0.0;
        S->done[ticket] = r;
    }
    for (const lp_spectrum* sp : refs) lp_spectrum_unref(ctx, sp);
    S->cv_done.notify_all();
    return LP_OK;
}

extern "C" lp_status lp_serve_log(lp_ctx* ctx, const char* path)
{
    if (!ctx) return lp_fail(LP_ERR_INVALID, "lp_serve_log: NULL context");
    ServeState* S = ctx->serve;
    if (!S) return lp_fail(LP_ERR_BUSY, "lp_serve_log: serving not started");
    FILE* f = nullptr;
    if (path && path[0]) {
        f = std::fopen(path, "a");
        if (!f) return lp_fail(LP_ERR_INVALID, "lp_serve_log: cannot open %s for appending", path);
    }
    FILE* old;
    {
        std::lock_guard<std::mutex> g(S->mu);
        old = S->log;
        S->log = f;
    }
    if (old) std::fclose(old);
    return LP_OK;
}

extern "C" lp_status lp_serve_stop(lp_ctx* ctx)
{
    if (!ctx) return lp_fail(LP_ERR_INVALID, "lp_serve_stop: NULL context");
    ServeState* S = ctx->serve;
    if (!S) return lp_fail(LP_ERR_BUSY, "lp_serve_stop: serving not started");
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    for (auto& sl : S->slots) {
        cudaStreamSynchronize(sl.stream);
        // the slot's workspace belongs to the context; drop it with the stream
        {
            std::lock_guard<std::mutex> g(ctx->ws_mu);
            for (size_t i = 0; i < ctx->ws.size(); ++i)
                if (ctx->ws[i].stream == sl.stream) {
                    lp_ctx_free(ctx, ctx->ws[i].ptr, ctx->ws[i].bytes);
                    ctx->ws.erase(ctx->ws.begin() + i);
                    break;
                }
        }
        cudaEventDestroy(sl.done);
        cudaStreamDestroy(sl.stream);
    }
    if (S->log) std::fclose(S->log);
    ctx->serve = nullptr;
    delete S;
    if (prev >= 0) cudaSetDevice(prev);
    return LP_OK;
}

void lp_serve_shutdown(lp_ctx* ctx)
{
    if (ctx && ctx->serve) lp_serve_stop(ctx);
}
