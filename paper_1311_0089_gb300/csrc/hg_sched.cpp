// Request scheduler behind hg_submit / hg_poll / hg_cancel.
//
// Continuous batching at the granularity of one CG chunk (a CUDA graph of
// `check_every` iterations): every admitted request keeps its CG state
// resident on the device and runs its chunks on its own stream, so the
// iterations of all admitted requests are in flight on the GPU together.
// Requests that arrive while others run are admitted as soon as a slot and
// device memory (within the context budget) are free; a finished request
// releases its memory at once.  The worker thread never blocks on the GPU: it
// polls each request's tick event and advances the requests whose last
// chunk has completed.
#include "hg.h"
#include "hg_internal.h"
#include "hg_runtime.h"

#include <cuda_runtime.h>

#include <cmath>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace hgrt {

namespace {
enum TicketState { T_QUEUED = 0, T_RUNNING = 1, T_DONE = 2 };
}

struct Ticket {
    uint64_t id = 0;
    hg_grid* g = nullptr;
    int state = T_QUEUED;
    std::atomic<bool> cancel_req{false};
    Job job;
    hg_result res{};
    int status = HG_OK;
};

struct Scheduler {
    hg_ctx* ctx = nullptr;
    std::thread th;
    std::mutex m;
    std::condition_variable cv_work, cv_done;
    std::deque<Ticket*> queue;
    std::map<uint64_t, std::unique_ptr<Ticket>> tickets;
    std::vector<Ticket*> running;
    std::vector<cudaStream_t> streams;
    size_t next_stream = 0;
    uint64_t next_id = 1;
    bool stop = false;
    bool started = false;
    int max_running = 64;
};

static void complete(Scheduler* S, Ticket* t, int status) {
    // the ticket's work is finished or abandoned: make sure nothing is in flight.
    // Its device buffers stay allocated (reused by the next request on this
    // grid; reclaimed by admission when the budget is short).
    if (t->job.s) cudaStreamSynchronize(t->job.s);
    std::lock_guard<std::mutex> lk(S->m);
    t->status = status;
    t->res.status = status;
    t->state = T_DONE;
    t->g->borrowed -= 1;
    S->running.erase(std::remove(S->running.begin(), S->running.end(), t), S->running.end());
    S->cv_done.notify_all();
}

static void worker(Scheduler* S) {
    cudaSetDevice(S->ctx->device);
    for (;;) {
        std::vector<Ticket*> admit;
        {
            std::unique_lock<std::mutex> lk(S->m);
            if (S->stop) break;
            if (S->running.empty() && S->queue.empty()) {
                S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
                if (S->stop) break;
            }
            while (!S->queue.empty() && (int)(S->running.size() + admit.size()) < S->max_running) {
                admit.push_back(S->queue.front());
                S->queue.pop_front();
            }
        }
        // admission: allocate the request's resident state, enqueue its first steps
        for (size_t i = 0; i < admit.size(); ++i) {
            Ticket* t = admit[i];
            if (t->cancel_req) { complete(S, t, HG_ERR_CANCELLED); continue; }
            int st;
            {
                std::lock_guard<std::recursive_mutex> lk(S->ctx->mu);
                t->job.g = t->g;
                t->job.s = S->streams[S->next_stream++ % S->streams.size()];
                t->job.ev0 = t->g->ev0;
                t->job.ev1 = t->g->ev1;
                t->job.tick = t->g->ev_tick;
                st = job_begin(t->job);
                if (st == HG_ERR_NO_MEMORY) {
                    // over the budget: release idle grids' solver state and retry once
                    cudaStreamSynchronize(t->job.s);
                    grid_free_work(t->g);
                    if (ctx_reclaim(S->ctx, t->g) > 0) st = job_begin(t->job);
                }
            }
            if (st == HG_ERR_NO_MEMORY) {
                bool none_running;
                {
                    std::lock_guard<std::mutex> lk(S->m);
                    none_running = S->running.empty();
                }
                cudaStreamSynchronize(t->job.s);
                {
                    std::lock_guard<std::recursive_mutex> lk(S->ctx->mu);
                    grid_free_work(t->g);
                }
                if (none_running) {   // it can never fit
                    complete(S, t, HG_ERR_NO_MEMORY);
                    continue;
                }
                std::lock_guard<std::mutex> lk(S->m);
                // wait for memory: back to the front of the queue, with the rest
                for (size_t k = admit.size(); k-- > i;) S->queue.push_front(admit[k]);
                break;
            }
            if (st != HG_OK) { complete(S, t, st); continue; }
            std::lock_guard<std::mutex> lk(S->m);
            t->state = T_RUNNING;
            S->running.push_back(t);
        }
        // progress every running request whose last step has completed
        std::vector<Ticket*> snap;
        {
            std::lock_guard<std::mutex> lk(S->m);
            snap = S->running;
        }
        bool progressed = false;
        for (Ticket* t : snap) {
            if (t->cancel_req) { complete(S, t, HG_ERR_CANCELLED); progressed = true; continue; }
            cudaError_t q = cudaEventQuery(t->job.tick);
            if (q == cudaErrorNotReady) continue;
            progressed = true;
            if (q != cudaSuccess) {
                set_last_cuda_error(q, "cudaEventQuery");
                complete(S, t, HG_ERR_CUDA);
                continue;
            }
            bool done = false;
            int st;
            {
                std::lock_guard<std::recursive_mutex> lk(S->ctx->mu);
                st = job_advance(t->job, &done);
            }
            if (st != HG_OK) { complete(S, t, st); continue; }
            if (done) {
                t->res = t->job.res;
                complete(S, t, t->job.result);
            }
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

Scheduler* sched_create(hg_ctx* ctx) {
    Scheduler* S = new Scheduler();
    S->ctx = ctx;
    return S;
}

static void ensure_started(Scheduler* S) {
    // caller holds S->m
    if (S->started) return;
    cudaSetDevice(S->ctx->device);
    for (int i = 0; i < 16; ++i) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess) S->streams.push_back(s);
    }
    if (S->streams.empty()) S->streams.push_back(S->ctx->stream);
    S->th = std::thread(worker, S);
    S->started = true;
}

void sched_destroy(Scheduler* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->m);
        S->stop = true;
        for (Ticket* t : S->running) t->cancel_req = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    for (Ticket* t : S->running) {
        if (t->job.s) cudaStreamSynchronize(t->job.s);
        grid_free_work(t->g);
        t->g->borrowed -= 1;
    }
    for (Ticket* t : S->queue) t->g->borrowed -= 1;
    for (cudaStream_t s : S->streams)
        if (s != S->ctx->stream) cudaStreamDestroy(s);
    delete S;
}

int sched_submit(Scheduler* S, hg_grid* g, const hg_solve_opts* opts, uint64_t* ticket) {
    hg_solve_opts o;
    if (opts) o = *opts; else hg_default_opts(&o);
    const int vst = validate_solve_opts(g, &o);
    if (vst) return vst;
    o.time_pass = -1;   // per-pass timing is a blocking-solve diagnostic
    if (g->coeff_mode < 0) return HG_ERR_NO_COEFFS;
    int expect = 0;
    if (!g->borrowed.compare_exchange_strong(expect, 1)) return HG_ERR_BUSY;
    std::unique_ptr<Ticket> t(new Ticket());
    t->g = g;
    t->job.o = o;
    std::lock_guard<std::mutex> lk(S->m);
    ensure_started(S);
    t->id = S->next_id++;
    *ticket = t->id;
    S->queue.push_back(t.get());
    S->tickets[t->id] = std::move(t);
    S->cv_work.notify_all();
    return HG_OK;
}

int sched_poll(Scheduler* S, uint64_t ticket, hg_result* out, int timeout_us) {
    std::unique_lock<std::mutex> lk(S->m);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return HG_ERR_ARG;
    Ticket* t = it->second.get();
    if (t->state != T_DONE && timeout_us != 0) {
        auto pred = [&] { return t->state == T_DONE; };
        if (timeout_us < 0) S->cv_done.wait(lk, pred);
        else S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred);
    }
    if (t->state != T_DONE) return HG_PENDING;
    if (out) *out = t->res;
    const int st = t->status;
    S->tickets.erase(it);
    return st;
}

int sched_cancel(Scheduler* S, uint64_t ticket) {
    std::lock_guard<std::mutex> lk(S->m);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return HG_ERR_ARG;
    Ticket* t = it->second.get();
    if (t->state == T_DONE) return HG_OK;
    if (t->state == T_QUEUED) {
        auto q = std::find(S->queue.begin(), S->queue.end(), t);
        if (q == S->queue.end()) {   // being admitted right now: the worker ends it
            t->cancel_req = true;
            return HG_OK;
        }
        S->queue.erase(q);
        t->state = T_DONE;
        t->status = HG_ERR_CANCELLED;
        t->res.status = HG_ERR_CANCELLED;
        t->g->borrowed -= 1;
        S->cv_done.notify_all();
        return HG_OK;
    }
    t->cancel_req = true;
    return HG_OK;
}

}  // namespace hgrt
