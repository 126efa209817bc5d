// Request scheduler behind hg_submit / hg_poll / hg_cancel.
//
// Continuous batching across requests.  Requests for the standard CG on
// Eq. final_system (primal, A0 = I) join the rolling batch of their precision
// (hg_batch.cpp): every chunk steps ALL of them by check_every iterations, with
// one batched launch per pass and grid shape for every request of that shape,
// and their FP64 refinement steps batched per shape beside the next chunk; a
// tick enqueues one chunk and reads the one before, so the device always has
// the next chunk queued; new requests join and finished ones leave between
// ticks.  Other requests (Moulinec-Suquet, the
// dual formulation, a general reference medium) run as resumable per-request
// jobs on their own streams, overlapping the batch on the device.  Every
// admitted request keeps its CG state resident on the device.  Admission
// compares the bytes a request still has to allocate with the context budget
// before allocating anything; a request that does not fit waits (in arrival
// order) until a completed request has released memory.
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
    bool rolling = false;     // a member of a rolling batch (else a per-request job)
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
    int max_running = 64;       // per-request jobs in flight
    int max_rolling = 1024;     // members of the rolling batches
    Rolling* roll[2] = {nullptr, nullptr};   // per precision (0 FP64, 1 mixed)
    std::atomic<bool> mem_released{true};    // a completion freed memory since the last blocked admission
};

static bool rolling_eligible(const hg_solve_opts& o) {
    return o.method == HG_CG && o.formulation == HG_PRIMAL && o.A0[0] == 0.0 && o.time_pass < 0;
}

static void complete(Scheduler* S, Ticket* t, int status) {
    // the ticket's work is finished or abandoned: make sure nothing is in flight.
    // Its device buffers stay allocated (reused by the next request on this
    // grid; reclaimed by admission when the budget is short).
    if (t->job.s) cudaStreamSynchronize(t->job.s);
    S->mem_released = true;
    std::lock_guard<std::mutex> lk(S->m);
    t->status = status;
    t->res.status = status;
    t->state = T_DONE;
    t->g->borrowed -= 1;
    S->running.erase(std::remove(S->running.begin(), S->running.end(), t), S->running.end());
    S->cv_done.notify_all();
}

// Whether a request fits the budget now.  When it does not and some memory
// has been released since the last blocked admission, the solver state of
// idle grids (no ticket) is released and the test repeated.
static bool fits_budget(Scheduler* S, hg_grid* g, size_t need) {
    hg_ctx* c = S->ctx;
    if (!c->budget || c->used.load() + need <= c->budget) return true;
    if (!S->mem_released.exchange(false)) return false;
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    ctx_reclaim(c, g);
    return c->used.load() + need <= c->budget;
}

static bool nothing_running(Scheduler* S) {
    std::lock_guard<std::mutex> lk(S->m);
    return S->running.empty();
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
            int jobs = 0, members = 0;
            for (Ticket* t : S->running) (t->rolling ? members : jobs) += 1;
            while (!S->queue.empty()) {
                Ticket* t = S->queue.front();
                const bool roll = rolling_eligible(t->job.o);
                if (roll ? members >= S->max_rolling : jobs >= S->max_running) break;
                (roll ? members : jobs) += 1;
                admit.push_back(t);
                S->queue.pop_front();
            }
        }
        // admission: the request's resident state, then its first steps
        for (size_t i = 0; i < admit.size(); ++i) {
            Ticket* t = admit[i];
            if (t->cancel_req) { complete(S, t, HG_ERR_CANCELLED); continue; }
            const hg_solve_opts& o = t->job.o;
            const int prec = o.prec == HG_MIXED ? 1 : 0;
            Rolling* R = nullptr;
            if (rolling_eligible(o)) {
                if (!S->roll[prec]) S->roll[prec] = rolling_create(S->ctx, prec, o.check_every);
                R = S->roll[prec];
                if (R && rolling_chunk(R) != std::max(1, o.check_every)) R = nullptr;   // its own job
            }
            size_t need;
            {
                std::lock_guard<std::recursive_mutex> lk(S->ctx->mu);
                if (R) t->g->use_plane = o.resident != 0;   // its shape in the batch
                need = solve_bytes_needed(t->g, prec, R ? rolling_nbx(R, t->g) : 0);
            }
            int st = HG_ERR_NO_MEMORY;
            if (fits_budget(S, t->g, need)) {
                std::lock_guard<std::recursive_mutex> lk(S->ctx->mu);
                if (R) {
                    st = rolling_add(R, t->g, o, t->id);
                } else {
                    t->job.g = t->g;
                    t->job.s = S->streams[S->next_stream++ % S->streams.size()];
                    t->job.ev0 = t->g->ev0;
                    t->job.ev1 = t->g->ev1;
                    t->job.tick = t->g->ev_tick;
                    st = job_begin(t->job);
                }
                if (st == HG_ERR_NO_MEMORY) {
                    // the estimate missed (fragmentation, another context): drop
                    // what this attempt allocated before waiting
                    if (t->job.s) cudaStreamSynchronize(t->job.s);
                    if (R) cudaDeviceSynchronize();
                    grid_free_work(t->g);
                }
            }
            if (st == HG_ERR_NO_MEMORY) {
                if (nothing_running(S)) {   // it can never fit
                    complete(S, t, HG_ERR_NO_MEMORY);
                    continue;
                }
                // wait for a completion to release memory: back to the front of
                // the queue, with the rest of this admission round
                std::lock_guard<std::mutex> lk(S->m);
                for (size_t k = admit.size(); k-- > i;) S->queue.push_front(admit[k]);
                break;
            }
            if (st != HG_OK) { complete(S, t, st); continue; }
            std::lock_guard<std::mutex> lk(S->m);
            t->rolling = R != nullptr;
            t->state = T_RUNNING;
            S->running.push_back(t);
        }
        // per-request jobs whose last step has completed
        std::vector<Ticket*> snap;
        {
            std::lock_guard<std::mutex> lk(S->m);
            snap = S->running;
        }
        bool progressed = false;
        for (Ticket* t : snap) {
            if (t->rolling) {
                if (t->cancel_req) {
                    {
                        std::lock_guard<std::recursive_mutex> lk(S->ctx->mu);
                        for (Rolling* R : S->roll)
                            if (R) rolling_remove(R, t->id);
                    }
                    complete(S, t, HG_ERR_CANCELLED);
                    progressed = true;
                }
                continue;
            }
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
        // one tick of every rolling batch: all its members step together
        for (int pr = 0; pr < 2; ++pr) {
            Rolling* R = S->roll[pr];
            if (!R || rolling_size(R) == 0) continue;
            std::vector<RollDone> fin;
            int st;
            {
                std::lock_guard<std::recursive_mutex> lk(S->ctx->mu);
                st = rolling_tick(R, &fin);
            }
            progressed = true;
            std::vector<Ticket*> members;
            {
                std::lock_guard<std::mutex> lk(S->m);
                for (Ticket* t : S->running)
                    if (t->rolling && t->job.o.prec == (pr ? HG_MIXED : HG_FP64)) members.push_back(t);
            }
            if (st != HG_OK) {
                // the batch cannot go on: every member ends with the error
                {
                    std::lock_guard<std::recursive_mutex> lk(S->ctx->mu);
                    rolling_destroy(R);
                }
                S->roll[pr] = nullptr;
                for (Ticket* t : members) complete(S, t, st);
                continue;
            }
            for (const RollDone& d : fin)
                for (Ticket* t : members)
                    if (t->id == d.tag) {
                        t->res = d.res;
                        complete(S, t, d.status);
                        break;
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
    for (Rolling*& R : S->roll) {
        rolling_destroy(R);
        R = nullptr;
    }
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
