// hg_solve_batch: many problems stepped together.
//
// Problems of one grid shape form a group.  Every pass of the CG iteration
// (and of the right-hand side, the projection of the correction and the FP64
// residual) is one launch for all problems of a group: the pass kernels take
// the arguments of problem p from a device array (grid z = problem), so a
// group of small grids fills the GPU in one launch where single solves would
// each be bound by launch latency.  The CG iterations of the whole batch are
// captured `check_every` at a time in ONE CUDA graph with one branch per
// group, so the groups' passes overlap on the device and one graph launch
// steps every problem; each problem keeps its own scalars, convergence status
// and reduction slots, and a converged problem's tiles exit at once.  In mixed
// precision a problem whose inner FP32 solve has stopped gets its FP64
// refinement step (batched per shape) on a second stream while the next
// chunk runs, so problems progress independently.  The small per-problem
// steps (scalar set-up, inner set-up, x64 += delta, A_H) are plain per-grid
// launches.
#include "hg.h"
#include "hg_internal.h"
#include "hg_runtime.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <vector>

using namespace hgk;
using namespace hgrt;

#define HG_CU(call)                                  \
    do {                                             \
        cudaError_t _e = (call);                     \
        if (_e != cudaSuccess) {                     \
            set_last_cuda_error(_e, #call);          \
            return HG_ERR_CUDA;                      \
        }                                            \
    } while (0)

namespace {

double wall_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// Device copies of the per-problem arguments of one operator application.
struct BatchItems {
    RowFwdArgs* fa = nullptr;
    StrArgs* sa[3] = {nullptr, nullptr, nullptr};
    RowInvArgs* ia = nullptr;
    PassArgs first;   // problem 0's arguments: the shared geometry of the launches
};

// One device allocation per batch call, freed at the end.
struct Arena {
    hg_ctx* ctx = nullptr;
    std::vector<void*> blocks;
    ~Arena() {
        for (void* p : blocks) dev_free(ctx, p);
    }
    int get(size_t bytes, void** out) {
        int st = dev_alloc(ctx, out, bytes);
        if (st == HG_OK) blocks.push_back(*out);
        return st;
    }
};

// Device arrays for the items of up to cap problems.
int alloc_items(Arena& ar, size_t cap, BatchItems* it) {
    int st;
    if ((st = ar.get(cap * sizeof(RowFwdArgs), (void**)&it->fa))) return st;
    if ((st = ar.get(cap * sizeof(RowInvArgs), (void**)&it->ia))) return st;
    for (int k = 0; k < 3; ++k)
        if ((st = ar.get(cap * sizeof(StrArgs), (void**)&it->sa[k]))) return st;
    return HG_OK;
}

// Copies the items of pas into it's arrays (allocated for at least
// pas.size() problems), on stream s after the work already enqueued there.
int copy_items(const std::vector<PassArgs>& pas, cudaStream_t s, BatchItems* it) {
    const size_t P = pas.size();
    std::vector<RowFwdArgs> fa(P);
    std::vector<RowInvArgs> ia(P);
    std::vector<StrArgs> sa(P);
    for (size_t p = 0; p < P; ++p) { fa[p] = pas[p].fa; ia[p] = pas[p].ia; }
    HG_CU(cudaMemcpyAsync(it->fa, fa.data(), P * sizeof(RowFwdArgs), cudaMemcpyHostToDevice, s));
    HG_CU(cudaMemcpyAsync(it->ia, ia.data(), P * sizeof(RowInvArgs), cudaMemcpyHostToDevice, s));
    for (int k = 0; k < pas[0].nstr; ++k) {
        for (size_t p = 0; p < P; ++p) sa[p] = pas[p].sa[k];
        HG_CU(cudaMemcpyAsync(it->sa[k], sa.data(), P * sizeof(StrArgs), cudaMemcpyHostToDevice, s));
    }
    // the host vectors are pageable: cudaMemcpyAsync has staged them on return
    it->first = pas[0];
    return HG_OK;
}

int upload_items(Arena& ar, const std::vector<PassArgs>& pas, cudaStream_t s, BatchItems* it) {
    int st = alloc_items(ar, pas.size(), it);
    return st ? st : copy_items(pas, s, it);
}

// The launches of one operator application for all P problems.
// rc: the row tile of the last-axis passes (the group's), the strided passes
// run g0's geometry.
int launch_batch(hg_grid* g0, const RowCfg& rc, int prec, const BatchItems& it, int P, cudaStream_t s) {
    const GridDev& gd = g0->gd;
    const int last = gd.d - 1;
    const int L = it.first.fa.L;
    if (it.first.plane) {
        const float2* tw = static_cast<const float2*>(g0->tw[1]) + g0->plan[last].tw_off;
        const StrArgs& a = it.first.sa[0];
        HG_CU(launch_plane_fwd_batch(gd, tw, it.fa, P, L, s));
        HG_CU(launch_strided_batch(prec, gd, g0->plan[0], g0->tw[prec], g0->strcfg[prec][0], it.sa[0], P, L, a.n,
                                   a.inner, a.outer, s));
        HG_CU(launch_plane_inv_batch(gd, tw, it.ia, P, L, s));
        g0->ctx->launches += 3;
        return HG_OK;
    }
    HG_CU(launch_row_fwd_batch(prec, gd, g0->plan[last], g0->tw[prec], rc, it.fa, P, L, s));
    g0->ctx->launches++;
    for (int k = 0; k < it.first.nstr; ++k) {
        const StrArgs& a = it.first.sa[k];
        HG_CU(launch_strided_batch(prec, gd, g0->plan[a.axis], g0->tw[prec], g0->strcfg[prec][a.axis], it.sa[k],
                                   P, L, a.n, a.inner, a.outer, s));
        g0->ctx->launches++;
    }
    HG_CU(launch_row_inv_batch(prec, gd, g0->plan[last], g0->tw[prec], rc, it.ia, P, L, s));
    g0->ctx->launches++;
    return HG_OK;
}

// Problems of one grid shape: every pass one launch for all of them.
struct Group {
    std::vector<hg_grid*> gs;
    std::vector<int> pos;        // their positions in the batch
    int P = 0, L = 0;
    RowCfg rc[2];                // row tile of the last-axis passes, per precision
    BatchItems refine[3];        // items of the refinement launches (FP32 projection,
                                 // FP64 projection, FP64 residual), capacity P
    cudaStream_t side = nullptr; // capture branch of this group
    cudaEvent_t join = nullptr;
};

struct Batch {
    std::vector<hg_grid*> gs;    // every problem, in the caller's order
    std::vector<Group> groups;
    hg_solve_opts o{};
    int P = 0, prec = 0;
    cudaStream_t s = nullptr;
    Arena ar;
    const Scalars** d_src = nullptr;         // per-problem outer, then inner, scalar pointers (device)
    Scalars* d_gather = nullptr;
    Scalars* h_gather = nullptr;              // pinned
    cudaGraphExec_t cg_exec = nullptr;
    long long nk = 0;                        // launches per iteration of the captured graph
    cudaEvent_t fork = nullptr;
    cudaStream_t side = nullptr;             // refinement steps (mixed), beside the graph chunks
    cudaEvent_t refined = nullptr;
    ~Batch() {
        if (cg_exec) cudaGraphExecDestroy(cg_exec);
        if (h_gather) cudaFreeHost(h_gather);
        for (Group& gr : groups) {
            if (gr.join) cudaEventDestroy(gr.join);
            if (gr.side) cudaStreamDestroy(gr.side);
        }
        if (fork) cudaEventDestroy(fork);
        if (refined) cudaEventDestroy(refined);
        if (side) cudaStreamDestroy(side);
    }
};

// Copies every problem's outer scalars (inner = false) to h_gather[0, P), or
// the outer and the inner ones (inner = true) to h_gather[0, P) and [P, 2P).
int read_scalars(Batch& b, bool inner) {
    const int n = inner ? 2 * b.P : b.P;
    HG_CU(launch_gather_scalars(b.d_src, b.d_gather, n, b.s));
    HG_CU(cudaMemcpyAsync(b.h_gather, b.d_gather, sizeof(Scalars) * MAXL * n, cudaMemcpyDeviceToHost, b.s));
    HG_CU(cudaStreamSynchronize(b.s));
    return HG_OK;
}

bool any_load(const Batch& b, int p, bool inner, int status) {
    const Scalars* h = b.h_gather + (size_t)(inner ? b.P + p : p) * MAXL;
    for (int l = 0; l < b.gs[p]->gd.d; ++l)
        if (h[l].status == status) return true;
    return false;
}

int make_items(Batch& b, Group& gr, BatchItems* it, int prec, const void* const* u, bool unit_loads, bool withA,
               int inv_mode, bool outer_status) {
    std::vector<PassArgs> pas(gr.P);
    for (int p = 0; p < gr.P; ++p) {
        hg_grid* g = gr.gs[p];
        matvec_args(g, prec, gr.L, u ? u[p] : nullptr, unit_loads, withA, nullptr, nullptr, inv_mode, nullptr, 1,
                    outer_status ? g->work[0].sc : nullptr, &pas[p]);
    }
    return upload_items(b.ar, pas, b.s, it);
}

// The CUDA graph of check_every batched CG iterations of precision prec over
// the problems marked in `member`: one branch per grid shape (the shapes'
// passes overlap on the device), each a chain of that shape's batched
// launches with its group's launch geometry.  Returns the problems captured.
int make_cg_graph(Batch& b, int prec, const std::vector<char>& member, int* captured) {
    const size_t G = b.groups.size();
    std::vector<BatchItems> its(G);
    std::vector<int> cnt(G, 0);
    int st;
    *captured = 0;
    for (size_t k = 0; k < G; ++k) {
        Group& gr = b.groups[k];
        std::vector<PassArgs> pas;
        for (int p = 0; p < gr.P; ++p) {
            if (!member[gr.pos[p]]) continue;
            pas.emplace_back();
            cg_iteration_args(gr.gs[p], prec, gr.L, &pas.back());
        }
        cnt[k] = (int)pas.size();
        *captured += cnt[k];
        if (cnt[k] && (st = upload_items(b.ar, pas, b.s, &its[k]))) return st;
    }
    HG_CU(cudaStreamSynchronize(b.s));
    hg_ctx* c = b.gs[0]->ctx;
    cudaStream_t cs = c->cap_stream;
    const long long before = c->launches.load();
    const int chunk = std::max(1, b.o.check_every);
    b.nk = 0;
    HG_CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(b.fork, cs);
    st = HG_OK;
    int on_cs = -1;   // the first captured group runs on the capture stream itself
    for (size_t k = 0; k < G && e == cudaSuccess && st == HG_OK; ++k) {
        if (!cnt[k]) continue;
        Group& gr = b.groups[k];
        b.nk += gr.gs[0]->gd.d + 1;
        cudaStream_t ss = cs;
        if (on_cs < 0) {
            on_cs = (int)k;
        } else {
            ss = gr.side;
            e = cudaStreamWaitEvent(ss, b.fork, 0);
        }
        for (int i = 0; i < chunk && e == cudaSuccess && st == HG_OK; ++i)
            st = launch_batch(gr.gs[0], gr.rc[prec], prec, its[k], cnt[k], ss);
        if (ss != cs && e == cudaSuccess) e = cudaEventRecord(gr.join, ss);
    }
    for (size_t k = 0; k < G && e == cudaSuccess; ++k)
        if (cnt[k] && (int)k != on_cs) e = cudaStreamWaitEvent(cs, b.groups[k].join, 0);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    c->launches -= c->launches.load() - before;   // capture is not execution
    if (st || e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (st) return st;
        set_last_cuda_error(e != cudaSuccess ? e : e2, "batched CG graph capture");
        return HG_ERR_CUDA;
    }
    if (b.cg_exec) { cudaGraphExecDestroy(b.cg_exec); b.cg_exec = nullptr; }
    e = cudaGraphInstantiate(&b.cg_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { set_last_cuda_error(e, "cudaGraphInstantiate"); b.cg_exec = nullptr; return HG_ERR_CUDA; }
    return HG_OK;
}

// The FP64 refinement step of the mixed path for the problems marked in
// `due` (whose inner FP32 solves have stopped), the steps of their single
// solves: delta <- Gamma_N delta (FP32), x64 += delta, x64 <- Gamma_N x64
// (FP64, tol < 1e-8), r = -G A (E + x64) (FP64).  Per grid shape the
// projections and the residual are one launch per pass for all its due
// problems.  Enqueued on stream s; restart_due() then starts their next inner
// solves (idle for the loads the residual found converged).
int refine_due(Batch& b, const std::vector<char>& due, cudaStream_t s) {
    hg_ctx* c = b.gs[0]->ctx;
    int st;
    for (Group& gr : b.groups) {
        std::vector<hg_grid*> sub;
        for (int i = 0; i < gr.P; ++i)
            if (due[gr.pos[i]]) sub.push_back(gr.gs[i]);
        if (sub.empty()) continue;
        const int n = (int)sub.size(), L = gr.L;
        std::vector<PassArgs> pas(n);
        for (int i = 0; i < n; ++i)
            matvec_args(sub[i], 1, L, sub[i]->work[1].x, false, false, nullptr, nullptr, INV_PROJ, nullptr, 1,
                        sub[i]->work[0].sc, &pas[i]);
        if ((st = copy_items(pas, s, &gr.refine[0])) || (st = launch_batch(gr.gs[0], gr.rc[1], 1, gr.refine[0], n, s)))
            return st;
        for (hg_grid* g : sub) {
            HG_CU(launch_outer_update(g->gd, L, (double*)g->work[0].x, (const float*)g->work[1].x, g->work[0].sc,
                                      g->work[1].sc, s));
            c->launches++;
        }
        if (b.o.tol < 1e-8) {
            for (int i = 0; i < n; ++i)
                matvec_args(sub[i], 0, L, sub[i]->work[0].x, false, false, nullptr, nullptr, INV_PROJ, nullptr, 1,
                            nullptr, &pas[i]);
            if ((st = copy_items(pas, s, &gr.refine[1])) || (st = launch_batch(gr.gs[0], gr.rc[0], 0, gr.refine[1], n, s)))
                return st;
        }
        for (int i = 0; i < n; ++i)
            matvec_args(sub[i], 0, L, sub[i]->work[0].x, true, true, nullptr, nullptr, INV_RESID, nullptr, 1, nullptr,
                        &pas[i]);
        if ((st = copy_items(pas, s, &gr.refine[2])) || (st = launch_batch(gr.gs[0], gr.rc[0], 0, gr.refine[2], n, s)))
            return st;
    }
    return HG_OK;
}

// A_H (energy and flux forms) of a problem whose iteration has ended, and its
// copy to the host, on stream s.
int finish_one(Batch& b, hg_grid* g, cudaStream_t s) {
    const GridDev& gd = g->gd;
    HG_CU(launch_energy(gd, gd.d, coeffs_for(g, 0, true), (const double*)g->work[0].x,
                        b.o.loads_mask & ((1u << gd.d) - 1u), g->partial, g->counters + 5, g->d_AH, s));
    g->ctx->launches++;
    HG_CU(cudaMemcpyAsync(g->h_AH, g->d_AH, sizeof(double) * 2 * gd.d * gd.d, cudaMemcpyDeviceToHost, s));
    return HG_OK;
}

int restart_due(Batch& b, const std::vector<char>& due, cudaStream_t s) {
    for (int p = 0; p < b.P; ++p) {
        if (!due[p]) continue;
        hg_grid* g = b.gs[p];
        HG_CU(launch_inner_init(g->gd, g->gd.d, (const double*)g->work[0].r, (float*)g->work[1].r,
                                (float*)g->work[1].p, (float*)g->work[1].x, g->work[0].sc, g->work[1].sc,
                                b.o.inner_tol, b.o.max_iter, 64, grid_weight(g), g->partial, g->counters + 4, s));
        g->ctx->launches++;
    }
    return HG_OK;
}

// Steps the batch in graph chunks until no problem is active.  FP64: the CG
// of every problem.  Mixed: the inner FP32 CG in the graph; a problem whose
// inner solve has stopped gets its FP64 refinement step on a second stream
// while the next chunk runs (its tiles in that chunk exit at once: its inner
// status is not active), and its next inner solve starts before the chunk
// after, so the problems progress independently and the FP64 refinement
// overlaps the FP32 iterations of the others.  When the problems still
// running fall to 3/4 of those captured, the graph is captured again over them
// alone (converged problems cost no launches).
int run_batch(Batch& b) {
    const bool mixed = b.prec == 1;
    const int chunk = std::max(1, b.o.check_every);
    std::vector<char> member(b.P, 1);
    int captured = 0, st;
    if ((st = make_cg_graph(b, b.prec, member, &captured))) return st;
    const long long max_chunks =
        (mixed ? (long long)std::max(1, b.o.max_outer) : 1LL) * ((long long)b.o.max_iter / chunk + 3) + 2;
    std::vector<char> due(b.P, 0), refining(b.P, 0), finished(b.P, 0);
    int nrefining = 0;
    for (long long k = 0;; ++k) {
        HG_CU(cudaGraphLaunch(b.cg_exec, b.s));
        b.gs[0]->ctx->launches += b.nk * chunk;
        if (nrefining) {
            // the refinement steps enqueued on the side stream during this chunk
            HG_CU(cudaEventRecord(b.refined, b.side));
            HG_CU(cudaStreamWaitEvent(b.s, b.refined, 0));
        }
        if ((st = read_scalars(b, mixed))) return st;
        // refined problems start their next inner solve in the next chunk
        if (nrefining && (st = restart_due(b, refining, b.s))) return st;
        int running = 0, ndue = 0;
        for (int p = 0; p < b.P; ++p) {
            member[p] = 0;
            due[p] = 0;
            if (!any_load(b, p, false, ST_ACTIVE)) continue;
            member[p] = 1;
            ++running;
            if (!mixed || refining[p] || any_load(b, p, true, ST_ACTIVE)) continue;
            // inner solve stopped: refine, unless the refinement steps are spent
            // (the outer scalars count them)
            const Scalars* ho = b.h_gather + (size_t)p * MAXL;
            int steps = 0;
            for (int l = 0; l < b.gs[p]->gd.d; ++l)
                if (ho[l].status == ST_ACTIVE) steps = std::max(steps, ho[l].iters);
            if (steps >= std::max(1, b.o.max_outer)) {
                member[p] = 0;
                --running;
                continue;
            }
            due[p] = 1;
            ++ndue;
        }
        refining.swap(due);
        nrefining = ndue;
        // problems whose iteration ended in this chunk: their A_H on the side
        // stream, beside the chunks of the others
        bool any_new = false;
        for (int p = 0; p < b.P; ++p) any_new |= !member[p] && !finished[p];
        if (nrefining || any_new) {
            // after this chunk's reads, before the next chunk
            HG_CU(cudaEventRecord(b.refined, b.s));
            HG_CU(cudaStreamWaitEvent(b.side, b.refined, 0));
        }
        for (int p = 0; p < b.P; ++p) {
            if (member[p] || finished[p]) continue;
            finished[p] = 1;
            if ((st = finish_one(b, b.gs[p], b.side))) return st;
        }
        if (nrefining && (st = refine_due(b, refining, b.side))) return st;
        if (running == 0 || k + 1 >= max_chunks) break;
        if (4 * running <= 3 * captured && (st = make_cg_graph(b, b.prec, member, &captured))) return st;
    }
    // A_H of the problems still running at the chunk limit; then the side
    // stream's work (refinements in flight, A_H) joins the main stream
    for (int p = 0; p < b.P; ++p)
        if (!finished[p]) {
            finished[p] = 1;
            if ((st = finish_one(b, b.gs[p], b.side))) return st;
        }
    HG_CU(cudaEventRecord(b.refined, b.side));
    HG_CU(cudaStreamWaitEvent(b.s, b.refined, 0));
    return HG_OK;
}

void load_status(const Batch& b, int L, int* init_st) {
    for (int l = 0; l < MAXL; ++l) init_st[l] = (l < L && ((b.o.loads_mask >> l) & 1u)) ? ST_ACTIVE : ST_IDLE;
}

int start_rhs(Batch& b, bool fp32) {
    for (hg_grid* g : b.gs) {
        int init_st[MAXL];
        load_status(b, g->gd.d, init_st);
        HG_CU(launch_init_scalars(g->work[0].sc, g->gd.d, init_st, b.o.tol, b.prec ? b.o.max_outer : b.o.max_iter,
                                  0.0, 1.0, b.s));
        g->ctx->launches++;
    }
    int st;
    for (Group& gr : b.groups) {
        BatchItems it;
        if (!fp32) {
            if ((st = make_items(b, gr, &it, 0, nullptr, true, true, INV_RHS, false))) return st;
            if ((st = launch_batch(gr.gs[0], gr.rc[0], 0, it, gr.P, b.s))) return st;
            if (b.prec == 0) continue;
            for (hg_grid* g : gr.gs) {
                const GridDev& gd = g->gd;
                HG_CU(launch_inner_init(gd, gr.L, (const double*)g->work[0].r, (float*)g->work[1].r,
                                        (float*)g->work[1].p, (float*)g->work[1].x, g->work[0].sc, g->work[1].sc,
                                        b.o.inner_tol, b.o.max_iter, 64, grid_weight(g), g->partial,
                                        g->counters + 4, b.s));
                g->ctx->launches++;
            }
            continue;
        }
        for (hg_grid* g : gr.gs)
            HG_CU(cudaMemsetAsync(g->work[0].x, 0, sizeof(double) * (size_t)gr.L * g->gd.d * g->gd.M, b.s));
        if ((st = make_items(b, gr, &it, 1, nullptr, true, true, INV_RHS, true))) return st;
        if ((st = launch_batch(gr.gs[0], gr.rc[1], 1, it, gr.P, b.s))) return st;
        for (hg_grid* g : gr.gs) {
            HG_CU(launch_inner_init(g->gd, gr.L, nullptr, nullptr, nullptr, nullptr, g->work[0].sc, g->work[1].sc,
                                    b.o.inner_tol, b.o.max_iter, 64, grid_weight(g), g->partial, g->counters + 4,
                                    b.s));
            g->ctx->launches++;
        }
    }
    return HG_OK;
}

// One problem's right-hand side in FP64 and its inner start from it.
int restart_rhs64(Batch& b, hg_grid* g) {
    const int L = g->gd.d;
    int init_st[MAXL];
    load_status(b, L, init_st);
    HG_CU(launch_init_scalars(g->work[0].sc, L, init_st, b.o.tol, b.o.max_outer, 0.0, 1.0, b.s));
    g->ctx->launches++;
    int st = enqueue_matvec(g, 0, L, nullptr, true, true, nullptr, nullptr, INV_RHS, nullptr, 1, b.s);
    if (st) return st;
    HG_CU(launch_inner_init(g->gd, L, (const double*)g->work[0].r, (float*)g->work[1].r, (float*)g->work[1].p,
                            (float*)g->work[1].x, g->work[0].sc, g->work[1].sc, b.o.inner_tol, b.o.max_iter, 64,
                            grid_weight(g), g->partial, g->counters + 4, b.s));
    g->ctx->launches++;
    return HG_OK;
}

int map_status(int s) {
    switch (s) {
        case ST_CONVERGED: case ST_ZERO_RHS: case ST_IDLE: case ST_STAGNATED: return HG_OK;
        case ST_MAXITER: case ST_ACTIVE: return HG_ERR_NOT_CONVERGED;
        case ST_BREAKDOWN: return HG_ERR_BREAKDOWN;
        default: return HG_ERR_CUDA;
    }
}

// Row tile of the last-axis passes for P problems of lead's shape in one
// launch: all loads per CTA and the most grid rows per CTA the kernels accept
// while the launch still has at least two CTAs per SM (a batched launch has P
// times the CTAs of a single one, so larger tiles, which stage their twiddles,
// coefficient table and reduction once for more voxels, pay off).  Falls back
// to lead's own tile.
RowCfg batch_row_cfg(const hg_grid* lead, int prec, int P, int sms) {
    const GridDev& gd = lead->gd;
    const int d = gd.d, L = d;
    const size_t csize = prec == 0 ? 16 : 8;
    for (int RB = MAX_REAL_ROWS_HOST; RB >= 1; --RB) {
        RowCfg c{};
        if (!make_row_cfg(prec, gd.Nl, d, L, RB, L, min_radix(lead->plan[d - 1]), csize, lead->ctx->max_smem,
                          gd.rows, c))
            continue;
        if ((long long)P * c.nbx * c.nby >= 2LL * sms) return c;
    }
    return lead->rowcfg[prec];
}

int solve_batch(Batch& b, hg_result* results) {
    hg_grid* g0 = b.gs[0];
    hg_ctx* c = g0->ctx;
    const double t0 = wall_ms();
    const long long launches0 = c->launches.load();
    int st;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    for (Group& gr : b.groups) {
        // every problem of a group runs the group's launch geometry: its
        // reduction slots must hold that many CTAs
        hg_grid* lead = gr.gs[0];
        for (int p = 0; p < 2; ++p)
            gr.rc[p] = b.o.batch_tiles ? batch_row_cfg(lead, p, gr.P, std::max(sms, 1)) : lead->rowcfg[p];
        const long long nbx = std::max(std::max(lead->rowcfg[0].nbx, lead->rowcfg[1].nbx),
                                       std::max(gr.rc[0].nbx, gr.rc[1].nbx));
        for (hg_grid* g : gr.gs) {
            if ((st = grid_alloc_common(g))) return st;
            if ((st = grid_ensure_partial(g, nbx))) return st;
            if ((st = grid_alloc_work(g, 0))) return st;
            if (b.prec == 1 && (st = grid_alloc_work(g, 1))) return st;
            g->form = 0;
            g->has_ref = 0;
            g->use_plane = b.o.resident != 0;
        }
        HG_CU(cudaStreamCreateWithFlags(&gr.side, cudaStreamNonBlocking));
        HG_CU(cudaEventCreateWithFlags(&gr.join, cudaEventDisableTiming));
        if (b.prec == 1)
            for (int k = 0; k < 3; ++k)
                if ((st = alloc_items(b.ar, gr.P, &gr.refine[k]))) return st;
    }
    HG_CU(cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming));
    HG_CU(cudaEventCreateWithFlags(&b.refined, cudaEventDisableTiming));
    HG_CU(cudaStreamCreateWithFlags(&b.side, cudaStreamNonBlocking));
    // per-problem scalar pointers for the gathers: outer, then inner
    std::vector<const Scalars*> src(2 * b.P);
    for (int p = 0; p < b.P; ++p) {
        src[p] = b.gs[p]->work[0].sc;
        src[b.P + p] = b.gs[p]->work[b.prec].sc;
    }
    if ((st = b.ar.get(2 * b.P * sizeof(Scalars*), (void**)&b.d_src))) return st;
    if ((st = b.ar.get(2 * b.P * MAXL * sizeof(Scalars), (void**)&b.d_gather))) return st;
    HG_CU(cudaMallocHost((void**)&b.h_gather, 2 * b.P * MAXL * sizeof(Scalars)));
    HG_CU(cudaMemcpyAsync(b.d_src, src.data(), 2 * b.P * sizeof(Scalars*), cudaMemcpyHostToDevice, b.s));
    HG_CU(cudaEventRecord(g0->ev0, b.s));

    if (b.prec == 0) {
        if ((st = start_rhs(b, false))) return st;
    } else {
        if ((st = start_rhs(b, true))) return st;
        // a problem whose FP32 right-hand side is too small to decide the zero
        // test starts over with the FP64 one, as its single solve does
        if ((st = read_scalars(b, false))) return st;
        for (int p = 0; p < b.P; ++p)
            if (any_load(b, p, false, ST_RHS_RECHECK) && (st = restart_rhs64(b, b.gs[p]))) return st;
    }
    if ((st = run_batch(b))) return st;
    // (run_batch has enqueued every problem's A_H and joined its side stream)
    HG_CU(cudaEventRecord(g0->ev1, b.s));
    if ((st = read_scalars(b, false))) return st;   // outer scalars hold the inner totals
    float dms = 0.f;
    cudaEventElapsedTime(&dms, g0->ev0, g0->ev1);
    const double wall = wall_ms() - t0;
    int overall = HG_OK;
    for (int p = 0; p < b.P; ++p) {
        hg_grid* g = b.gs[p];
        const GridDev& gd = g->gd;
        hg_result& r = results[p];
        memset(&r, 0, sizeof(r));
        r.d = gd.d;
        for (int i = 0; i < gd.d * gd.d; ++i) { r.AH[i] = g->h_AH[i]; r.AH_flux[i] = g->h_AH[gd.d * gd.d + i]; }
        int res = HG_OK;
        for (int l = 0; l < gd.d; ++l) {
            const Scalars& sc = b.h_gather[p * MAXL + l];
            const int ms = map_status(sc.status);
            if (b.prec == 0) {
                r.iters[l] = sc.iters;
            } else {
                r.iters[l] = sc.total_iters;
                r.outer[l] = sc.iters;
            }
            if (ms != HG_OK && res == HG_OK) res = ms;
            r.rel_res[l] = sc.relres;
        }
        r.status = res;
        r.device_ms = dms;   // of the whole batch
        r.wall_ms = wall;
        r.launches = c->launches.load() - launches0;
        g->last_prec = b.prec;
        if (res != HG_OK && overall == HG_OK) overall = res;
    }
    return overall;
}

bool same_shape(const hg_grid* a, const hg_grid* b) {
    if (a->gd.d != b->gd.d) return false;
    for (int k = 0; k < 3; ++k)
        if (a->gd.N[k] != b->gd.N[k] || a->gd.Y[k] != b->gd.Y[k]) return false;
    return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// Rolling batch: cross-request batching for the request scheduler
// ---------------------------------------------------------------------------
// Admitted requests of one precision (standard CG, primal, A0 = I) form one
// rolling batch.  A chunk steps all of them by check_every CG iterations: per
// grid shape each pass is ONE launch for all its requests (the batched pass
// kernels, grid z = request), then every request's scalars are gathered into
// pinned host memory.  Two chunks are in flight: a tick enqueues the next
// chunk, then reads the scalars of the previous one while the GPU runs the
// new one, and enqueues behind it what they call for: the FP64 refinement
// steps (batched per shape) and next inner solves of requests whose inner
// FP32 solve has stopped, the A_H of requests that have finished.  A request
// with host work enqueued sits out (its passes find no active system) until a
// chunk gathered after that work; a finished request's result is returned
// once its A_H has been copied.  New requests join and finished ones leave
// between ticks.  A shape's row tile is fixed when the shape first appears
// (the batch tile for a nominal 64 requests), never taken from the current
// mix, and a batched launch computes every request's tiles and reductions as
// it would alone: a request's result depends neither on which others share
// its chunks nor on when the host reads them.
namespace hgrt {

struct RollShape {
    RowCfg rc[2]{};
    std::vector<int> members;     // indices into Rolling::mem
    BatchItems cg, ref[3];        // CG iteration and refinement items, capacity cap
    std::vector<void*> blocks;    // their device arrays
    int cap = 0;
    cudaStream_t s = nullptr;     // the shape's branch of a chunk
    cudaEvent_t join = nullptr;
    int d = 0, N[3] = {0, 0, 0};
    double Y[3] = {0, 0, 0};
    bool plane = true;            // its members' use_plane (members of a shape agree)
};

struct RollMember {
    hg_grid* g = nullptr;
    uint64_t tag = 0;
    hg_solve_opts o{};
    int shape = -1;
    bool checked = false;         // mixed: the FP32 right-hand side's zero test has been read
    long long valid_from = 0;     // first chunk whose scalars follow the host work enqueued for it
    long long ticks = 0;          // chunks read for it
    double t0 = 0.0;
    long long launches0 = 0;
};

// A chunk whose scalars the host has not read yet.
struct RollGather {
    long long id = -1;
    std::vector<uint64_t> tags;   // its members, in gather order
    Scalars* h = nullptr;         // pinned: outer scalars of every member, then inner
    int cap = 0;                  // members h holds
    cudaEvent_t ev = nullptr;     // recorded after the copy into h
};

// Finished members whose A_H (and FP64 true residual) are being copied.
struct RollRetired {
    RollMember m;
    Scalars outer[MAXL];
};
struct RollRetire {
    std::vector<RollRetired> items;
    cudaEvent_t ev = nullptr;
};

// Pinned staging of the host-to-device uploads of one tick (launch items,
// gather pointers), one per stream that copies (the batch's and the
// refinement stream); a buffer is reused three ticks later, after the copies
// from it have run.
constexpr int ROLL_STAGES = 3;
struct RollStage {
    char* h = nullptr;
    size_t cap = 0, used = 0;
    cudaEvent_t ev = nullptr;
    bool pending = false;
};

struct Rolling {
    hg_ctx* ctx = nullptr;
    int prec = 0, chunk = 8, sms = 1;
    cudaStream_t s = nullptr;
    std::vector<RollMember> mem;
    std::vector<RollShape> shapes;
    bool dirty = true;
    int gcap = 0;                      // members d_src and d_gather hold
    const Scalars** d_src = nullptr;
    Scalars* d_gather = nullptr;
    long long seq = 0;                 // chunks enqueued
    long long nticks = 0;
    RollGather gat[2];                 // chunk id parity
    std::deque<RollGather*> unread;    // enqueue order, at most two
    std::deque<RollRetire> retiring;
    std::vector<cudaEvent_t> ev_pool;
    RollStage stage[2][ROLL_STAGES];   // [0] batch stream, [1] refinement stream
    cudaEvent_t fork = nullptr;
    // FP64 refinement steps run on their own stream, beside the next chunk;
    // the refined members' next inner solves start on the batch's stream
    // before the chunk after that
    cudaStream_t side = nullptr;
    cudaEvent_t refined = nullptr;
    std::vector<uint64_t> restart;
};

static RollStage& roll_stage(Rolling* R, int k) { return R->stage[k][R->nticks % ROLL_STAGES]; }
static cudaStream_t stage_stream(Rolling* R, int k) { return k ? R->side : R->s; }

static int stage_begin(Rolling* R) {
    for (int k = 0; k < 2; ++k) {
        RollStage& st = roll_stage(R, k);
        if (st.pending) {
            HG_CU(cudaEventSynchronize(st.ev));
            st.pending = false;
        }
        st.used = 0;
    }
    return HG_OK;
}

// bytes from host src to device dst on stream k (0 the batch's, 1 the
// refinement stream), through the tick's pinned stage (the copy runs in
// stream order; src may go out of scope)
static int stage_copy(Rolling* R, int k, void* dst, const void* src, size_t bytes) {
    RollStage& st = roll_stage(R, k);
    cudaStream_t s = stage_stream(R, k);
    size_t off = (st.used + 15) & ~size_t(15);
    if (off + bytes > st.cap) {
        // growing: the copies enqueued from this buffer run first
        HG_CU(cudaStreamSynchronize(s));
        const size_t cap = std::max(off + bytes, 2 * st.cap) + ((size_t)64 << 10);
        char* h = nullptr;
        HG_CU(cudaMallocHost((void**)&h, cap));
        if (st.h) cudaFreeHost(st.h);
        st.h = h;
        st.cap = cap;
        off = 0;
    }
    if (!st.ev) HG_CU(cudaEventCreateWithFlags(&st.ev, cudaEventDisableTiming));
    memcpy(st.h + off, src, bytes);
    HG_CU(cudaMemcpyAsync(dst, st.h + off, bytes, cudaMemcpyHostToDevice, s));
    st.used = off + bytes;
    st.pending = true;
    return HG_OK;
}

static int stage_end(Rolling* R) {
    for (int k = 0; k < 2; ++k) {
        RollStage& st = roll_stage(R, k);
        if (st.pending) HG_CU(cudaEventRecord(st.ev, stage_stream(R, k)));
    }
    return HG_OK;
}

static int roll_copy_items(Rolling* R, int k, const std::vector<PassArgs>& pas, BatchItems* it) {
    const size_t P = pas.size();
    std::vector<RowFwdArgs> fa(P);
    std::vector<RowInvArgs> ia(P);
    std::vector<StrArgs> sa(P);
    for (size_t p = 0; p < P; ++p) { fa[p] = pas[p].fa; ia[p] = pas[p].ia; }
    int st;
    if ((st = stage_copy(R, k, it->fa, fa.data(), P * sizeof(RowFwdArgs)))) return st;
    if ((st = stage_copy(R, k, it->ia, ia.data(), P * sizeof(RowInvArgs)))) return st;
    for (int j = 0; j < pas[0].nstr; ++j) {
        for (size_t p = 0; p < P; ++p) sa[p] = pas[p].sa[j];
        if ((st = stage_copy(R, k, it->sa[j], sa.data(), P * sizeof(StrArgs)))) return st;
    }
    it->first = pas[0];
    return HG_OK;
}

static void roll_free_shape(Rolling* R, RollShape& sh) {
    for (void* b : sh.blocks) dev_free(R->ctx, b);
    sh.blocks.clear();
    sh.cap = 0;
}

static int roll_items_alloc(Rolling* R, RollShape& sh, int need) {
    if (need <= sh.cap) return HG_OK;
    const int cap = std::max(need, std::max(8, 2 * sh.cap));
    if (sh.cap) {   // chunks and refinement steps in flight read the old arrays
        HG_CU(cudaStreamSynchronize(R->s));
        HG_CU(cudaStreamSynchronize(R->side));
    }
    roll_free_shape(R, sh);
    BatchItems* all[4] = {&sh.cg, &sh.ref[0], &sh.ref[1], &sh.ref[2]};
    for (BatchItems* it : all) {
        void* p = nullptr;
        int st;
        if ((st = dev_alloc(R->ctx, &p, cap * sizeof(RowFwdArgs)))) return st;
        sh.blocks.push_back(p);
        it->fa = (RowFwdArgs*)p;
        if ((st = dev_alloc(R->ctx, &p, cap * sizeof(RowInvArgs)))) return st;
        sh.blocks.push_back(p);
        it->ia = (RowInvArgs*)p;
        for (int k = 0; k < 3; ++k) {
            if ((st = dev_alloc(R->ctx, &p, cap * sizeof(StrArgs)))) return st;
            sh.blocks.push_back(p);
            it->sa[k] = (StrArgs*)p;
        }
    }
    sh.cap = cap;
    return HG_OK;
}

Rolling* rolling_create(hg_ctx* ctx, int prec, int chunk) {
    Rolling* R = new Rolling();
    R->ctx = ctx;
    R->prec = prec;
    R->chunk = std::max(1, chunk);
    R->sms = std::max(1, ctx->nsm);
    if (cudaStreamCreateWithFlags(&R->s, cudaStreamNonBlocking) != cudaSuccess) {
        delete R;
        return nullptr;
    }
    if (cudaStreamCreateWithFlags(&R->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&R->refined, cudaEventDisableTiming) != cudaSuccess) {
        if (R->side) cudaStreamDestroy(R->side);
        cudaStreamDestroy(R->s);
        delete R;
        return nullptr;
    }
    return R;
}

void rolling_destroy(Rolling* R) {
    if (!R) return;
    cudaStreamSynchronize(R->side);
    cudaStreamSynchronize(R->s);
    for (RollShape& sh : R->shapes) {
        roll_free_shape(R, sh);
        if (sh.s) cudaStreamDestroy(sh.s);
        if (sh.join) cudaEventDestroy(sh.join);
    }
    if (R->fork) cudaEventDestroy(R->fork);
    dev_free(R->ctx, (void*)R->d_src);
    dev_free(R->ctx, R->d_gather);
    for (RollGather& G : R->gat) {
        if (G.h) cudaFreeHost(G.h);
        if (G.ev) cudaEventDestroy(G.ev);
    }
    for (auto& ring : R->stage)
        for (RollStage& st : ring) {
            if (st.h) cudaFreeHost(st.h);
            if (st.ev) cudaEventDestroy(st.ev);
        }
    for (RollRetire& rt : R->retiring) R->ev_pool.push_back(rt.ev);
    for (cudaEvent_t e : R->ev_pool) cudaEventDestroy(e);
    cudaEventDestroy(R->refined);
    cudaStreamDestroy(R->side);
    cudaStreamDestroy(R->s);
    delete R;
}

int rolling_chunk(const Rolling* R) { return R->chunk; }
int rolling_size(const Rolling* R) {
    return (int)(R->mem.size() + R->unread.size() + R->retiring.size());
}

static bool roll_same_shape(const RollShape& sh, const hg_grid* g) {
    if (sh.d != g->gd.d || sh.plane != g->use_plane) return false;
    for (int k = 0; k < 3; ++k)
        if (sh.N[k] != g->gd.N[k] || sh.Y[k] != g->gd.Y[k]) return false;
    return true;
}

static int roll_shape_of(Rolling* R, const hg_grid* g) {
    for (size_t k = 0; k < R->shapes.size(); ++k)
        if (roll_same_shape(R->shapes[k], g)) return (int)k;
    RollShape sh;
    sh.d = g->gd.d;
    sh.plane = g->use_plane;
    for (int k = 0; k < 3; ++k) { sh.N[k] = g->gd.N[k]; sh.Y[k] = g->gd.Y[k]; }
    for (int p = 0; p < 2; ++p) sh.rc[p] = batch_row_cfg(g, p, 64, R->sms);
    R->shapes.push_back(sh);
    return (int)R->shapes.size() - 1;
}

long long rolling_nbx(Rolling* R, const hg_grid* g) {
    const RollShape& sh = R->shapes[roll_shape_of(R, g)];
    return std::max(std::max(g->rowcfg[0].nbx, g->rowcfg[1].nbx), std::max(sh.rc[0].nbx, sh.rc[1].nbx));
}

static void roll_load_status(const hg_solve_opts& o, int L, int* init_st) {
    for (int l = 0; l < MAXL; ++l) init_st[l] = (l < L && ((o.loads_mask >> l) & 1u)) ? ST_ACTIVE : ST_IDLE;
}

int rolling_add(Rolling* R, hg_grid* g, const hg_solve_opts& o, uint64_t tag) {
    const int L = g->gd.d;
    g->use_plane = o.resident != 0;   // (part of the shape key)
    const long long nbx = rolling_nbx(R, g);
    int st;
    if ((st = grid_alloc_common(g))) return st;
    if ((st = grid_ensure_partial(g, nbx))) return st;
    if ((st = grid_alloc_work(g, 0))) return st;
    if (R->prec == 1 && (st = grid_alloc_work(g, 1))) return st;
    g->form = 0;
    g->has_ref = 0;
    // the right-hand side (as a single solve computes it), on the batch's
    // stream behind the chunks already enqueued
    int init_st[MAXL];
    roll_load_status(o, L, init_st);
    HG_CU(launch_init_scalars(g->work[0].sc, L, init_st, o.tol, R->prec ? o.max_outer : o.max_iter, 0.0, 1.0, R->s));
    g->ctx->launches++;
    if (R->prec == 0) {
        if ((st = enqueue_matvec(g, 0, L, nullptr, true, true, nullptr, nullptr, INV_RHS, nullptr, 1, R->s))) return st;
    } else {
        HG_CU(cudaMemsetAsync(g->work[0].x, 0, sizeof(double) * (size_t)L * g->gd.d * g->gd.M, R->s));
        if ((st = enqueue_matvec(g, 1, L, nullptr, true, true, nullptr, nullptr, INV_RHS, nullptr, 1, R->s,
                                 g->work[0].sc)))
            return st;
        HG_CU(launch_inner_init(g->gd, L, nullptr, nullptr, nullptr, nullptr, g->work[0].sc, g->work[1].sc,
                                o.inner_tol, o.max_iter, 64, grid_weight(g), g->partial, g->counters + 4, R->s));
        g->ctx->launches++;
    }
    RollMember m;
    m.g = g;
    m.tag = tag;
    m.o = o;
    m.shape = roll_shape_of(R, g);
    m.checked = R->prec == 0;
    m.valid_from = R->seq;
    m.t0 = wall_ms();
    m.launches0 = g->ctx->launches.load();
    R->mem.push_back(m);
    R->dirty = true;
    return HG_OK;
}

void rolling_remove(Rolling* R, uint64_t tag) {
    cudaStreamSynchronize(R->side);
    cudaStreamSynchronize(R->s);
    for (size_t i = 0; i < R->mem.size(); ++i)
        if (R->mem[i].tag == tag) {
            R->mem.erase(R->mem.begin() + (long)i);
            R->dirty = true;
            break;
        }
    for (RollRetire& rt : R->retiring)
        for (size_t i = 0; i < rt.items.size(); ++i)
            if (rt.items[i].m.tag == tag) {
                rt.items.erase(rt.items.begin() + (long)i);
                break;
            }
}

// Member lists per shape, CG items and gather pointers of the current members
// (uploaded in stream order, behind the chunks in flight).
static int roll_rebuild(Rolling* R) {
    for (RollShape& sh : R->shapes) sh.members.clear();
    for (size_t i = 0; i < R->mem.size(); ++i) R->shapes[R->mem[i].shape].members.push_back((int)i);
    int st;
    for (RollShape& sh : R->shapes) {
        if (sh.members.empty()) continue;
        if ((st = roll_items_alloc(R, sh, (int)sh.members.size()))) return st;
        std::vector<PassArgs> pas(sh.members.size());
        for (size_t i = 0; i < sh.members.size(); ++i) {
            hg_grid* g = R->mem[sh.members[i]].g;
            cg_iteration_args(g, R->prec, g->gd.d, &pas[i]);
        }
        if ((st = roll_copy_items(R, 0, pas, &sh.cg))) return st;
    }
    const int P = (int)R->mem.size();
    if (P > R->gcap) {
        const int cap = std::max(P, std::max(64, 2 * R->gcap));
        HG_CU(cudaStreamSynchronize(R->s));   // the chunk in flight gathers through them
        dev_free(R->ctx, (void*)R->d_src);
        dev_free(R->ctx, R->d_gather);
        R->d_src = nullptr; R->d_gather = nullptr; R->gcap = 0;
        if ((st = dev_alloc(R->ctx, (void**)&R->d_src, 2 * (size_t)cap * sizeof(Scalars*)))) return st;
        if ((st = dev_alloc(R->ctx, (void**)&R->d_gather, 2 * (size_t)cap * MAXL * sizeof(Scalars)))) return st;
        R->gcap = cap;
    }
    std::vector<const Scalars*> src(2 * P);
    for (int p = 0; p < P; ++p) {
        src[p] = R->mem[p].g->work[0].sc;
        src[P + p] = R->mem[p].g->work[R->prec].sc;
    }
    if ((st = stage_copy(R, 0, (void*)R->d_src, src.data(), 2 * P * sizeof(Scalars*)))) return st;
    R->dirty = false;
    return HG_OK;
}

static bool roll_any(const Scalars* h, int L, int status) {
    for (int l = 0; l < L; ++l)
        if (h[l].status == status) return true;
    return false;
}

// check_every iterations of every member, then the gather of their scalars.
// Each shape's iterations run on a stream of their own, so that the launches
// of different shapes overlap on the device (a shape of small grids does not
// fill the GPU alone); the batch's stream waits for all of them.
static int roll_enqueue_chunk(Rolling* R) {
    int st;
    if (!R->fork) HG_CU(cudaEventCreateWithFlags(&R->fork, cudaEventDisableTiming));
    HG_CU(cudaEventRecord(R->fork, R->s));
    for (RollShape& sh : R->shapes) {
        if (sh.members.empty()) continue;
        if (!sh.s) HG_CU(cudaStreamCreateWithFlags(&sh.s, cudaStreamNonBlocking));
        if (!sh.join) HG_CU(cudaEventCreateWithFlags(&sh.join, cudaEventDisableTiming));
        HG_CU(cudaStreamWaitEvent(sh.s, R->fork, 0));
        hg_grid* g0 = R->mem[sh.members[0]].g;   // plans and twiddles of the shape
        for (int i = 0; i < R->chunk; ++i)
            if ((st = launch_batch(g0, sh.rc[R->prec], R->prec, sh.cg, (int)sh.members.size(), sh.s))) return st;
        HG_CU(cudaEventRecord(sh.join, sh.s));
        HG_CU(cudaStreamWaitEvent(R->s, sh.join, 0));
    }
    RollGather& G = R->gat[R->seq & 1];
    for (const RollGather* u : R->unread)
        if (u == &G) return HG_ERR_ARG;   // (a tick leaves at most the newest chunk unread)
    const int P = (int)R->mem.size();
    if (G.cap < P) {
        // (its previous chunk has been read: nothing copies into h)
        const int cap = std::max(P, std::max(64, 2 * G.cap));
        if (G.h) cudaFreeHost(G.h);
        G.h = nullptr;
        G.cap = 0;
        HG_CU(cudaMallocHost((void**)&G.h, 2 * (size_t)cap * MAXL * sizeof(Scalars)));
        G.cap = cap;
    }
    if (!G.ev) HG_CU(cudaEventCreateWithFlags(&G.ev, cudaEventDisableTiming));
    const int n = R->prec == 1 ? 2 * P : P;
    HG_CU(launch_gather_scalars(R->d_src, R->d_gather, n, R->s));
    HG_CU(cudaMemcpyAsync(G.h, R->d_gather, sizeof(Scalars) * MAXL * n, cudaMemcpyDeviceToHost, R->s));
    HG_CU(cudaEventRecord(G.ev, R->s));
    G.id = R->seq++;
    G.tags.resize(P);
    for (int p = 0; p < P; ++p) G.tags[p] = R->mem[p].tag;
    R->unread.push_back(&G);
    return HG_OK;
}

// A_H and the scalars of a finished member as a result.
static RollDone roll_result(const Rolling* R, const RollRetired& it) {
    const bool mixed = R->prec == 1;
    const RollMember& m = it.m;
    hg_grid* g = m.g;
    const GridDev& gd = g->gd;
    RollDone dn;
    memset(&dn, 0, sizeof(dn));
    dn.tag = m.tag;
    hg_result& r = dn.res;
    r.d = gd.d;
    for (int i = 0; i < gd.d * gd.d; ++i) { r.AH[i] = g->h_AH[i]; r.AH_flux[i] = g->h_AH[gd.d * gd.d + i]; }
    int res = HG_OK;
    for (int l = 0; l < gd.d; ++l) {
        const Scalars& sc = it.outer[l];
        const int ms = map_status(sc.status);
        if (mixed) {
            r.iters[l] = sc.total_iters;
            r.outer[l] = sc.iters;
        } else {
            r.iters[l] = sc.iters;
        }
        if (ms != HG_OK && res == HG_OK) res = ms;
        r.rel_res[l] = sc.relres;
        const bool solved = sc.status != ST_IDLE && sc.status != ST_ZERO_RHS && sc.bnorm > 0.0;
        r.true_rel_res[l] = !solved ? 0.0 : (mixed ? sc.relres : g->h_sc[MAXL + l].relres);
    }
    r.status = res;
    r.wall_ms = wall_ms() - m.t0;
    r.launches = g->ctx->launches.load() - m.launches0;
    g->last_prec = R->prec;
    dn.status = res;
    return dn;
}

// Reads the scalars of chunk G and enqueues the host work they call for.
static int roll_read(Rolling* R, RollGather& G) {
    HG_CU(cudaEventSynchronize(G.ev));
    const bool mixed = R->prec == 1;
    const int PG = (int)G.tags.size();
    const int P = (int)R->mem.size();
    std::vector<int> at(P, -1);   // gather position of each current member
    {
        std::vector<std::pair<uint64_t, int>> tj(PG);
        for (int j = 0; j < PG; ++j) tj[j] = {G.tags[j], j};
        std::sort(tj.begin(), tj.end());
        for (int p = 0; p < P; ++p) {
            auto f = std::lower_bound(tj.begin(), tj.end(), std::make_pair(R->mem[p].tag, -1));
            if (f != tj.end() && f->first == R->mem[p].tag) at[p] = f->second;
        }
    }
    std::vector<char> due(P, 0), fin(P, 0);
    bool any_due = false, any_fin = false;
    int st;
    for (int p = 0; p < P; ++p) {
        RollMember& m = R->mem[p];
        const int j = at[p];
        if (j < 0 || G.id < m.valid_from) continue;
        hg_grid* g = m.g;
        const int L = g->gd.d;
        const Scalars* ho = G.h + (size_t)j * MAXL;
        const Scalars* hi = G.h + (size_t)(PG + j) * MAXL;
        m.ticks++;
        if (!m.checked) {
            m.checked = true;
            if (roll_any(ho, L, ST_RHS_RECHECK)) {
                // FP32 right-hand side too small to decide the zero test: the
                // FP64 one, as the single solve does
                int init_st[MAXL];
                roll_load_status(m.o, L, init_st);
                HG_CU(launch_init_scalars(g->work[0].sc, L, init_st, m.o.tol, m.o.max_outer, 0.0, 1.0, R->s));
                g->ctx->launches++;
                if ((st = enqueue_matvec(g, 0, L, nullptr, true, true, nullptr, nullptr, INV_RHS, nullptr, 1, R->s)))
                    return st;
                HG_CU(launch_inner_init(g->gd, L, (const double*)g->work[0].r, (float*)g->work[1].r,
                                        (float*)g->work[1].p, (float*)g->work[1].x, g->work[0].sc, g->work[1].sc,
                                        m.o.inner_tol, m.o.max_iter, 64, grid_weight(g), g->partial,
                                        g->counters + 4, R->s));
                g->ctx->launches++;
                m.valid_from = R->seq;
                continue;
            }
        }
        const long long max_ticks =
            (mixed ? (long long)std::max(1, m.o.max_outer) : 1LL) * ((long long)m.o.max_iter / R->chunk + 3) + 2;
        if (!roll_any(ho, L, ST_ACTIVE) || m.ticks > max_ticks) {
            fin[p] = 1;
            any_fin = true;
            continue;
        }
        if (!mixed || roll_any(hi, L, ST_ACTIVE)) continue;
        // inner solve stopped: refine, unless the refinement steps are spent
        // (the outer scalars count them)
        int steps = 0;
        for (int l = 0; l < L; ++l)
            if (ho[l].status == ST_ACTIVE) steps = std::max(steps, ho[l].iters);
        if (steps >= std::max(1, m.o.max_outer)) {
            fin[p] = 1;
            any_fin = true;
            continue;
        }
        due[p] = 1;
        any_due = true;
    }
    // FP64 refinement steps of the due members, batched per shape (the steps of
    // a single solve: delta <- Gamma delta, x64 += delta, [x64 <- Gamma x64],
    // r = -G A (E + x64)), on the refinement stream beside the chunk now
    // running (whose passes find no active inner system of theirs, so touch
    // none of their buffers); their next inner solves (which start only where
    // the outer residual is still above the tolerance) are launched on the
    // batch's stream before the next chunk
    if (any_due) {
        cudaStream_t sd = R->side;
        for (RollShape& sh : R->shapes) {
            std::vector<int> sub;
            for (int i : sh.members)
                if (i < P && due[i]) sub.push_back(i);
            if (sub.empty()) continue;
            const int ns = (int)sub.size();
            hg_grid* g0 = R->mem[sub[0]].g;
            const int L = g0->gd.d;
            std::vector<PassArgs> pas(ns);
            for (int i = 0; i < ns; ++i) {
                hg_grid* g = R->mem[sub[i]].g;
                matvec_args(g, 1, L, g->work[1].x, false, false, nullptr, nullptr, INV_PROJ, nullptr, 1,
                            g->work[0].sc, &pas[i]);
            }
            if ((st = roll_copy_items(R, 1, pas, &sh.ref[0])) || (st = launch_batch(g0, sh.rc[1], 1, sh.ref[0], ns, sd)))
                return st;
            for (int i : sub) {
                hg_grid* g = R->mem[i].g;
                HG_CU(launch_outer_update(g->gd, L, (double*)g->work[0].x, (const float*)g->work[1].x,
                                          g->work[0].sc, g->work[1].sc, sd));
                g->ctx->launches++;
            }
            std::vector<int> tsub;
            for (int i : sub)
                if (R->mem[i].o.tol < 1e-8) tsub.push_back(i);
            if (!tsub.empty()) {
                std::vector<PassArgs> pt(tsub.size());
                for (size_t i = 0; i < tsub.size(); ++i) {
                    hg_grid* g = R->mem[tsub[i]].g;
                    matvec_args(g, 0, L, g->work[0].x, false, false, nullptr, nullptr, INV_PROJ, nullptr, 1, nullptr,
                                &pt[i]);
                }
                if ((st = roll_copy_items(R, 1, pt, &sh.ref[1])) ||
                    (st = launch_batch(g0, sh.rc[0], 0, sh.ref[1], (int)tsub.size(), sd)))
                    return st;
            }
            for (int i = 0; i < ns; ++i) {
                hg_grid* g = R->mem[sub[i]].g;
                matvec_args(g, 0, L, g->work[0].x, true, true, nullptr, nullptr, INV_RESID, nullptr, 1, nullptr,
                            &pas[i]);
            }
            if ((st = roll_copy_items(R, 1, pas, &sh.ref[2])) || (st = launch_batch(g0, sh.rc[0], 0, sh.ref[2], ns, sd)))
                return st;
            for (int i : sub) {
                RollMember& m = R->mem[i];
                R->restart.push_back(m.tag);
                m.valid_from = R->seq;   // the next chunk follows its inner start
            }
        }
        HG_CU(cudaEventRecord(R->refined, sd));
    }
    if (!any_fin) return HG_OK;
    // finished members: FP64 true residual (FP64 path), A_H; they leave the
    // batch now and their results follow the copies
    RollRetire rt;
    std::vector<RollMember> keep;
    for (int p = 0; p < P; ++p) {
        RollMember& m = R->mem[p];
        if (!fin[p]) {
            keep.push_back(m);
            continue;
        }
        hg_grid* g = m.g;
        const GridDev& gd = g->gd;
        if (!mixed) {
            HG_CU(cudaMemcpyAsync(g->d_sc_aux, g->work[0].sc, sizeof(Scalars) * MAXL, cudaMemcpyDeviceToDevice, R->s));
            if ((st = enqueue_matvec(g, 0, gd.d, g->work[0].x, true, true, nullptr, nullptr, INV_RESID, nullptr, 0,
                                     R->s, g->d_sc_aux)))
                return st;
            HG_CU(cudaMemcpyAsync(g->h_sc + MAXL, g->d_sc_aux, sizeof(Scalars) * MAXL, cudaMemcpyDeviceToHost, R->s));
        }
        HG_CU(launch_energy(gd, gd.d, coeffs_for(g, 0, true), (const double*)g->work[0].x,
                            m.o.loads_mask & ((1u << gd.d) - 1u), g->partial, g->counters + 5, g->d_AH, R->s));
        g->ctx->launches++;
        HG_CU(cudaMemcpyAsync(g->h_AH, g->d_AH, sizeof(double) * 2 * gd.d * gd.d, cudaMemcpyDeviceToHost, R->s));
        RollRetired it;
        it.m = m;
        memcpy(it.outer, G.h + (size_t)at[p] * MAXL, sizeof(it.outer));
        rt.items.push_back(it);
    }
    if (R->ev_pool.empty()) {
        cudaEvent_t e;
        HG_CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        R->ev_pool.push_back(e);
    }
    rt.ev = R->ev_pool.back();
    R->ev_pool.pop_back();
    HG_CU(cudaEventRecord(rt.ev, R->s));
    R->retiring.push_back(rt);
    R->mem.swap(keep);
    R->dirty = true;
    return HG_OK;
}

// Results of retired members whose copies have completed (all of them, waiting,
// when `block`).
static int roll_collect(Rolling* R, std::vector<RollDone>* done, bool block) {
    while (!R->retiring.empty()) {
        RollRetire& rt = R->retiring.front();
        if (block) {
            HG_CU(cudaEventSynchronize(rt.ev));
        } else {
            const cudaError_t q = cudaEventQuery(rt.ev);
            if (q == cudaErrorNotReady) break;
            HG_CU(q);
        }
        for (const RollRetired& it : rt.items) done->push_back(roll_result(R, it));
        R->ev_pool.push_back(rt.ev);
        R->retiring.pop_front();
    }
    return HG_OK;
}

// The next inner solves of the members refined in the last tick, behind their
// refinement steps, on the batch's stream.
static int roll_restart(Rolling* R) {
    if (R->restart.empty()) return HG_OK;
    HG_CU(cudaStreamWaitEvent(R->s, R->refined, 0));
    for (uint64_t tag : R->restart)
        for (RollMember& m : R->mem) {
            if (m.tag != tag) continue;
            hg_grid* g = m.g;
            HG_CU(launch_inner_init(g->gd, g->gd.d, (const double*)g->work[0].r, (float*)g->work[1].r,
                                    (float*)g->work[1].p, (float*)g->work[1].x, g->work[0].sc, g->work[1].sc,
                                    m.o.inner_tol, m.o.max_iter, 64, grid_weight(g), g->partial, g->counters + 4,
                                    R->s));
            g->ctx->launches++;
            break;
        }
    R->restart.clear();
    return HG_OK;
}

int rolling_tick(Rolling* R, std::vector<RollDone>* done) {
    int st;
    if ((st = stage_begin(R))) return st;
    if ((st = roll_restart(R))) return st;
    // the next chunk of the current members (the previous one may still run)
    if (!R->mem.empty()) {
        if (R->dirty && (st = roll_rebuild(R))) return st;
        if ((st = roll_enqueue_chunk(R))) return st;
    }
    // the oldest chunk not read yet, unless it is the only one in flight
    // while members remain (the next tick reads it behind a new chunk)
    if (R->unread.size() >= 2 || (R->mem.empty() && !R->unread.empty())) {
        RollGather* G = R->unread.front();
        R->unread.pop_front();
        if ((st = roll_read(R, *G))) return st;
    }
    if ((st = stage_end(R))) return st;
    R->nticks++;
    return roll_collect(R, done, R->mem.empty() && R->unread.empty());
}

}  // namespace hgrt

extern "C" int hg_solve_batch(hg_grid* const* grids, int n, const hg_solve_opts* opts, hg_result* results) {
    if (!grids || n < 1 || !results) return HG_ERR_ARG;
    hg_grid* g0 = grids[0];
    if (!g0) return HG_ERR_ARG;
    hg_solve_opts o;
    if (opts) o = *opts; else hg_default_opts(&o);
    hg_ctx* c = g0->ctx;
    for (int p = 0; p < n; ++p) {
        hg_grid* g = grids[p];
        if (!g || g->ctx != c) return HG_ERR_ARG;
        hg_solve_opts og = o;
        int st = validate_solve_opts(g, &og);
        if (st) return st;
        if (g->coeff_mode < 0) return HG_ERR_NO_COEFFS;
        if (g->borrowed.load() > 0) return HG_ERR_BUSY;
        for (int q = 0; q < p; ++q)
            if (grids[q] == g) return HG_ERR_ARG;   // each problem needs its own buffers
    }
    if (o.method != HG_CG || o.formulation != HG_PRIMAL || o.A0[0] != 0.0 || o.time_pass != -1) return HG_ERR_ARG;
    if (o.batch_tiles != 0 && o.batch_tiles != 1) return HG_ERR_ARG;
    // loads beyond a problem's d are ignored per problem (its own d loads)
    cudaSetDevice(c->device);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    Batch b;
    b.gs.assign(grids, grids + n);
    b.o = o;
    b.P = n;
    b.prec = o.prec == HG_MIXED ? 1 : 0;
    b.s = c->stream;
    b.ar.ctx = c;
    for (int p = 0; p < n; ++p) {
        Group* gr = nullptr;
        for (Group& q : b.groups)
            if (same_shape(q.gs[0], grids[p])) { gr = &q; break; }
        if (!gr) {
            b.groups.emplace_back();
            gr = &b.groups.back();
            gr->L = grids[p]->gd.d;
        }
        gr->gs.push_back(grids[p]);
        gr->pos.push_back(p);
        gr->P++;
    }
    int st = solve_batch(b, results);
    if (st != HG_OK && st != HG_ERR_NOT_CONVERGED && st != HG_ERR_BREAKDOWN) cudaStreamSynchronize(b.s);
    return st;
}
