// hg_solve_batch: many problems of one grid shape stepped together.
//
// Every pass of the CG iteration (and of the right-hand side, the projection
// of the correction and the FP64 residual) is one launch for all P problems:
// the pass kernels take the arguments of problem p from a device array
// (grid z = problem), so a batch of small grids fills the GPU in one launch
// where P single solves would each be bound by launch latency.  The CG
// iterations are captured `check_every` at a time in one CUDA graph for the
// whole batch; each problem keeps its own scalars, convergence status and
// reduction slots, and a converged problem's tiles exit at once.  The small
// per-problem steps (scalar set-up, inner set-up, x64 += delta, A_H) are
// plain per-grid launches.
#include "hg.h"
#include "hg_internal.h"
#include "hg_runtime.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
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

int upload_items(Arena& ar, const std::vector<PassArgs>& pas, cudaStream_t s, BatchItems* it) {
    const size_t P = pas.size();
    std::vector<RowFwdArgs> fa(P);
    std::vector<RowInvArgs> ia(P);
    std::vector<StrArgs> sa(P);
    for (size_t p = 0; p < P; ++p) { fa[p] = pas[p].fa; ia[p] = pas[p].ia; }
    int st;
    if ((st = ar.get(P * sizeof(RowFwdArgs), (void**)&it->fa))) return st;
    if ((st = ar.get(P * sizeof(RowInvArgs), (void**)&it->ia))) return st;
    HG_CU(cudaMemcpyAsync(it->fa, fa.data(), P * sizeof(RowFwdArgs), cudaMemcpyHostToDevice, s));
    HG_CU(cudaMemcpyAsync(it->ia, ia.data(), P * sizeof(RowInvArgs), cudaMemcpyHostToDevice, s));
    for (int k = 0; k < pas[0].nstr; ++k) {
        for (size_t p = 0; p < P; ++p) sa[p] = pas[p].sa[k];
        if ((st = ar.get(P * sizeof(StrArgs), (void**)&it->sa[k]))) return st;
        HG_CU(cudaMemcpyAsync(it->sa[k], sa.data(), P * sizeof(StrArgs), cudaMemcpyHostToDevice, s));
    }
    // the host vectors are pageable: cudaMemcpyAsync has staged them on return
    it->first = pas[0];
    return HG_OK;
}

// The launches of one operator application for all P problems.
int launch_batch(hg_grid* g0, int prec, const BatchItems& it, int P, cudaStream_t s) {
    const GridDev& gd = g0->gd;
    const int last = gd.d - 1;
    const int L = it.first.fa.L;
    HG_CU(launch_row_fwd_batch(prec, gd, g0->plan[last], g0->tw[prec], g0->rowcfg[prec], it.fa, P, L, s));
    g0->ctx->launches++;
    for (int k = 0; k < it.first.nstr; ++k) {
        const StrArgs& a = it.first.sa[k];
        HG_CU(launch_strided_batch(prec, gd, g0->plan[a.axis], g0->tw[prec], g0->strcfg[prec][a.axis], it.sa[k],
                                   P, L, a.n, a.inner, a.outer, s));
        g0->ctx->launches++;
    }
    HG_CU(launch_row_inv_batch(prec, gd, g0->plan[last], g0->tw[prec], g0->rowcfg[prec], it.ia, P, L, s));
    g0->ctx->launches++;
    return HG_OK;
}

struct Batch {
    std::vector<hg_grid*> gs;
    hg_solve_opts o{};
    int P = 0, L = 0, prec = 0;
    cudaStream_t s = nullptr;
    Arena ar;
    const Scalars** d_src_outer = nullptr;   // per-problem scalar pointers (device)
    const Scalars** d_src_inner = nullptr;
    Scalars* d_gather = nullptr;
    Scalars* h_gather = nullptr;              // pinned
    cudaGraphExec_t cg_exec = nullptr;
    ~Batch() {
        if (cg_exec) cudaGraphExecDestroy(cg_exec);
        if (h_gather) cudaFreeHost(h_gather);
    }
};

// Copies every problem's scalars (inner or outer) to b.h_gather.
int read_scalars(Batch& b, bool inner) {
    HG_CU(launch_gather_scalars(inner ? b.d_src_inner : b.d_src_outer, b.d_gather, b.P, b.s));
    HG_CU(cudaMemcpyAsync(b.h_gather, b.d_gather, sizeof(Scalars) * MAXL * b.P, cudaMemcpyDeviceToHost, b.s));
    HG_CU(cudaStreamSynchronize(b.s));
    return HG_OK;
}

bool any_status(const Batch& b, int status) {
    for (int p = 0; p < b.P; ++p)
        for (int l = 0; l < b.L; ++l)
            if (b.h_gather[p * MAXL + l].status == status) return true;
    return false;
}

int make_items(Batch& b, BatchItems* it, int prec, const void* const* u, bool unit_loads, bool withA,
               int inv_mode, bool outer_status) {
    std::vector<PassArgs> pas(b.P);
    for (int p = 0; p < b.P; ++p) {
        hg_grid* g = b.gs[p];
        matvec_args(g, prec, b.L, u ? u[p] : nullptr, unit_loads, withA, nullptr, nullptr, inv_mode, nullptr, 1,
                    outer_status ? g->work[0].sc : nullptr, &pas[p]);
    }
    return upload_items(b.ar, pas, b.s, it);
}

// The CUDA graph of check_every batched CG iterations of precision prec.
int make_cg_graph(Batch& b, int prec) {
    std::vector<PassArgs> pas(b.P);
    for (int p = 0; p < b.P; ++p) cg_iteration_args(b.gs[p], prec, b.L, &pas[p]);
    BatchItems it;
    int st;
    if ((st = upload_items(b.ar, pas, b.s, &it))) return st;
    HG_CU(cudaStreamSynchronize(b.s));
    hg_ctx* c = b.gs[0]->ctx;
    cudaStream_t cs = c->cap_stream;
    const long long before = c->launches.load();
    HG_CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < std::max(1, b.o.check_every) && st == HG_OK; ++i) st = launch_batch(b.gs[0], prec, it, b.P, cs);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    c->launches -= c->launches.load() - before;   // capture is not execution
    if (st) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e != cudaSuccess) { set_last_cuda_error(e, "cudaStreamEndCapture"); return HG_ERR_CUDA; }
    if (b.cg_exec) { cudaGraphExecDestroy(b.cg_exec); b.cg_exec = nullptr; }
    e = cudaGraphInstantiate(&b.cg_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { set_last_cuda_error(e, "cudaGraphInstantiate"); b.cg_exec = nullptr; return HG_ERR_CUDA; }
    return HG_OK;
}

// Runs graph chunks until no system of the batch is active (inner scalars for
// the mixed path, outer for FP64) or max_iter + 2 chunks have been launched.
int run_cg(Batch& b, bool inner) {
    const int chunk = std::max(1, b.o.check_every);
    const long long nk = (long long)(b.gs[0]->gd.d + 1);
    for (long long launched = 0;; launched += chunk) {
        HG_CU(cudaGraphLaunch(b.cg_exec, b.s));
        b.gs[0]->ctx->launches += nk * chunk;
        int st = read_scalars(b, inner);
        if (st) return st;
        if (!any_status(b, ST_ACTIVE) || launched + chunk > (long long)b.o.max_iter + 2 * chunk) break;
    }
    return HG_OK;
}

int start_rhs(Batch& b, bool fp32) {
    int init_st[MAXL];
    for (int l = 0; l < MAXL; ++l) init_st[l] = (l < b.L && ((b.o.loads_mask >> l) & 1u)) ? ST_ACTIVE : ST_IDLE;
    for (hg_grid* g : b.gs) {
        HG_CU(launch_init_scalars(g->work[0].sc, b.L, init_st, b.o.tol, b.prec ? b.o.max_outer : b.o.max_iter,
                                  0.0, 1.0, b.s));
        g->ctx->launches++;
    }
    BatchItems it;
    int st;
    if (!fp32) {
        if ((st = make_items(b, &it, 0, nullptr, true, true, INV_RHS, false))) return st;
        if ((st = launch_batch(b.gs[0], 0, it, b.P, b.s))) return st;
        if (b.prec == 0) return HG_OK;
        for (hg_grid* g : b.gs) {
            const GridDev& gd = g->gd;
            HG_CU(launch_inner_init(gd, b.L, (const double*)g->work[0].r, (float*)g->work[1].r, (float*)g->work[1].p,
                                    (float*)g->work[1].x, g->work[0].sc, g->work[1].sc, b.o.inner_tol, b.o.max_iter,
                                    64, grid_weight(g), g->partial, g->counters + 4, b.s));
            g->ctx->launches++;
        }
        return HG_OK;
    }
    for (hg_grid* g : b.gs)
        HG_CU(cudaMemsetAsync(g->work[0].x, 0, sizeof(double) * (size_t)b.L * g->gd.d * g->gd.M, b.s));
    if ((st = make_items(b, &it, 1, nullptr, true, true, INV_RHS, true))) return st;
    if ((st = launch_batch(b.gs[0], 1, it, b.P, b.s))) return st;
    for (hg_grid* g : b.gs) {
        HG_CU(launch_inner_init(g->gd, b.L, nullptr, nullptr, nullptr, nullptr, g->work[0].sc, g->work[1].sc,
                                b.o.inner_tol, b.o.max_iter, 64, grid_weight(g), g->partial, g->counters + 4, b.s));
        g->ctx->launches++;
    }
    return HG_OK;
}

// One problem's right-hand side in FP64 and its inner start from it.
int restart_rhs64(Batch& b, hg_grid* g) {
    int init_st[MAXL];
    for (int l = 0; l < MAXL; ++l) init_st[l] = (l < b.L && ((b.o.loads_mask >> l) & 1u)) ? ST_ACTIVE : ST_IDLE;
    HG_CU(launch_init_scalars(g->work[0].sc, b.L, init_st, b.o.tol, b.o.max_outer, 0.0, 1.0, b.s));
    g->ctx->launches++;
    int st = enqueue_matvec(g, 0, b.L, nullptr, true, true, nullptr, nullptr, INV_RHS, nullptr, 1, b.s);
    if (st) return st;
    HG_CU(launch_inner_init(g->gd, b.L, (const double*)g->work[0].r, (float*)g->work[1].r, (float*)g->work[1].p,
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

int solve_batch(Batch& b, hg_result* results) {
    hg_grid* g0 = b.gs[0];
    hg_ctx* c = g0->ctx;
    const double t0 = wall_ms();
    const long long launches0 = c->launches.load();
    int st;
    for (hg_grid* g : b.gs) {
        if ((st = grid_alloc_common(g))) return st;
        if ((st = grid_alloc_work(g, 0))) return st;
        if (b.prec == 1 && (st = grid_alloc_work(g, 1))) return st;
        g->form = 0;
        g->has_ref = 0;
    }
    // per-problem scalar pointers for the gathers
    std::vector<const Scalars*> outer(b.P), inner(b.P);
    for (int p = 0; p < b.P; ++p) {
        outer[p] = b.gs[p]->work[0].sc;
        inner[p] = b.gs[p]->work[b.prec].sc;
    }
    if ((st = b.ar.get(b.P * sizeof(Scalars*), (void**)&b.d_src_outer))) return st;
    if ((st = b.ar.get(b.P * sizeof(Scalars*), (void**)&b.d_src_inner))) return st;
    if ((st = b.ar.get(b.P * MAXL * sizeof(Scalars), (void**)&b.d_gather))) return st;
    HG_CU(cudaMallocHost((void**)&b.h_gather, b.P * MAXL * sizeof(Scalars)));
    HG_CU(cudaMemcpyAsync(b.d_src_outer, outer.data(), b.P * sizeof(Scalars*), cudaMemcpyHostToDevice, b.s));
    HG_CU(cudaMemcpyAsync(b.d_src_inner, inner.data(), b.P * sizeof(Scalars*), cudaMemcpyHostToDevice, b.s));
    HG_CU(cudaEventRecord(g0->ev0, b.s));

    if ((st = make_cg_graph(b, b.prec))) return st;
    if (b.prec == 0) {
        if ((st = start_rhs(b, false))) return st;
        if ((st = run_cg(b, false))) return st;
    } else {
        if ((st = start_rhs(b, true))) return st;
        // FP32 projection, FP64 projection (tol < 1e-8) and FP64 residual items
        std::vector<const void*> x32(b.P), x64(b.P);
        for (int p = 0; p < b.P; ++p) { x32[p] = b.gs[p]->work[1].x; x64[p] = b.gs[p]->work[0].x; }
        BatchItems proj32, proj64, resid;
        if ((st = make_items(b, &proj32, 1, x32.data(), false, false, INV_PROJ, true))) return st;
        if ((st = make_items(b, &proj64, 0, x64.data(), false, false, INV_PROJ, false))) return st;
        if ((st = make_items(b, &resid, 0, x64.data(), true, true, INV_RESID, false))) return st;
        // a problem whose FP32 right-hand side is too small to decide the zero
        // test starts over with the FP64 one, as its single solve does
        if ((st = read_scalars(b, false))) return st;
        for (int p = 0; p < b.P; ++p) {
            bool recheck = false;
            for (int l = 0; l < b.L; ++l) recheck |= b.h_gather[p * MAXL + l].status == ST_RHS_RECHECK;
            if (recheck && (st = restart_rhs64(b, b.gs[p]))) return st;
        }
        for (int outer_it = 0;;) {
            if ((st = run_cg(b, true))) return st;
            if ((st = launch_batch(g0, 1, proj32, b.P, b.s))) return st;
            for (hg_grid* g : b.gs) {
                HG_CU(launch_outer_update(g->gd, b.L, (double*)g->work[0].x, (const float*)g->work[1].x,
                                          g->work[0].sc, g->work[1].sc, b.s));
                c->launches++;
            }
            if (b.o.tol < 1e-8 && (st = launch_batch(g0, 0, proj64, b.P, b.s))) return st;
            if ((st = launch_batch(g0, 0, resid, b.P, b.s))) return st;
            if ((st = read_scalars(b, false))) return st;
            ++outer_it;
            if (!any_status(b, ST_ACTIVE) || outer_it >= std::max(1, b.o.max_outer)) break;
            for (hg_grid* g : b.gs) {
                HG_CU(launch_inner_init(g->gd, b.L, (const double*)g->work[0].r, (float*)g->work[1].r,
                                        (float*)g->work[1].p, (float*)g->work[1].x, g->work[0].sc, g->work[1].sc,
                                        b.o.inner_tol, b.o.max_iter, 64, grid_weight(g), g->partial,
                                        g->counters + 4, b.s));
                c->launches++;
            }
        }
    }
    // A_H per problem, then every problem's outer scalars
    for (hg_grid* g : b.gs) {
        const GridDev& gd = g->gd;
        HG_CU(launch_energy(gd, b.L, coeffs_for(g, 0, true), (const double*)g->work[0].x, b.o.loads_mask,
                            g->partial, g->counters + 5, g->d_AH, b.s));
        c->launches++;
        HG_CU(cudaMemcpyAsync(g->h_AH, g->d_AH, sizeof(double) * 2 * gd.d * gd.d, cudaMemcpyDeviceToHost, b.s));
    }
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
        for (int l = 0; l < b.L; ++l) {
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

}  // namespace

extern "C" int hg_solve_batch(hg_grid* const* grids, int n, const hg_solve_opts* opts, hg_result* results) {
    if (!grids || n < 1 || !results) return HG_ERR_ARG;
    hg_grid* g0 = grids[0];
    if (!g0) return HG_ERR_ARG;
    hg_solve_opts o;
    if (opts) o = *opts; else hg_default_opts(&o);
    int st = validate_solve_opts(g0, &o);
    if (st) return st;
    if (o.method != HG_CG || o.formulation != HG_PRIMAL || o.A0[0] != 0.0 || o.time_pass != -1) return HG_ERR_ARG;
    hg_ctx* c = g0->ctx;
    for (int p = 0; p < n; ++p) {
        const hg_grid* g = grids[p];
        if (!g || g->ctx != c || g->gd.d != g0->gd.d) return HG_ERR_ARG;
        for (int a = 0; a < 3; ++a)
            if (g->gd.N[a] != g0->gd.N[a] || g->gd.Y[a] != g0->gd.Y[a]) return HG_ERR_ARG;
        if (g->coeff_mode < 0) return HG_ERR_NO_COEFFS;
        if (g->borrowed.load() > 0) return HG_ERR_BUSY;
        for (int q = 0; q < p; ++q)
            if (grids[q] == g) return HG_ERR_ARG;   // each problem needs its own buffers
    }
    cudaSetDevice(c->device);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    Batch b;
    b.gs.assign(grids, grids + n);
    b.o = o;
    b.P = n;
    b.L = g0->gd.d;
    b.prec = o.prec == HG_MIXED ? 1 : 0;
    b.s = c->stream;
    b.ar.ctx = c;
    st = solve_batch(b, results);
    if (st != HG_OK && st != HG_ERR_NOT_CONVERGED && st != HG_ERR_BREAKDOWN) cudaStreamSynchronize(b.s);
    return st;
}
