// Host runtime of libhg: contexts, grids, FFT plans, device buffers, the
// CUDA-graph-captured CG loop, mixed-precision refinement and the request
// scheduler behind hg_submit / hg_poll.  See include/hg.h for the contract.
#include "hg.h"
#include "hg_internal.h"
#include "hg_runtime.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

using namespace hgk;

namespace hgrt {

// ----------------------------------------------------------------------------
// helpers
// ----------------------------------------------------------------------------
static double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

#define HG_CU(call)                                  \
    do {                                             \
        cudaError_t _e = (call);                     \
        if (_e != cudaSuccess) {                     \
            set_last_cuda_error(_e, #call);          \
            return HG_ERR_CUDA;                      \
        }                                            \
    } while (0)

static thread_local char g_last_err[256];
void set_last_cuda_error(cudaError_t e, const char* what) {
    snprintf(g_last_err, sizeof(g_last_err), "%s: %s", what, cudaGetErrorString(e));
}
const char* last_cuda_error() { return g_last_err; }

int dev_alloc(hg_ctx* ctx, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (ctx->budget) {
        size_t cur = ctx->used.load();
        if (cur + bytes > ctx->budget) return HG_ERR_NO_MEMORY;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return HG_ERR_NO_MEMORY;
    }
    ctx->used += bytes;
    ctx->alloc_sizes[*p] = bytes;
    return HG_OK;
}

void dev_free(hg_ctx* ctx, void* p) {
    if (!p) return;
    auto it = ctx->alloc_sizes.find(p);
    if (it != ctx->alloc_sizes.end()) {
        ctx->used -= it->second;
        ctx->alloc_sizes.erase(it);
    }
    cudaFree(p);
}

// Factor n into radices 3, 5, 7 (application order: 3s, then 5s, then 7s).
bool factor(int n, AxisPlanH& pl) {
    pl.n = n;
    pl.nstages = 0;
    int m = n;
    for (int r : {3, 5, 7}) {
        while (m % r == 0) {
            if (pl.nstages >= 16) return false;
            pl.radix[pl.nstages++] = r;
            m /= r;
        }
    }
    return m == 1;
}

int min_radix(const AxisPlanH& pl) {
    int r = 7;
    for (int s = 0; s < pl.nstages; ++s) r = std::min(r, pl.radix[s]);
    return pl.nstages ? r : 1;
}

// Row pass geometry with RB grid rows and LB loads per CTA, if the kernels
// can run it: the compile-time kernels stage at most ct_npmax complex pencils
// of 256 threads, the runtime kernels at most MAXB butterflies per thread of
// at most row_max_threads() threads in max_smem bytes; both keep the offsets
// of at most MAX_REAL_ROWS_HOST real rows.
bool make_row_cfg(int prec, int n, int d, int L, int RB, int LB, int minR, size_t csize, int max_smem,
                  long long rows, RowCfg& cfg) {
    const int maxb = 2, maxt = row_max_threads();
    if (RB < 1 || LB < 1 || LB > L || RB > rows) return false;
    const int nreal = RB * LB * d;
    const int ncplx = (nreal + 1) / 2;
    if (nreal > MAX_REAL_ROWS_HOST) return false;
    if (ct_length(d, n)) {
        if (ncplx > ct_npmax(prec, n)) return false;
        cfg.threads = CT_THREADS_HOST;
        cfg.smem = (int)((size_t)(ncplx + 1) * n * csize);
        cfg.ct = 1;
    } else {
        const long long bfly = std::max<long long>((long long)ncplx * n / std::max(minR, 1), 1);
        const size_t smem = (size_t)ncplx * n * csize;
        if (bfly > (long long)maxb * maxt || smem > (size_t)max_smem) return false;
        int thr = (int)((bfly + maxb - 1) / maxb);
        cfg.threads = std::max(64, std::min(maxt, ((thr + 31) / 32) * 32));
        cfg.smem = (int)smem;
        cfg.ct = 0;
    }
    cfg.RB = RB;
    cfg.LB = LB;
    cfg.nbx = (rows + RB - 1) / RB;
    cfg.nby = (L + LB - 1) / LB;
    return true;
}

// Row pass: choose loads-per-CTA LB and rows-per-CTA RB.  The most loads per
// CTA first, then the most rows that keep at least two CTAs per SM (and, for
// the runtime kernels, at most 32 KB of pencils).
bool choose_row_cfg(int prec, int n, int d, int L, int minR, size_t csize, int max_smem,
                    long long rows, RowCfg& cfg) {
    const size_t target = 32 * 1024;
    for (int LB = L; LB >= 1; --LB) {
        RowCfg best{};
        bool found = false;
        for (int RB = 1; RB <= 64; ++RB) {
            RowCfg c{};
            if (!make_row_cfg(prec, n, d, L, RB, LB, minR, csize, max_smem, rows, c)) break;
            if (RB > 1 && (rows / RB < 2 * 152 || (!c.ct && (size_t)c.smem > target))) break;
            best = c;
            found = true;
        }
        if (found) {
            cfg = best;
            return true;
        }
    }
    return false;
}

// Strided pass geometry with Cl lanes (pencils per component, a power of two)
// per CTA, if the kernels can run it.
bool make_str_cfg(int prec, int n, int d, int Cl, int minR, size_t csize, int max_smem, long long inner,
                  StrCfg& cfg) {
    const int maxb = 2, maxt = row_max_threads();
    if (Cl < 1 || (Cl & (Cl - 1)) || (Cl > 1 && Cl > inner)) return false;
    if (ct_length(d, n)) {
        if (d * Cl > ct_npmax(prec, n) || Cl > ct_max_lanes(d)) return false;
        cfg.threads = CT_THREADS_HOST;
        cfg.smem = (int)((size_t)(d * Cl + 1) * n * csize);
        cfg.ct = 1;
    } else {
        if (Cl > 32) return false;
        const long long bfly = std::max<long long>((long long)d * Cl * n / std::max(minR, 1), 1);
        const size_t smem = (size_t)d * Cl * n * csize;
        if (bfly > (long long)maxb * maxt || smem > (size_t)max_smem) return false;
        int thr = (int)((bfly + maxb - 1) / maxb);
        cfg.threads = std::max(64, std::min(maxt, ((thr + 31) / 32) * 32));
        cfg.smem = (int)smem;
        cfg.ct = 0;
    }
    cfg.Cl = Cl;
    return true;
}

bool choose_str_cfg(int prec, int n, int d, int minR, size_t csize, int max_smem,
                    long long inner, long long outer, int L, StrCfg& cfg) {
    const int prefer_lanes = 2;   // more, smaller CTAs beat full 32-byte rows here
    const bool ct = ct_length(d, n);
    int best = 0;
    for (int Cl = 1; Cl <= 32; Cl *= 2) {
        StrCfg c{};
        if (!make_str_cfg(prec, n, d, Cl, minR, csize, max_smem, inner, c)) break;
        if (Cl > prefer_lanes && (!ct || ((inner + Cl - 1) / Cl) * outer * L < 4 * 152)) break;
        if (Cl > 2 * prefer_lanes) break;
        best = Cl;
        cfg = c;
    }
    return best > 0;
}

// ----------------------------------------------------------------------------
// grid construction
// ----------------------------------------------------------------------------
int grid_init_plans(hg_grid* g) {
    GridDev& gd = g->gd;
    const int d = gd.d;
    // twiddles, one table per distinct length
    std::map<int, int> off;
    std::vector<double> tw64;
    for (int a = 0; a < d; ++a) {
        const int n = gd.N[a];
        if (!factor(n, g->plan[a])) return HG_ERR_UNSUPPORTED_SIZE;
        if (!off.count(n)) {
            off[n] = (int)(tw64.size() / 2);
            for (int m = 0; m < n; ++m) {
                // W_n^m = exp(-2 pi i m / n), evaluated in extended precision
                const long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)m / (long double)n;
                tw64.push_back((double)cosl(ang));
                tw64.push_back((double)sinl(ang));
            }
        }
        g->plan[a].tw_off = off[n];
    }
    std::vector<float> tw32(tw64.size());
    for (size_t i = 0; i < tw64.size(); ++i) tw32[i] = (float)tw64[i];
    int st = dev_alloc(g->ctx, &g->tw[0], tw64.size() * sizeof(double));
    if (st) return st;
    st = dev_alloc(g->ctx, &g->tw[1], tw32.size() * sizeof(float));
    if (st) return st;
    HG_CU(cudaMemcpyAsync(g->tw[0], tw64.data(), tw64.size() * sizeof(double), cudaMemcpyHostToDevice, g->ctx->stream));
    HG_CU(cudaMemcpyAsync(g->tw[1], tw32.data(), tw32.size() * sizeof(float), cudaMemcpyHostToDevice, g->ctx->stream));
    HG_CU(cudaStreamSynchronize(g->ctx->stream));

    // launch geometry per precision
    const int max_smem = g->ctx->max_smem;
    for (int prec = 0; prec < 2; ++prec) {
        const size_t cs = prec == 0 ? 16 : 8;
        const int last = d - 1;
        if (!choose_row_cfg(prec, gd.Nl, d, d, min_radix(g->plan[last]), cs, max_smem, gd.rows, g->rowcfg[prec]))
            return HG_ERR_UNSUPPORTED_SIZE;
        for (int a = 0; a < last; ++a) {
            // axis 0: lanes run over all other axes; axis 1 (3D): over the last
            const long long inner = (a == 0) ? gd.Ms / gd.N[0] : gd.H;
            const long long outer = (a == 0) ? 1 : gd.N[0];
            if (!choose_str_cfg(prec, gd.N[a], d, min_radix(g->plan[a]), cs, max_smem, inner, outer, d,
                                g->strcfg[prec][a]))
                return HG_ERR_UNSUPPORTED_SIZE;
        }
    }
    return HG_OK;
}

int grid_alloc_work(hg_grid* g, int prec) {
    if (g->work[prec].ready) return HG_OK;
    const GridDev& gd = g->gd;
    const int L = gd.d;
    const size_t ts = prec == 0 ? 8 : 4;
    const size_t nv = (size_t)L * gd.d * gd.M;
    // the FP32 half spectra leave room for rows padded to an even length (the
    // resident solver's layout, 16-byte aligned rows for bulk copies)
    const size_t ns = (size_t)L * gd.d * (prec == 1 ? gd.rows * ((gd.H + 1) & ~1) : gd.Ms);
    Work& w = g->work[prec];
    int st;
    if ((st = dev_alloc(g->ctx, &w.x, nv * ts))) return st;
    if ((st = dev_alloc(g->ctx, &w.r, nv * ts))) return st;
    if ((st = dev_alloc(g->ctx, &w.p, nv * ts))) return st;
    if ((st = dev_alloc(g->ctx, &w.S, ns * 2 * ts))) return st;
    if ((st = dev_alloc(g->ctx, (void**)&w.sc, sizeof(Scalars) * MAXL))) return st;
    HG_CU(cudaMemsetAsync(w.sc, 0, sizeof(Scalars) * MAXL, g->ctx->stream));
    HG_CU(cudaMemsetAsync(w.x, 0, nv * ts, g->ctx->stream));
    HG_CU(cudaMemsetAsync(w.p, 0, nv * ts, g->ctx->stream));
    w.ready = true;
    return HG_OK;
}

// Releases the solver state (work buffers, graphs that point at them and the
// reduction scratch); the plans, twiddles and coefficients stay.
void grid_free_work(hg_grid* g) {
    hg_ctx* c = g->ctx;
    for (int p = 0; p < 2; ++p) {
        if (g->graphs[p].exec) cudaGraphExecDestroy(g->graphs[p].exec);
        g->graphs[p] = GraphCache();
        Work& w = g->work[p];
        dev_free(c, w.x); dev_free(c, w.r); dev_free(c, w.p); dev_free(c, w.S); dev_free(c, w.sc);
        w = Work();
    }
    dev_free(c, g->partial); g->partial = nullptr;
    dev_free(c, g->counters); g->counters = nullptr;
    dev_free(c, g->d_AH); g->d_AH = nullptr;
    dev_free(c, g->d_E); g->d_E = nullptr;
    dev_free(c, g->d_A0); g->d_A0 = nullptr;
    dev_free(c, g->d_sc_aux); g->d_sc_aux = nullptr;
}

size_t ctx_reclaim(hg_ctx* ctx, hg_grid* keep) {
    const size_t before = ctx->used.load();
    for (hg_grid* g : ctx->grids) {
        if (g == keep || g->borrowed.load() > 0) continue;
        if (g->work[0].ready || g->work[1].ready) grid_free_work(g);
    }
    return before - ctx->used.load();
}

// Device bytes a solve of precision prec (1: mixed, FP32 buffers as well)
// still has to allocate on g, row-pass reduction slots for nbx CTAs included:
// admission compares it with the budget before allocating anything.
size_t solve_bytes_needed(const hg_grid* g, int prec, long long nbx) {
    const GridDev& gd = g->gd;
    const int L = gd.d;
    size_t need = 0;
    auto work = [&](int pr) {
        const size_t ts = pr == 0 ? 8 : 4;
        const size_t nv = (size_t)L * gd.d * gd.M;
        const size_t ns = (size_t)L * gd.d * (pr == 1 ? gd.rows * ((gd.H + 1) & ~1) : gd.Ms);
        return 3 * nv * ts + ns * 2 * ts + sizeof(Scalars) * MAXL;
    };
    if (!g->work[0].ready) need += work(0);
    if (prec == 1 && !g->work[1].ready) need += work(1);
    long long slots = std::max<long long>(std::max(g->rowcfg[0].nbx, g->rowcfg[1].nbx) * MAXL, 18LL * 8 * 1024);
    slots = std::max<long long>(slots, nbx * MAXL);
    if (!g->partial) {
        need += (size_t)slots * sizeof(double) + 16 * sizeof(unsigned) + 32 * sizeof(double) +
                (MAXL * MAXD + 16) * sizeof(double) + sizeof(Scalars) * MAXL;
    } else if (slots > g->partial_slots) {
        need += (size_t)slots * sizeof(double);
    }
    return need;
}

int grid_alloc_common(hg_grid* g) {
    if (g->partial) return HG_OK;
    const GridDev& gd = g->gd;
    long long slots = std::max<long long>(g->rowcfg[0].nbx, g->rowcfg[1].nbx) * MAXL;
    slots = std::max<long long>(slots, 18LL * 8 * 1024);
    int st;
    if ((st = dev_alloc(g->ctx, (void**)&g->partial, slots * sizeof(double)))) return st;
    g->partial_slots = slots;
    if ((st = dev_alloc(g->ctx, (void**)&g->counters, 16 * sizeof(unsigned)))) return st;
    HG_CU(cudaMemsetAsync(g->counters, 0, 16 * sizeof(unsigned), g->ctx->stream));
    if ((st = dev_alloc(g->ctx, (void**)&g->d_AH, 32 * sizeof(double)))) return st;
    if ((st = dev_alloc(g->ctx, (void**)&g->d_E, MAXL * MAXD * sizeof(double)))) return st;
    double E[MAXL * MAXD] = {0};
    for (int l = 0; l < gd.d; ++l) E[l * gd.d + l] = 1.0;
    HG_CU(cudaMemcpyAsync(g->d_E, E, sizeof(E), cudaMemcpyHostToDevice, g->ctx->stream));
    if ((st = dev_alloc(g->ctx, (void**)&g->d_A0, 16 * sizeof(double)))) return st;
    if ((st = dev_alloc(g->ctx, (void**)&g->d_sc_aux, sizeof(Scalars) * MAXL))) return st;
    HG_CU(cudaStreamSynchronize(g->ctx->stream));
    (void)gd;
    return HG_OK;
}

int grid_ensure_partial(hg_grid* g, long long nbx) {
    int st;
    if ((st = grid_alloc_common(g))) return st;
    const long long need = nbx * MAXL;
    if (need <= g->partial_slots) return HG_OK;
    double* fresh = nullptr;
    if ((st = dev_alloc(g->ctx, (void**)&fresh, (size_t)need * sizeof(double)))) return st;
    HG_CU(cudaStreamSynchronize(g->ctx->stream));
    dev_free(g->ctx, g->partial);
    g->partial = fresh;
    g->partial_slots = need;
    // cached CG graphs hold the old pointer
    for (int p = 0; p < 2; ++p) {
        if (g->graphs[p].exec) cudaGraphExecDestroy(g->graphs[p].exec);
        g->graphs[p] = GraphCache();
    }
    return HG_OK;
}

Weight grid_weight(const hg_grid* g) {
    Weight w;
    memset(&w, 0, sizeof(w));
    w.has = g->has_ref;
    for (int i = 0; i < 9; ++i) { w.w[i] = g->ref[i]; w.wf[i] = (float)g->ref[i]; }
    return w;
}

CoeffsDev coeffs_for(const hg_grid* g, int prec, bool withA) {
    CoeffsDev c;
    c.phase = g->d_phase;
    c.table = g->form ? g->d_table_inv[prec] : g->d_table[prec];
    c.field = g->form ? g->d_field_inv[prec] : g->d_field[prec];
    c.mode = !withA ? 2 : (g->coeff_mode == 0 ? 0 : 1);
    c.n_phases = g->n_phases;
    return c;
}

// ----------------------------------------------------------------------------
// pass enqueueing (every CG iteration / operator application)
// ----------------------------------------------------------------------------
int enqueue_forward_strided(hg_grid* g, int prec, int L, int check_status, int gamma_mode,
                            const double* A0, cudaStream_t s, Scalars* status_sc) {
    // 3D: axis 1 forward, axis 0 (fwd + Gamma + inv | fwd+scale), axis 1 inverse
    const GridDev& gd = g->gd;
    Work& w = g->work[prec];
    const int d = gd.d;
    StrArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.early_stage = 1;
    sa.L = L;
    sa.S = w.S;
    sa.sc = status_sc ? status_sc : w.sc;
    sa.check_status = check_status;
    sa.dual = g->form;
    if (A0) {
        sa.has_A0 = 1;
        for (int i = 0; i < d * d; ++i) sa.A0[i] = A0[i];
    }
    if (d == 3) {
        sa.mode = STR_FWD; sa.axis = 1; sa.outer = gd.N[0]; sa.n = gd.N[1]; sa.inner = gd.H;
        HG_CU(launch_strided(prec, gd, g->plan[1], g->tw[prec], g->strcfg[prec][1], sa, s));
        g->ctx->launches++;
    }
    sa.mode = gamma_mode; sa.axis = 0; sa.outer = 1; sa.n = gd.N[0]; sa.inner = gd.Ms / gd.N[0];
    HG_CU(launch_strided(prec, gd, g->plan[0], g->tw[prec], g->strcfg[prec][0], sa, s));
    g->ctx->launches++;
    if (d == 3 && gamma_mode == STR_GAMMA) {
        sa.mode = STR_INV; sa.axis = 1; sa.outer = gd.N[0]; sa.n = gd.N[1]; sa.inner = gd.H;
        HG_CU(launch_strided(prec, gd, g->plan[1], g->tw[prec], g->strcfg[prec][1], sa, s));
        g->ctx->launches++;
    }
    return HG_OK;
}

// Strided passes of an operator application in launch order (3D: axis 1
// forward, axis 0, axis 1 inverse; 2D: axis 0), from a template carrying the
// common fields.
static void strided_sequence(const hg_grid* g, StrArgs base, int gamma_mode, PassArgs* pa) {
    const GridDev& gd = g->gd;
    pa->nstr = 0;
    if (gd.d == 3) {
        StrArgs a = base;
        a.mode = STR_FWD; a.axis = 1; a.outer = gd.N[0]; a.n = gd.N[1]; a.inner = gd.H;
        pa->sa[pa->nstr++] = a;
    }
    StrArgs a = base;
    a.mode = gamma_mode; a.axis = 0; a.outer = 1; a.n = gd.N[0]; a.inner = gd.Ms / gd.N[0];
    pa->sa[pa->nstr++] = a;
    if (gd.d == 3 && gamma_mode == STR_GAMMA) {
        StrArgs b = base;
        b.mode = STR_INV; b.axis = 1; b.outer = gd.N[0]; b.n = gd.N[1]; b.inner = gd.H;
        pa->sa[pa->nstr++] = b;
    }
}

// Whether g's FP32 CG iterations run as the plane passes: N0 x N x N grids of
// the compiled plane lengths, the plain scalar product (A0 = I), and
// reduction slots for one CTA per (plane, component).
bool plane_path(const hg_grid* g, int prec) {
    return prec == 1 && g->use_plane && !g->has_ref && plane_supported(g->gd) &&
           plane_units(g->gd) * MAXL <= g->partial_slots;
}

void cg_iteration_args(hg_grid* g, int prec, int L, PassArgs* pa) {
    const GridDev& gd = g->gd;
    Work& w = g->work[prec];
    const int d = gd.d;
    RowFwdArgs& fa = pa->fa;
    memset(&fa, 0, sizeof(fa));
    fa.early_stage = 1;
    fa.mode = FWD_CG; fa.L = L; fa.co = coeffs_for(g, prec, true);
    fa.p = w.p; fa.r = w.r; fa.S = w.S; fa.sc = w.sc;
    fa.partial = g->partial; fa.counter = g->counters + 0; fa.check_status = 1;
    StrArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.early_stage = 1;
    sa.L = L; sa.S = w.S; sa.sc = w.sc; sa.check_status = 1; sa.dual = g->form;
    for (int a = 0; a < 3; ++a) sa.band[a] = g->band[a];
    if (g->has_ref) {   // Gamma_hat of the reference medium (its denominator xi . A0 xi)
        sa.has_A0 = 1;
        for (int i = 0; i < d * d; ++i) sa.A0[i] = g->ref[i];
    }
    pa->plane = plane_path(g, prec) ? 1 : 0;
    if (pa->plane) {
        // axis 0 only: the plane passes take axes 1 and 2
        StrArgs a = sa;
        a.mode = STR_GAMMA; a.axis = 0; a.outer = 1; a.n = gd.N[0]; a.inner = gd.Ms / gd.N[0];
        pa->sa[0] = a;
        pa->nstr = 1;
    } else {
        strided_sequence(g, sa, STR_GAMMA, pa);
    }
    RowInvArgs& ia = pa->ia;
    memset(&ia, 0, sizeof(ia));
    ia.early_stage = 1;
    ia.mode = INV_CG; ia.L = L; ia.S = w.S; ia.x = w.x; ia.r = w.r; ia.p = w.p;
    ia.W = grid_weight(g);
    ia.sc = w.sc; ia.partial = g->partial; ia.counter = g->counters + 1; ia.check_status = 1;
}

void matvec_args(hg_grid* g, int prec, int L, const void* u, bool unit_loads, bool withA,
                 const double* A0dev, const double* A0host, int inv_mode, void* out, int check_status,
                 Scalars* status_sc, PassArgs* pa) {
    const GridDev& gd = g->gd;
    const int d = gd.d;
    // the right-hand side and the residual of the iteration use its reference
    // medium; projections (INV_PROJ) stay orthogonal
    const bool iter_op = inv_mode == INV_RHS || inv_mode == INV_RESID;
    if (iter_op && g->has_ref && !A0host) A0host = g->ref;
    Work& w = g->work[prec];
    Scalars* sc = status_sc ? status_sc : w.sc;
    RowFwdArgs& fa = pa->fa;
    memset(&fa, 0, sizeof(fa));
    fa.early_stage = 1;
    fa.mode = FWD_APPLY; fa.L = L; fa.co = coeffs_for(g, prec, withA);
    fa.u = u; fa.A0 = A0dev; fa.S = w.S; fa.sc = sc;
    if (unit_loads) {          // E_l = e_l (Eq. grad_field_split with E = e_j)
        fa.has_E = 1;
        for (int l = 0; l < L; ++l) { fa.Ed[l * gd.d + l] = 1.0; fa.Ef[l * gd.d + l] = 1.0f; }
    }
    fa.partial = g->partial; fa.counter = g->counters + 2; fa.check_status = check_status;
    StrArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.early_stage = 1;
    sa.L = L; sa.S = w.S; sa.sc = sc; sa.check_status = check_status; sa.dual = g->form;
    for (int a = 0; a < 3; ++a) sa.band[a] = g->band[a];
    if (A0host) {
        sa.has_A0 = 1;
        for (int i = 0; i < d * d; ++i) sa.A0[i] = A0host[i];
    }
    strided_sequence(g, sa, STR_GAMMA, pa);
    RowInvArgs& ia = pa->ia;
    memset(&ia, 0, sizeof(ia));
    ia.early_stage = 1;
    ia.mode = inv_mode; ia.L = L; ia.S = w.S; ia.x = w.x; ia.r = w.r; ia.p = w.p; ia.out = out;
    if (iter_op) ia.W = grid_weight(g);
    ia.sc = sc; ia.partial = g->partial; ia.counter = g->counters + 3; ia.check_status = check_status;
}

// The launches of pa on g; mark(before, pass) brackets pass `pass`
// (0 row_fwd, 1..nstr strided, nstr + 1 row_inv) with event records.
template <typename Mark>
static int launch_passes(hg_grid* g, int prec, const PassArgs& pa, cudaStream_t s, Mark mark) {
    const GridDev& gd = g->gd;
    const int last = gd.d - 1;
    int pass = 0;
    if (pa.plane) {
        const float2* tw = static_cast<const float2*>(g->tw[1]) + g->plan[last].tw_off;
        HG_CU(mark(true, pass));
        HG_CU(launch_plane_fwd(gd, tw, pa.fa, s));
        HG_CU(mark(false, pass));
        ++pass;
        HG_CU(mark(true, pass));
        HG_CU(launch_strided(prec, gd, g->plan[0], g->tw[prec], g->strcfg[prec][0], pa.sa[0], s));
        HG_CU(mark(false, pass));
        ++pass;
        HG_CU(mark(true, pass));
        HG_CU(launch_plane_inv(gd, tw, pa.ia, s));
        HG_CU(mark(false, pass));
        g->ctx->launches += 3;
        return HG_OK;
    }
    HG_CU(mark(true, pass));
    HG_CU(launch_row_fwd(prec, gd, g->plan[last], g->tw[prec], g->rowcfg[prec], pa.fa, s));
    HG_CU(mark(false, pass));
    g->ctx->launches++;
    ++pass;
    for (int k = 0; k < pa.nstr; ++k) {
        const int ax = pa.sa[k].axis;
        HG_CU(mark(true, pass));
        HG_CU(launch_strided(prec, gd, g->plan[ax], g->tw[prec], g->strcfg[prec][ax], pa.sa[k], s));
        HG_CU(mark(false, pass));
        g->ctx->launches++;
        ++pass;
    }
    HG_CU(mark(true, pass));
    HG_CU(launch_row_inv(prec, gd, g->plan[last], g->tw[prec], g->rowcfg[prec], pa.ia, s));
    HG_CU(mark(false, pass));
    g->ctx->launches++;
    return HG_OK;
}

// One CG iteration (d + 1 launches).  prof_pass >= 0: event records bracket
// that pass (0 row_fwd, 1..d-1 strided in launch order, d row_inv); inside
// stream capture only an external event record becomes a real event record
// node (a plain record just orders the graph).
int enqueue_cg_iteration(hg_grid* g, int prec, int L, cudaStream_t s, int prof_pass,
                         cudaEvent_t ev_before, cudaEvent_t ev_after) {
    PassArgs pa;
    cg_iteration_args(g, prec, L, &pa);
    return launch_passes(g, prec, pa, s, [&](bool before, int pass) -> cudaError_t {
        if (prof_pass != pass) return cudaSuccess;
        return cudaEventRecordWithFlags(before ? ev_before : ev_after, s, cudaEventRecordExternal);
    });
}

// q = G A (E + u) followed by the epilogue `inv_mode` (INV_RHS / INV_RESID /
// INV_OUT / INV_PROJ); u may be null.
int enqueue_matvec(hg_grid* g, int prec, int L, const void* u, bool unit_loads, bool withA,
                   const double* A0dev, const double* A0host, int inv_mode, void* out,
                   int check_status, cudaStream_t s, Scalars* status_sc) {
    PassArgs pa;
    matvec_args(g, prec, L, u, unit_loads, withA, A0dev, A0host, inv_mode, out, check_status, status_sc, &pa);
    return launch_passes(g, prec, pa, s, [](bool, int) { return cudaSuccess; });
}

// A CUDA graph of `chunk` CG iterations, cached per precision.
int get_cg_graph(hg_grid* g, int prec, int chunk, cudaGraphExec_t* out, int* nkern, int prof_pass) {
    GraphCache& gc = g->graphs[prec];
    const int plane = plane_path(g, prec) ? 1 : 0;
    if (gc.exec && gc.chunk == chunk && gc.prof_pass == prof_pass && gc.form == g->form && gc.plane == plane &&
        gc.has_ref == g->has_ref && (!g->has_ref || memcmp(gc.ref, g->ref, sizeof(gc.ref)) == 0)) {
        *out = gc.exec;
        *nkern = gc.nkern;
        return HG_OK;
    }
    if (gc.exec) {
        cudaGraphExecDestroy(gc.exec);
        gc.exec = nullptr;
    }
    cudaStream_t s = g->ctx->cap_stream;
    const long long before = g->ctx->launches.load();
    int st = HG_OK;
    HG_CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    // time_pass: the pass is bracketed in the first iteration of the chunk only,
    // so that the event nodes (which break the programmatic launch overlap
    // around it) perturb one iteration in `chunk`
    if (prof_pass >= 0) {
        for (int i = 0; i < 2; ++i)
            if (!g->prof_ev[i] && cudaEventCreate(&g->prof_ev[i]) != cudaSuccess) st = HG_ERR_CUDA;
    }
    for (int i = 0; i < chunk && st == HG_OK; ++i)
        st = (prof_pass >= 0 && i == 0)
                 ? enqueue_cg_iteration(g, prec, g->gd.d, s, prof_pass, g->prof_ev[0], g->prof_ev[1])
                 : enqueue_cg_iteration(g, prec, g->gd.d, s);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    const long long nk = g->ctx->launches.load() - before;
    g->ctx->launches -= nk;   // capture is not execution
    if (st) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e != cudaSuccess) { set_last_cuda_error(e, "cudaStreamEndCapture"); return HG_ERR_CUDA; }
    e = cudaGraphInstantiate(&gc.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { set_last_cuda_error(e, "cudaGraphInstantiate"); gc.exec = nullptr; return HG_ERR_CUDA; }
    gc.chunk = chunk;
    gc.prof_pass = prof_pass;
    gc.form = g->form;
    gc.plane = plane;
    gc.has_ref = g->has_ref;
    memcpy(gc.ref, g->ref, sizeof(gc.ref));
    gc.nkern = (int)nk;
    *out = gc.exec;
    *nkern = gc.nkern;
    return HG_OK;
}

static int map_status(int s) {
    switch (s) {
        case ST_CONVERGED: case ST_ZERO_RHS: case ST_IDLE: case ST_STAGNATED: return HG_OK;
        case ST_MAXITER: case ST_ACTIVE: return HG_ERR_NOT_CONVERGED;
        case ST_BREAKDOWN: return HG_ERR_BREAKDOWN;
        case ST_TIMEOUT: return HG_ERR_DEVICE_TIMEOUT;
        default: return HG_ERR_CUDA;
    }
}

// ----------------------------------------------------------------------------
// resumable solve (shared by the blocking call and the request scheduler)
// ----------------------------------------------------------------------------
// Enqueue one graph chunk of CG iterations of precision `prec`, then the copy
// of that precision's scalars to pinned host memory and the tick event.
// time_pass: add the duration of the timed pass in the first iteration of the
// chunk that just completed, if a system was active in it.
static void job_collect_pass_times(Job& j) {
    if (j.o.time_pass < 0) return;
    const Scalars* h = j.g->h_sc;
    int it = 0;
    for (int l = 0; l < j.g->gd.d; ++l) it = std::max(it, h[l].iters);
    if (it > j.prof_prev_iters) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, j.g->prof_ev[0], j.g->prof_ev[1]) == cudaSuccess) {
            j.prof_ms += ms;
            j.prof_n += 1;
        } else {
            cudaGetLastError();   // a timing failure must not reach later status checks
        }
    }
    j.prof_prev_iters = it;
}

// The resident FP32 solver (one cooperative launch for a whole inner solve,
// r and p kept on chip; hg_resident.cu) when the job allows it and the grid's
// state fits: square 2D grids of the resident lengths.  Returns 1 if it
// launched, 0 if the pass kernels are to be used, < 0 on error.
static int job_launch_resident(Job& j) {
    hg_grid* g = j.g;
    const GridDev& gd = g->gd;
    if (!j.allow_resident || j.o.resident == 0 || gd.d != 2 || gd.N[0] != gd.N[1] ||
        g->coeff_mode < 0 || !resident_length(gd.N[0]))
        return 0;
    ResCfg cfg;
    if (!resident_cfg(gd.N[0], gd.d, j.o.resident > 0 ? j.o.resident : 0, g->ctx->nsm, g->ctx->max_smem, cfg))
        return 0;
    // barrier targets count 3 per iteration and CTA in 32 bits
    if ((long long)j.o.max_iter * 3 * cfg.T >= (1LL << 31)) return 0;
    if ((long long)2 * cfg.T * MAXL > g->partial_slots) return 0;
    ResArgs a;
    memset(&a, 0, sizeof(a));
    a.g = gd;
    a.co = coeffs_for(g, 1, true);
    a.L = gd.d;
    a.units = gd.N[0] * gd.d;
    a.cunits = gd.H * gd.d;
    a.umax = cfg.umax;
    a.bufp = cfg.bufp;
    a.r0 = static_cast<const float*>(g->work[1].r);
    a.x = static_cast<float*>(g->work[1].x);
    a.S = static_cast<float2*>(g->work[1].S);
    a.tw = static_cast<const float2*>(g->tw[1]) + g->plan[0].tw_off;
    a.sc = g->work[1].sc;
    a.part = g->partial;
    a.bar = g->counters + 8;
    a.err = reinterpret_cast<int*>(g->counters + 9);
    a.dual = g->form;
    a.has_A0 = g->has_ref;
    for (int i = 0; i < 4; ++i) a.A0[i] = (float)g->ref[i];
    a.band[0] = g->band[0];
    a.band[1] = g->band[1];
    a.W = grid_weight(g);
    a.drop_cta = j.res_drop_cta;
    a.wait_ns = j.res_drop_cta > 0 ? 100000000ull : 1000000000ull;   // 1 s per barrier wait (0.1 s in the test)
    HG_CU(cudaMemsetAsync(g->counters + 8, 0, 2 * sizeof(unsigned), j.s));
    const bool timed = j.o.time_pass >= 0;
    if (timed) {
        for (int i = 0; i < 2; ++i)
            if (!g->prof_ev[i]) HG_CU(cudaEventCreate(&g->prof_ev[i]));
        HG_CU(cudaEventRecord(g->prof_ev[0], j.s));
    }
    HG_CU(launch_resident(gd.N[0], a, cfg, j.s));
    if (timed) HG_CU(cudaEventRecord(g->prof_ev[1], j.s));
    g->ctx->launches++;
    j.res_ctas = cfg.T;
    j.launched = (long long)j.o.max_iter + 4LL * j.chunk;   // the launch ran every iteration
    j.cg_prec = 1;
    HG_CU(cudaMemcpyAsync(g->h_sc, g->work[1].sc, sizeof(Scalars) * MAXL, cudaMemcpyDeviceToHost, j.s));
    HG_CU(cudaEventRecord(j.tick, j.s));
    return 1;
}

static int job_launch_chunk(Job& j, int prec) {
    hg_grid* g = j.g;
    if (prec == 1) {
        const int r = job_launch_resident(j);
        if (r != 0) return r > 0 ? HG_OK : r;
    }
    cudaGraphExec_t ge;
    int nk = 0;
    int st = get_cg_graph(g, prec, j.chunk, &ge, &nk, j.o.time_pass);
    if (st) return st;
    HG_CU(cudaGraphLaunch(ge, j.s));
    g->ctx->launches += nk;
    j.launched += j.chunk;
    j.cg_prec = prec;
    HG_CU(cudaMemcpyAsync(g->h_sc, g->work[prec].sc, sizeof(Scalars) * MAXL, cudaMemcpyDeviceToHost, j.s));
    HG_CU(cudaEventRecord(j.tick, j.s));
    return HG_OK;
}

static int job_tick_copy(Job& j, int prec) {
    HG_CU(cudaMemcpyAsync(j.g->h_sc, j.g->work[prec].sc, sizeof(Scalars) * MAXL, cudaMemcpyDeviceToHost, j.s));
    HG_CU(cudaEventRecord(j.tick, j.s));
    return HG_OK;
}

static bool any_active(const Scalars* h, int L) {
    for (int l = 0; l < L; ++l)
        if (h[l].status == ST_ACTIVE) return true;
    return false;
}

static int job_start_inner(Job& j) {
    hg_grid* g = j.g;
    const GridDev& gd = g->gd;
    HG_CU(launch_inner_init(gd, gd.d, (const double*)g->work[0].r, (float*)g->work[1].r,
                            (float*)g->work[1].p, (float*)g->work[1].x, g->work[0].sc, g->work[1].sc,
                            j.o.inner_tol, j.o.max_iter, j.stall_max, grid_weight(g), g->partial,
                            g->counters + 4, j.s));
    g->ctx->launches++;
    j.launched = 0;
    j.prof_prev_iters = 0;
    j.phase = Job::INNER;
    return job_launch_chunk(j, 1);
}

static int job_finish_enqueue(Job& j) {
    hg_grid* g = j.g;
    const GridDev& gd = g->gd;
    if (j.prec == 0) {
        // FP64 recursive residuals drift from b - K x: recompute the residual of
        // the returned iterate once (INV_RESID on scratch scalars that carry
        // this solve's ||b||; the mixed path's last outer step already is it)
        HG_CU(cudaMemcpyAsync(g->d_sc_aux, g->work[0].sc, sizeof(Scalars) * MAXL, cudaMemcpyDeviceToDevice, j.s));
        const int st = enqueue_matvec(g, 0, gd.d, g->work[0].x, true, true, nullptr, nullptr, INV_RESID,
                                      nullptr, 0, j.s, g->d_sc_aux);
        if (st) return st;
        HG_CU(cudaMemcpyAsync(g->h_sc + MAXL, g->d_sc_aux, sizeof(Scalars) * MAXL, cudaMemcpyDeviceToHost, j.s));
    }
    CoeffsDev c64 = coeffs_for(g, 0, true);
    HG_CU(launch_energy(gd, gd.d, c64, (const double*)g->work[0].x, j.o.loads_mask, g->partial,
                        g->counters + 5, g->d_AH, j.s));
    g->ctx->launches++;
    HG_CU(cudaEventRecord(j.ev1, j.s));
    HG_CU(cudaMemcpyAsync(g->h_AH, g->d_AH, sizeof(double) * 2 * gd.d * gd.d, cudaMemcpyDeviceToHost, j.s));
    j.phase = Job::FINAL;
    return job_tick_copy(j, 0);
}

// Eigenvalues of a symmetric d x d matrix (row-major) by cyclic Jacobi
// rotations (Golub and Van Loan, Sec. 8.5).
static void sym_eig_host(const double* m, int d, double* ev) {
    double a[3][3];
    for (int i = 0; i < d; ++i)
        for (int k = 0; k < d; ++k) a[i][k] = m[i * d + k];
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < d; ++p)
            for (int q = p + 1; q < d; ++q) off += std::fabs(a[p][q]);
        if (off == 0.0) break;
        for (int p = 0; p < d - 1; ++p)
            for (int q = p + 1; q < d; ++q) {
                const double apq = a[p][q];
                if (apq == 0.0) continue;
                const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                a[p][p] -= t * apq;
                a[q][q] += t * apq;
                a[p][q] = a[q][p] = 0.0;
                for (int r = 0; r < d; ++r) {
                    if (r == p || r == q) continue;
                    const double arp = a[r][p], arq = a[r][q];
                    a[r][p] = a[p][r] = c * arp - sn * arq;
                    a[r][q] = a[q][r] = sn * arp + c * arq;
                }
            }
    }
    for (int i = 0; i < d; ++i) ev[i] = a[i][i];
}

// A(x_k)^-1 for the dual formulation, made once per coefficient set: phase
// tables are inverted on the host (adjugate over determinant, at most 256
// small matrices), packed fields on the device.
static void invert_small(const double* a, double* r, int d) {
    if (d == 2) {
        const double det = a[0] * a[3] - a[1] * a[2];
        r[0] = a[3] / det; r[1] = -a[1] / det; r[2] = -a[2] / det; r[3] = a[0] / det;
        return;
    }
    const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
    const double c10 = a[2] * a[7] - a[1] * a[8], c11 = a[0] * a[8] - a[2] * a[6], c12 = a[1] * a[6] - a[0] * a[7];
    const double c20 = a[1] * a[5] - a[2] * a[4], c21 = a[2] * a[3] - a[0] * a[5], c22 = a[0] * a[4] - a[1] * a[3];
    const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    // inverse = transpose of the cofactor matrix / det
    r[0] = c00 / det; r[1] = c10 / det; r[2] = c20 / det;
    r[3] = c01 / det; r[4] = c11 / det; r[5] = c21 / det;
    r[6] = c02 / det; r[7] = c12 / det; r[8] = c22 / det;
}

static int grid_ensure_inverse(hg_grid* g, cudaStream_t s) {
    if (g->inv_ok) return HG_OK;
    hg_ctx* c = g->ctx;
    const int d = g->gd.d;
    int st;
    if (g->coeff_mode == 0) {
        const size_t n = (size_t)g->n_phases * d * d;
        std::vector<double> tb(n), inv(n);
        std::vector<float> inv32(n);
        HG_CU(cudaMemcpyAsync(tb.data(), g->d_table[0], n * sizeof(double), cudaMemcpyDeviceToHost, s));
        HG_CU(cudaStreamSynchronize(s));
        for (int p = 0; p < g->n_phases; ++p) invert_small(&tb[(size_t)p * d * d], &inv[(size_t)p * d * d], d);
        for (size_t i = 0; i < n; ++i) inv32[i] = (float)inv[i];
        if (!g->d_table_inv[0] && (st = dev_alloc(c, &g->d_table_inv[0], n * sizeof(double)))) return st;
        if (!g->d_table_inv[1] && (st = dev_alloc(c, &g->d_table_inv[1], n * sizeof(float)))) return st;
        HG_CU(cudaMemcpyAsync(g->d_table_inv[0], inv.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
        HG_CU(cudaMemcpyAsync(g->d_table_inv[1], inv32.data(), n * sizeof(float), cudaMemcpyHostToDevice, s));
        HG_CU(cudaStreamSynchronize(s));   // the host buffers go out of scope
    } else {
        const size_t n = (size_t)(d * (d + 1) / 2) * g->gd.M;
        if (!g->d_field_inv[0] && (st = dev_alloc(c, &g->d_field_inv[0], n * sizeof(double)))) return st;
        if (!g->d_field_inv[1] && (st = dev_alloc(c, &g->d_field_inv[1], n * sizeof(float)))) return st;
        HG_CU(launch_invert_field(d, g->gd.M, (const double*)g->d_field[0], (double*)g->d_field_inv[0],
                                  (float*)g->d_field_inv[1], s));
        c->launches++;
    }
    g->inv_ok = true;
    return HG_OK;
}

// Moulinec-Suquet (Sec. 5.3 comments): e_i = E - Gamma_N (A_N - lambda I)
// e_{i-1} with Gamma_N = (1 / lambda) G_N for A0 = lambda I.  Writing e_i = E +
// x_i with x_i in E_N (G_N E = 0, G_N x = x on E_N, Lemma FD_projection) gives
// x_i = x_{i-1} + r_{i-1} / lambda, r = -G_N A_N (E + x): the CG iteration with
// alpha fixed to 1 / lambda and beta = 0.  The series converges for the
// spectrum [c_A, C_A] of A_N when lambda > C_A / 2, with contraction
// q = max |1 - c / lambda| over c in {c_A, C_A}, least, (rho - 1) / (rho + 1),
// at lambda = (c_A + C_A) / 2.
static int job_method_setup(Job& j) {
    hg_grid* g = j.g;
    j.fixed_alpha = 0.0;
    j.lambda = 0.0;
    j.stall_max = 64;
    if (j.o.method != HG_MS) return HG_OK;
    const int f = g->form;
    if (!g->bounds_ok[f]) {
        double* db = g->d_AH + 24;
        HG_CU(launch_coeff_bounds(g->gd, coeffs_for(g, 0, true), db, j.s));
        g->ctx->launches++;
        double hb[2] = {0.0, 0.0};
        HG_CU(cudaMemcpyAsync(hb, db, sizeof(hb), cudaMemcpyDeviceToHost, j.s));
        HG_CU(cudaStreamSynchronize(j.s));
        g->c_A[f] = hb[0];
        g->C_A[f] = hb[1];
        g->bounds_ok[f] = true;
    }
    const double cA = g->c_A[f], CA = g->C_A[f];
    const double lam = j.o.lambda_ref > 0.0 ? j.o.lambda_ref : 0.5 * (cA + CA);
    if (!(lam > 0.5 * CA) || !(cA > 0.0)) return HG_ERR_ARG;
    const double q = std::max(std::fabs(1.0 - cA / lam), std::fabs(1.0 - CA / lam));
    // an inner FP32 solve is stagnating when (r, r) has not dropped 4x in
    // twice the iterations the contraction needs for that (q^2 per step)
    const double per4 = q > 0.0 ? std::log(4.0) / (-2.0 * std::log(q)) : 1.0;
    j.stall_max = (int)std::min(1e9, 64.0 + 2.0 * std::ceil(per4));
    j.lambda = lam;
    j.fixed_alpha = 1.0 / lam;
    return HG_OK;
}

// Right-hand side b = -G A E (Eq. final_system): r = p = b, x = 0.  The mixed
// path computes b in FP32: its first inner FP32 solve would see no more of an
// FP64 b than its FP32 rounding, and the FP64 refinement recomputes the
// residual from E + x.  An FP32 b too small to decide the zero right-hand-side
// reading (ST_RHS_RECHECK) makes job_advance start over with the FP64 one.
static int job_start_rhs(Job& j, bool fp32) {
    hg_grid* g = j.g;
    const GridDev& gd = g->gd;
    const int L = gd.d;
    int init_st[MAXL];
    for (int l = 0; l < MAXL; ++l) init_st[l] = (l < L && ((j.o.loads_mask >> l) & 1u)) ? ST_ACTIVE : ST_IDLE;
    HG_CU(launch_init_scalars(g->work[0].sc, L, init_st, j.o.tol, j.prec ? j.o.max_outer : j.o.max_iter,
                              j.fixed_alpha, j.zscale, j.s));
    g->ctx->launches++;
    j.launched = 0;
    j.prof_prev_iters = 0;
    int st;
    if (!fp32) {
        if ((st = enqueue_matvec(g, 0, L, nullptr, true, true, nullptr, nullptr, INV_RHS, nullptr, 1, j.s)))
            return st;
        if (j.prec == 0) {
            j.phase = Job::PLAIN;
            return job_launch_chunk(j, 0);
        }
        return job_start_inner(j);
    }
    HG_CU(cudaMemsetAsync(g->work[0].x, 0, sizeof(double) * (size_t)L * gd.d * gd.M, j.s));
    if ((st = enqueue_matvec(g, 1, L, nullptr, true, true, nullptr, nullptr, INV_RHS, nullptr, 1, j.s,
                             g->work[0].sc)))
        return st;
    HG_CU(launch_inner_init(gd, L, nullptr, nullptr, nullptr, nullptr, g->work[0].sc, g->work[1].sc,
                            j.o.inner_tol, j.o.max_iter, j.stall_max, grid_weight(g), g->partial,
                            g->counters + 4, j.s));
    g->ctx->launches++;
    j.phase = Job::INNER;
    return job_launch_chunk(j, 1);
}

int job_begin(Job& j) {
    hg_grid* g = j.g;
    hg_ctx* ctx = g->ctx;
    const GridDev& gd = g->gd;
    const int L = gd.d;
    j.t0 = now_ms();
    j.launches0 = ctx->launches.load();
    j.prec = j.o.prec == HG_MIXED ? 1 : 0;
    j.chunk = std::max(1, j.o.check_every);
    j.outer = 0;
    j.launched = 0;
    j.result = HG_OK;
    j.prof_prev_iters = 0;
    j.prof_ms = 0.0;
    j.prof_n = 0;
    j.res_ctas = 0;
    if (g->coeff_mode < 0) return HG_ERR_NO_COEFFS;
    int st;
    if ((st = grid_alloc_common(g))) return st;
    if ((st = grid_alloc_work(g, 0))) return st;
    if (j.prec == 1 && (st = grid_alloc_work(g, 1))) return st;
    g->form = j.o.formulation == HG_DUAL ? 1 : 0;
    g->has_ref = j.o.A0[0] != 0.0 ? 1 : 0;
    g->use_plane = j.o.resident != 0;
    j.zscale = 1.0;
    for (int i = 0; i < 9; ++i) g->ref[i] = g->has_ref && i < gd.d * gd.d ? j.o.A0[i] : 0.0;
    if (g->has_ref) {
        // ||b||_A0 <= sqrt(lmax(A0)) / lmin(A0) ||A E|| (reading of the zero test)
        double ev[3] = {0.0, 0.0, 0.0};
        sym_eig_host(g->ref, gd.d, ev);
        const double lmin = *std::min_element(ev, ev + gd.d), lmax = *std::max_element(ev, ev + gd.d);
        j.zscale = std::sqrt(lmax) / lmin;
    }
    if (g->form) {
        if ((j.o.loads_mask & ((1u << L) - 1u)) != ((1u << L) - 1u)) return HG_ERR_ARG;
        if ((st = grid_ensure_inverse(g, j.s))) return st;
    }
    if ((st = job_method_setup(j))) return st;
    HG_CU(cudaEventRecord(j.ev0, j.s));
    return job_start_rhs(j, j.prec == 1);
}

// Called once the job's tick event has completed.  Enqueues the next step or
// completes the job (*done = true, result in j.res).
int job_advance(Job& j, bool* done) {
    hg_grid* g = j.g;
    const GridDev& gd = g->gd;
    const int L = gd.d;
    *done = false;
    const Scalars* h = g->h_sc;
    switch (j.phase) {
        case Job::PLAIN:
        case Job::INNER: {
            for (int l = 0; l < L; ++l) {
                // a bounded wait of the resident solver gave up: its state is
                // incomplete, the solve ends here (the context stays usable)
                if (h[l].status == ST_TIMEOUT) return HG_ERR_DEVICE_TIMEOUT;
                if (h[l].status == ST_RHS_RECHECK) return job_start_rhs(j, false);
            }
            job_collect_pass_times(j);
            const int mi = j.o.max_iter;
            if (any_active(h, L) && j.launched <= (long long)mi + 2 * j.chunk)
                return job_launch_chunk(j, j.cg_prec);
            if (j.phase == Job::PLAIN) return job_finish_enqueue(j);
            // FP32 roundoff in q = G A p (relative to |A p|, up to rho |p|)
            // leaves a part of the FP32 correction delta outside E_N, which the
            // FP64 residual cannot see but A_H would, to first order.  Gamma_N
            // is the orthogonal projection onto E_N (Lemma FD_projection
            // (iii),(v)): delta <- Gamma_N delta in FP32 (error eps32 |delta|,
            // no contrast factor), x64 += delta, and for tolerances below 1e-8
            // also x64 <- Gamma_N x64 in FP64.  Then the FP64 residual
            // r = -G A (E + x).
            int st = enqueue_matvec(g, 1, L, g->work[1].x, false, false, nullptr, nullptr, INV_PROJ,
                                    nullptr, 1, j.s, g->work[0].sc);
            if (st) return st;
            HG_CU(launch_outer_update(gd, L, (double*)g->work[0].x, (const float*)g->work[1].x,
                                      g->work[0].sc, g->work[1].sc, j.s));
            g->ctx->launches++;
            if (j.o.tol < 1e-8) {
                st = enqueue_matvec(g, 0, L, g->work[0].x, false, false, nullptr, nullptr, INV_PROJ,
                                    nullptr, 1, j.s);
                if (st) return st;
            }
            st = enqueue_matvec(g, 0, L, g->work[0].x, true, true, nullptr, nullptr, INV_RESID,
                                nullptr, 1, j.s);
            if (st) return st;
            j.outer++;
            j.phase = Job::RESID;
            return job_tick_copy(j, 0);
        }
        case Job::RESID:
            if (any_active(h, L) && j.outer < std::max(1, j.o.max_outer)) return job_start_inner(j);
            return job_finish_enqueue(j);
        case Job::FINAL: {
            float dms = 0.f;
            cudaEventElapsedTime(&dms, j.ev0, j.ev1);
            int result = HG_OK;
            hg_result& r = j.res;
            memset(&r, 0, sizeof(r));
            r.d = gd.d;
            for (int i = 0; i < gd.d * gd.d; ++i) { r.AH[i] = g->h_AH[i]; r.AH_flux[i] = g->h_AH[gd.d * gd.d + i]; }
            if (g->form) {
                // the energy of the flux loads is the compliance: A_H = C_H^-1
                double ch[9], chf[9];
                for (int i = 0; i < gd.d * gd.d; ++i) { ch[i] = r.AH[i]; chf[i] = r.AH_flux[i]; r.CH[i] = ch[i]; }
                invert_small(ch, r.AH, gd.d);
                invert_small(chf, r.AH_flux, gd.d);
            }
            for (int l = 0; l < L; ++l) {
                const Scalars& sc = h[l];
                int ms = map_status(sc.status);
                if (j.prec == 0) {
                    r.iters[l] = sc.iters;
                } else {
                    r.iters[l] = sc.total_iters;
                    r.outer[l] = sc.iters;
                }
                if (ms != HG_OK && result == HG_OK) result = ms;
                r.rel_res[l] = sc.relres;
                const bool solved = sc.status != ST_IDLE && sc.status != ST_ZERO_RHS && sc.bnorm > 0.0;
                r.true_rel_res[l] = !solved ? 0.0 : (j.prec == 0 ? g->h_sc[MAXL + l].relres : sc.relres);
            }
            r.resident_ctas = j.res_ctas;
            r.status = result;
            r.device_ms = dms;
            r.wall_ms = now_ms() - j.t0;
            r.launches = g->ctx->launches.load() - j.launches0;
            r.pass_ms_total = j.prof_ms;
            r.pass_launches = j.prof_n;
            if (j.o.method == HG_MS) {
                r.lambda_ref = j.lambda;
                r.c_A = g->c_A[g->form];
                r.C_A = g->C_A[g->form];
            }
            g->last_prec = j.prec;
            j.result = result;
            j.phase = Job::DONE;
            *done = true;
            return HG_OK;
        }
        default:
            *done = true;
            return HG_OK;
    }
}

int solve_impl(hg_grid* g, const hg_solve_opts* o, double* AH_out, hg_result* info, int res_drop_cta) {
    Job j;
    j.g = g;
    j.o = *o;
    j.s = g->ctx->stream;
    j.allow_resident = true;
    j.res_drop_cta = res_drop_cta;
    j.ev0 = g->ev0;
    j.ev1 = g->ev1;
    j.tick = g->ev_tick;
    int st = job_begin(j);
    bool done = false;
    while (st == HG_OK && !done) {
        HG_CU(cudaEventSynchronize(j.tick));
        st = job_advance(j, &done);
    }
    if (st != HG_OK) {
        cudaStreamSynchronize(j.s);
        return st;
    }
    if (AH_out) memcpy(AH_out, j.res.AH, sizeof(double) * g->gd.d * g->gd.d);
    if (info) *info = j.res;
    return j.result;
}

}  // namespace hgrt
