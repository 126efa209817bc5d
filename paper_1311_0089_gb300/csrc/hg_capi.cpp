// extern "C" entry points of libhg (declared in include/hg.h).
#include "hg.h"
#include "hg_internal.h"
#include "hg_runtime.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
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

// A1-A2 (Sec. 3): symmetric and uniformly elliptic.  Checks one d x d tensor
// (row-major) by symmetry and a Cholesky factorisation.
bool is_spd(const double* a, int d) {
    double scale = 0.0;
    for (int i = 0; i < d * d; ++i) {
        if (!std::isfinite(a[i])) return false;
        scale = std::max(scale, std::fabs(a[i]));
    }
    if (scale == 0.0) return false;
    for (int i = 0; i < d; ++i)
        for (int j = i + 1; j < d; ++j)
            if (std::fabs(a[i * d + j] - a[j * d + i]) > 1e-12 * scale) return false;
    double L[9] = {0};
    for (int j = 0; j < d; ++j) {
        double s = a[j * d + j];
        for (int k = 0; k < j; ++k) s -= L[j * 3 + k] * L[j * 3 + k];
        if (!(s > 1e-14 * scale)) return false;
        L[j * 3 + j] = std::sqrt(s);
        for (int i = j + 1; i < d; ++i) {
            double t = a[i * d + j];
            for (int k = 0; k < j; ++k) t -= L[i * 3 + k] * L[j * 3 + k];
            L[i * 3 + j] = t / L[j * 3 + j];
        }
    }
    return true;
}

int check_size(int n) {
    if (n < 1 || n > 1024 || (n % 2) == 0) return HG_ERR_UNSUPPORTED_SIZE;
    int m = n;
    for (int r : {3, 5, 7})
        while (m % r == 0) m /= r;
    return m == 1 ? HG_OK : HG_ERR_UNSUPPORTED_SIZE;
}

void free_inverse_coeffs(hg_grid* g) {
    for (int p = 0; p < 2; ++p) {
        dev_free(g->ctx, g->d_table_inv[p]);
        dev_free(g->ctx, g->d_field_inv[p]);
        g->d_table_inv[p] = g->d_field_inv[p] = nullptr;
    }
    g->inv_ok = false;
}

void free_coeffs(hg_grid* g) {
    // cached CG graphs hold the coefficient pointers (and the band) they were captured with
    for (int p = 0; p < 2; ++p) {
        if (g->graphs[p].exec) cudaGraphExecDestroy(g->graphs[p].exec);
        g->graphs[p] = hgrt::GraphCache();
    }
    dev_free(g->ctx, g->d_phase);
    g->d_phase = nullptr;
    for (int p = 0; p < 2; ++p) {
        dev_free(g->ctx, g->d_table[p]);
        dev_free(g->ctx, g->d_field[p]);
        g->d_table[p] = g->d_field[p] = nullptr;
    }
    free_inverse_coeffs(g);
    g->coeff_mode = -1;
    g->exact = false;
    g->band[0] = g->band[1] = g->band[2] = 0;
}

struct DeviceGuard {
    explicit DeviceGuard(int dev) { cudaSetDevice(dev); }
};

}  // namespace

namespace hgrt {
// Options of hg_solve_AH and hg_submit.  Normalises loads_mask to the grid.
int validate_solve_opts(const hg_grid* g, hg_solve_opts* o) {
    if (!(o->tol > 0.0) || o->max_iter < 1 || (o->prec != HG_FP64 && o->prec != HG_MIXED) ||
        !(o->inner_tol > 0.0) || o->inner_tol >= 1.0 || (o->method != HG_CG && o->method != HG_MS) ||
        !std::isfinite(o->lambda_ref) || (o->formulation != HG_PRIMAL && o->formulation != HG_DUAL) ||
        o->resident < -1)
        return HG_ERR_ARG;
    if (o->A0[0] != 0.0) {
        if (o->method != HG_CG || o->formulation != HG_PRIMAL || g->exact) return HG_ERR_ARG;
        if (!is_spd(o->A0, g->gd.d)) return HG_ERR_NOT_SPD;
    }
    // exact-integration coefficients are not SPD pointwise: no eigenvalue bounds
    if (g->exact && o->method == HG_MS) return HG_ERR_ARG;
    o->loads_mask &= (1u << g->gd.d) - 1u;
    return HG_OK;
}

// Buffers and steady-state CG scalars (every system active, alpha = beta =
// 0.5, no convergence) for timing single passes of precision pr on the
// primal operator with A0 = I.  The work buffers are left with meaningless
// values: every solve starts from its own right-hand side.
int timing_state(hg_grid* g, int pr, cudaStream_t s) {
    g->form = 0;
    g->has_ref = 0;
    int st;
    if ((st = grid_alloc_common(g))) return st;
    if ((st = grid_alloc_work(g, pr))) return st;
    Scalars hs[MAXL];
    memset(hs, 0, sizeof(hs));
    for (int l = 0; l < MAXL; ++l) {
        hs[l].rr = 1.0; hs[l].alpha = 0.5; hs[l].beta = 0.5; hs[l].bnorm = 1.0; hs[l].tol = 0.0;
        hs[l].alpha_f = 0.5f; hs[l].beta_f = 0.5f;
        hs[l].max_iter = 1 << 30; hs[l].status = ST_ACTIVE;
    }
    HG_CU(cudaMemcpyAsync(g->work[pr].sc, hs, sizeof(hs), cudaMemcpyHostToDevice, s));
    return HG_OK;
}

// One launch of pass `pass` of the CG iteration (0 = last-axis forward pass,
// 1.. = strided passes in launch order, hg_num_passes - 1 = last-axis
// inverse pass) on the state timing_state() set up, with the grid's current
// launch geometry; nm (64 chars) receives the pass name if not null.
int enqueue_timing_pass(hg_grid* g, int pr, int pass, char* nm, cudaStream_t s) {
    const GridDev& gd = g->gd;
    const int L = gd.d, last = gd.d - 1;
    const int np = gd.d == 2 ? 3 : 5;
    Work& w = g->work[pr];
    if (pass == 0) {
        RowFwdArgs fa;
        memset(&fa, 0, sizeof(fa));
        fa.early_stage = 1;
        fa.mode = FWD_CG; fa.L = L; fa.co = coeffs_for(g, pr, true);
        fa.p = w.p; fa.r = w.r; fa.S = w.S; fa.sc = w.sc;
        fa.partial = g->partial; fa.counter = g->counters + 0; fa.check_status = 0;
        if (nm) snprintf(nm, 64, "k_row_fwd<%s,%d> (A.p + R2C DFT, axis %d)", pr ? "float" : "double", gd.d, last);
        HG_CU(launch_row_fwd(pr, gd, g->plan[last], g->tw[pr], g->rowcfg[pr], fa, s));
    } else if (pass == np - 1) {
        RowInvArgs ia;
        memset(&ia, 0, sizeof(ia));
        ia.early_stage = 1;
        ia.mode = INV_CG; ia.L = L; ia.S = w.S; ia.x = w.x; ia.r = w.r; ia.p = w.p;
        ia.sc = w.sc; ia.partial = g->partial; ia.counter = g->counters + 1; ia.check_status = 0;
        if (nm) snprintf(nm, 64, "k_row_inv<%s,%d> (C2R DFT + CG update, axis %d)", pr ? "float" : "double", gd.d, last);
        HG_CU(launch_row_inv(pr, gd, g->plan[last], g->tw[pr], g->rowcfg[pr], ia, s));
    } else if (pass > 0 && pass < np - 1) {
        StrArgs sa;
        memset(&sa, 0, sizeof(sa));
        sa.early_stage = 1;
        sa.L = L; sa.S = w.S; sa.sc = w.sc; sa.check_status = 0;
        int axis;
        if (gd.d == 2 || pass == 2) {
            axis = 0; sa.mode = STR_GAMMA; sa.outer = 1; sa.n = gd.N[0]; sa.inner = gd.Ms / gd.N[0];
        } else {
            axis = 1; sa.mode = pass == 1 ? STR_FWD : STR_INV; sa.outer = gd.N[0]; sa.n = gd.N[1]; sa.inner = gd.H;
        }
        sa.axis = axis;
        if (nm) snprintf(nm, 64, "k_strided<%s,%d> (%s, axis %d)", pr ? "float" : "double", gd.d,
                         sa.mode == STR_GAMMA ? "DFT + Gamma_hat + iDFT" : sa.mode == STR_FWD ? "DFT" : "iDFT", axis);
        HG_CU(launch_strided(pr, gd, g->plan[axis], g->tw[pr], g->strcfg[pr][axis], sa, s));
    } else {
        return HG_ERR_ARG;
    }
    g->ctx->launches++;
    return HG_OK;
}
}  // namespace hgrt

extern "C" {

void hg_default_opts(hg_solve_opts* o) {
    if (!o) return;
    o->tol = 1e-10;
    o->max_iter = 10000;
    o->prec = HG_FP64;
    o->lambda_ref = 0.0;
    o->loads_mask = 0x7u;
    o->inner_tol = 1e-4;
    o->check_every = 8;
    o->max_outer = 30;
    o->time_pass = -1;
    o->method = HG_CG;
    o->formulation = HG_PRIMAL;
    for (int i = 0; i < 9; ++i) o->A0[i] = 0.0;
    o->batch_tiles = 1;
    o->resident = -1;
}

const char* hg_strerror(int s) {
    switch (s) {
        case HG_OK: return "ok";
        case HG_PENDING: return "pending";
        case HG_ERR_ARG: return "invalid argument";
        case HG_ERR_UNSUPPORTED_SIZE: return "unsupported grid size (every N must be odd, 1..1024, with prime factors 3, 5, 7)";
        case HG_ERR_NOT_SPD: return "coefficients are not symmetric positive definite";
        case HG_ERR_NO_MEMORY: return "out of device memory or over the context budget";
        case HG_ERR_NOT_CONVERGED: return "not converged within max_iter";
        case HG_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
        case HG_ERR_BUSY: return "grid is borrowed by a pending ticket";
        case HG_ERR_CUDA: return last_cuda_error()[0] ? last_cuda_error() : "CUDA error";
        case HG_ERR_CANCELLED: return "cancelled";
        case HG_ERR_BREAKDOWN: return "CG breakdown ((p, A p) <= 0 or not finite)";
        case HG_ERR_NO_COEFFS: return "coefficients not set";
        case HG_ERR_TOO_LARGE: return "grid too large for the fixed 16 MiB scratch of hg_apply_noalloc";
        default: return "unknown status";
    }
}

int hg_create(hg_ctx** out, int device, size_t budget, void* stream) {
    if (!out) return HG_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    HG_CU(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return HG_ERR_ARG;
    HG_CU(cudaSetDevice(device));
    hg_ctx* c = new hg_ctx();
    c->device = device;
    c->budget = budget;
    if (stream) {
        c->stream = (cudaStream_t)stream;
        c->own_stream = false;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete c; set_last_cuda_error(e, "cudaStreamCreate"); return HG_ERR_CUDA; }
        c->own_stream = true;
    }
    {
        cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            if (c->own_stream) cudaStreamDestroy(c->stream);
            delete c;
            set_last_cuda_error(e, "cudaStreamCreate");
            return HG_ERR_CUDA;
        }
    }
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    c->max_smem = std::max(48 * 1024, optin - 4 * 1024);
    cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device);
    if (c->nsm < 1) c->nsm = 1;
    cudaError_t e = configure_kernels(c->max_smem);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "cudaFuncSetAttribute");
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return HG_ERR_CUDA;
    }
    c->sched = sched_create(c);
    *out = c;
    return HG_OK;
}

int hg_destroy(hg_ctx* c) {
    if (!c) return HG_ERR_ARG;
    if (c->ngrids.load() > 0) return HG_ERR_BUSY;
    DeviceGuard dg(c->device);
    if (c->sched) sched_destroy(c->sched);
    cudaStreamSynchronize(c->stream);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
    return HG_OK;
}

long long hg_launch_count(hg_ctx* c) { return c ? c->launches.load() : -1; }

int hg_create_grid(hg_ctx* c, int d, const int* N, const double* Y, hg_grid** out) {
    if (!c || !N || !out) return HG_ERR_ARG;
    *out = nullptr;
    if (d != 2 && d != 3) return HG_ERR_ARG;
    for (int a = 0; a < d; ++a) {
        int s = check_size(N[a]);
        if (s) return s;
        if (Y && !(Y[a] > 0.0 && std::isfinite(Y[a]))) return HG_ERR_ARG;
    }
    DeviceGuard dg(c->device);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    hg_grid* g = new hg_grid();
    g->ctx = c;
    GridDev& gd = g->gd;
    gd.d = d;
    gd.M = 1;
    for (int a = 0; a < 3; ++a) {
        gd.N[a] = a < d ? N[a] : 1;
        gd.Y[a] = (a < d && Y) ? Y[a] : 1.0;
        gd.invY[a] = 1.0 / gd.Y[a];
        gd.invYf[a] = (float)gd.invY[a];
    }
    for (int a = 0; a < d; ++a) gd.M *= N[a];
    gd.Nl = N[d - 1];
    gd.H = (gd.Nl + 1) / 2;
    gd.rows = gd.M / gd.Nl;
    gd.Ms = gd.rows * gd.H;
    gd.invM = 1.0 / (double)gd.M;
    gd.invMf = (float)gd.invM;
    int st = grid_init_plans(g);
    if (st == HG_OK) {
        cudaError_t e = cudaMallocHost((void**)&g->h_sc, sizeof(Scalars) * 2 * MAXL);
        if (e == cudaSuccess) e = cudaMallocHost((void**)&g->h_AH, sizeof(double) * 32);
        if (e == cudaSuccess) e = cudaEventCreate(&g->ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&g->ev1);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_tick, cudaEventDisableTiming);
        if (e != cudaSuccess) { set_last_cuda_error(e, "grid host state"); st = HG_ERR_CUDA; }
    }
    if (st != HG_OK) {
        hg_destroy_grid(g);
        return st;
    }
    c->ngrids += 1;
    c->grids.insert(g);
    g->counted = true;
    *out = g;
    return HG_OK;
}

int hg_destroy_grid(hg_grid* g) {
    if (!g) return HG_ERR_ARG;
    if (g->borrowed.load() > 0) return HG_ERR_BUSY;
    hg_ctx* c = g->ctx;
    DeviceGuard dg(c->device);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    cudaStreamSynchronize(c->stream);
    grid_free_work(g);
    for (int p = 0; p < 2; ++p) dev_free(c, g->tw[p]);
    free_coeffs(g);
    dev_free(c, g->partial);
    dev_free(c, g->counters);
    dev_free(c, g->d_AH);
    dev_free(c, g->d_E);
    dev_free(c, g->d_A0);
    if (g->h_sc) cudaFreeHost(g->h_sc);
    if (g->h_AH) cudaFreeHost(g->h_AH);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    if (g->ev_tick) cudaEventDestroy(g->ev_tick);
    for (int i = 0; i < 2 * hgrt::MAX_PROF_CHUNK; ++i)
        if (g->prof_ev[i]) cudaEventDestroy(g->prof_ev[i]);
    if (g->counted) {
        c->ngrids -= 1;
        c->grids.erase(g);
    }
    delete g;
    return HG_OK;
}

int hg_set_coeffs(hg_grid* g, const double* A, int layout, int on_device) {
    if (!g || !A || (layout != HG_COEFF_FULL && layout != HG_COEFF_PACKED)) return HG_ERR_ARG;
    if (g->borrowed.load() > 0) return HG_ERR_BUSY;
    hg_ctx* c = g->ctx;
    DeviceGuard dg(c->device);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    const int d = g->gd.d;
    const long long M = g->gd.M;
    const int npk = d * (d + 1) / 2;
    const size_t nin = (size_t)M * (layout == HG_COEFF_FULL ? d * d : npk);
    std::vector<double> host;
    const double* src = A;
    if (on_device) {
        host.resize(nin);
        HG_CU(cudaMemcpyAsync(host.data(), A, nin * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        HG_CU(cudaStreamSynchronize(c->stream));
        src = host.data();
    }
    // pack as component-major (11,22[,33],12[,13,23]) and check A1-A2 per voxel
    static const int pi2[3][2] = {{0, 0}, {1, 1}, {0, 1}};
    static const int pi3[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    std::vector<double> pk((size_t)npk * M);
    for (long long k = 0; k < M; ++k) {
        double a[9];
        if (layout == HG_COEFF_FULL) {
            for (int i = 0; i < d * d; ++i) a[i] = src[k * d * d + i];
        } else {
            for (int q = 0; q < npk; ++q) {
                const int i = d == 2 ? pi2[q][0] : pi3[q][0];
                const int j = d == 2 ? pi2[q][1] : pi3[q][1];
                a[i * d + j] = a[j * d + i] = src[(size_t)q * M + k];
            }
        }
        if (!is_spd(a, d)) return HG_ERR_NOT_SPD;
        for (int q = 0; q < npk; ++q) {
            const int i = d == 2 ? pi2[q][0] : pi3[q][0];
            const int j = d == 2 ? pi2[q][1] : pi3[q][1];
            pk[(size_t)q * M + k] = a[i * d + j];
        }
    }
    std::vector<float> pk32(pk.size());
    for (size_t i = 0; i < pk.size(); ++i) pk32[i] = (float)pk[i];
    HG_CU(cudaStreamSynchronize(c->stream));
    free_coeffs(g);
    int st;
    if ((st = dev_alloc(c, &g->d_field[0], pk.size() * sizeof(double)))) return st;
    if ((st = dev_alloc(c, &g->d_field[1], pk32.size() * sizeof(float)))) return st;
    HG_CU(cudaMemcpyAsync(g->d_field[0], pk.data(), pk.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    HG_CU(cudaMemcpyAsync(g->d_field[1], pk32.data(), pk32.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    HG_CU(cudaStreamSynchronize(c->stream));
    g->coeff_mode = 1;
    g->bounds_ok[0] = g->bounds_ok[1] = false;
    g->exact = false;
    g->band[0] = g->band[1] = g->band[2] = 0;
    return HG_OK;
}

int hg_set_coeffs_phase(hg_grid* g, const uint8_t* phase, int n_phases, const double* table,
                        int on_device) {
    if (!g || !phase || !table || n_phases < 1 || n_phases > 256) return HG_ERR_ARG;
    if (g->borrowed.load() > 0) return HG_ERR_BUSY;
    hg_ctx* c = g->ctx;
    DeviceGuard dg(c->device);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    const int d = g->gd.d;
    const long long M = g->gd.M;
    std::vector<double> tb((size_t)n_phases * d * d);
    std::vector<uint8_t> ph;
    const uint8_t* phsrc = phase;
    if (on_device) {
        HG_CU(cudaMemcpyAsync(tb.data(), table, tb.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        ph.resize(M);
        HG_CU(cudaMemcpyAsync(ph.data(), phase, M, cudaMemcpyDeviceToHost, c->stream));
        HG_CU(cudaStreamSynchronize(c->stream));
        phsrc = ph.data();
    } else {
        memcpy(tb.data(), table, tb.size() * sizeof(double));
    }
    for (int p = 0; p < n_phases; ++p)
        if (!is_spd(&tb[(size_t)p * d * d], d)) return HG_ERR_NOT_SPD;
    if (n_phases < 256) {
        for (long long k = 0; k < M; ++k)
            if (phsrc[k] >= n_phases) return HG_ERR_ARG;
    }
    std::vector<float> tb32(tb.size());
    for (size_t i = 0; i < tb.size(); ++i) tb32[i] = (float)tb[i];
    HG_CU(cudaStreamSynchronize(c->stream));
    // same shape as the current phase coefficients: overwrite in place (no
    // cudaFree/cudaMalloc, which would synchronise the device)
    const bool reuse = g->coeff_mode == 0 && g->n_phases == n_phases && g->d_phase;
    if (!reuse) {
        free_coeffs(g);
        int st;
        if ((st = dev_alloc(c, (void**)&g->d_phase, (size_t)M))) return st;
        if ((st = dev_alloc(c, &g->d_table[0], tb.size() * sizeof(double)))) return st;
        if ((st = dev_alloc(c, &g->d_table[1], tb32.size() * sizeof(float)))) return st;
    }
    HG_CU(cudaMemcpyAsync(g->d_phase, phase, (size_t)M,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    HG_CU(cudaMemcpyAsync(g->d_table[0], tb.data(), tb.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    HG_CU(cudaMemcpyAsync(g->d_table[1], tb32.data(), tb32.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    HG_CU(cudaStreamSynchronize(c->stream));
    g->coeff_mode = 0;
    g->bounds_ok[0] = g->bounds_ok[1] = false;
    g->inv_ok = false;   // a reused phase table keeps its buffers; the inverse is redone
    g->exact = false;
    g->band[0] = g->band[1] = g->band[2] = 0;
    g->n_phases = n_phases;
    return HG_OK;
}

int hg_set_coeffs_exact(hg_grid* g, const int* N_trial, const int* P, const uint8_t* phase, int n_phases,
                        const double* table) {
    if (!g || !N_trial || !P || !phase || !table || n_phases < 1 || n_phases > 256) return HG_ERR_ARG;
    if (g->borrowed.load() > 0) return HG_ERR_BUSY;
    const int d = g->gd.d;
    long long Pt = 1;
    for (int a = 0; a < d; ++a) {
        if (N_trial[a] < 1 || (N_trial[a] % 2) == 0 || 2 * N_trial[a] - 1 > g->gd.N[a]) return HG_ERR_ARG;
        if (P[a] < 1 || P[a] > 4096) return HG_ERR_ARG;
        Pt *= P[a];
    }
    std::vector<double> tb((size_t)n_phases * d * d), tinv(tb.size());
    memcpy(tb.data(), table, tb.size() * sizeof(double));
    for (int p = 0; p < n_phases; ++p) {
        const double* a = &tb[(size_t)p * d * d];
        if (!is_spd(a, d)) return HG_ERR_NOT_SPD;
        // A^-1 for the dual: adjugate over determinant
        double* r = &tinv[(size_t)p * d * d];
        if (d == 2) {
            const double det = a[0] * a[3] - a[1] * a[2];
            r[0] = a[3] / det; r[1] = -a[1] / det; r[2] = -a[2] / det; r[3] = a[0] / det;
        } else {
            const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8];
            const double c02 = a[3] * a[7] - a[4] * a[6], c10 = a[2] * a[7] - a[1] * a[8];
            const double c11 = a[0] * a[8] - a[2] * a[6], c12 = a[1] * a[6] - a[0] * a[7];
            const double c20 = a[1] * a[5] - a[2] * a[4], c21 = a[2] * a[3] - a[0] * a[5];
            const double c22 = a[0] * a[4] - a[1] * a[3];
            const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
            r[0] = c00 / det; r[1] = c10 / det; r[2] = c20 / det;
            r[3] = c01 / det; r[4] = c11 / det; r[5] = c21 / det;
            r[6] = c02 / det; r[7] = c12 / det; r[8] = c22 / det;
        }
    }
    if (n_phases < 256)
        for (long long k = 0; k < Pt; ++k)
            if (phase[k] >= n_phases) return HG_ERR_ARG;
    hg_ctx* c = g->ctx;
    DeviceGuard dg(c->device);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    cudaStream_t s = c->stream;
    const size_t nf = (size_t)(d * (d + 1) / 2) * g->gd.M;
    free_coeffs(g);
    int st;
    uint8_t* d_phase = nullptr;
    double* d_tab = nullptr;
    auto done = [&](int code) {
        dev_free(c, d_phase);
        dev_free(c, d_tab);
        return code;
    };
    if ((st = dev_alloc(c, (void**)&d_phase, (size_t)Pt))) return done(st);
    if ((st = dev_alloc(c, (void**)&d_tab, 2 * tb.size() * sizeof(double)))) return done(st);
    for (int p = 0; p < 2; ++p) {
        if ((st = dev_alloc(c, &g->d_field[p], nf * (p ? sizeof(float) : sizeof(double))))) return done(st);
        if ((st = dev_alloc(c, &g->d_field_inv[p], nf * (p ? sizeof(float) : sizeof(double))))) return done(st);
    }
    cudaError_t e = cudaMemcpyAsync(d_phase, phase, (size_t)Pt, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_tab, tb.data(), tb.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_tab + tb.size(), tinv.data(), tb.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "hg_set_coeffs_exact");
        return done(HG_ERR_CUDA);
    }
    if ((st = ga_build_field(g, N_trial, P, d_phase, d_tab, (double*)g->d_field[0], (float*)g->d_field[1], s)))
        return done(st);
    if ((st = ga_build_field(g, N_trial, P, d_phase, d_tab + tb.size(), (double*)g->d_field_inv[0],
                             (float*)g->d_field_inv[1], s)))
        return done(st);
    g->coeff_mode = 1;
    g->bounds_ok[0] = g->bounds_ok[1] = false;
    g->inv_ok = true;   // the dual's coefficients are (A^-1)_M, not the pointwise inverse of A_M
    g->exact = true;
    for (int a = 0; a < 3; ++a) g->band[a] = a < d ? N_trial[a] : 0;
    return done(HG_OK);
}

int hg_solve_AH(hg_grid* g, const hg_solve_opts* opts, double* AH_out, hg_result* info) {
    if (!g) return HG_ERR_ARG;
    hg_solve_opts o;
    if (opts) o = *opts; else hg_default_opts(&o);
    const int vst = validate_solve_opts(g, &o);
    if (vst) return vst;
    if (o.time_pass >= hg_num_iter_passes(g, &o) || (o.time_pass >= 0 && o.check_every > hgrt::MAX_PROF_CHUNK))
        return HG_ERR_ARG;
    if (g->borrowed.load() > 0) return HG_ERR_BUSY;
    hg_ctx* c = g->ctx;
    DeviceGuard dg(c->device);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    return solve_impl(g, &o, AH_out, info);
}

int hg_test_resident_timeout(hg_grid* g, const hg_solve_opts* opts, int drop_cta, hg_result* info) {
    if (!g || drop_cta < 1) return HG_ERR_ARG;
    hg_solve_opts o;
    if (opts) o = *opts; else hg_default_opts(&o);
    const int vst = validate_solve_opts(g, &o);
    if (vst) return vst;
    if (o.prec != HG_MIXED || o.resident == 0 || o.time_pass >= 0) return HG_ERR_ARG;
    if (g->borrowed.load() > 0) return HG_ERR_BUSY;
    hg_ctx* c = g->ctx;
    DeviceGuard dg(c->device);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    return solve_impl(g, &o, nullptr, info, drop_cta);
}

int hg_get_field(hg_grid* g, int load, double* e_out, int on_device) {
    if (!g || !e_out || load < 0 || load >= g->gd.d) return HG_ERR_ARG;
    if (!g->work[0].ready) return HG_ERR_ARG;
    hg_ctx* c = g->ctx;
    DeviceGuard dg(c->device);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    const size_t n = (size_t)g->gd.d * g->gd.M;
    const double* src = (const double*)g->work[0].x + (size_t)load * n;
    HG_CU(cudaMemcpyAsync(e_out, src, n * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    HG_CU(cudaStreamSynchronize(c->stream));
    return HG_OK;
}

int hg_apply(hg_grid* g, const double* u, double* out, int with_A, const double* A0, int prec,
             int on_device) {
    if (!g || !u || !out || (prec != HG_FP64 && prec != HG_MIXED)) return HG_ERR_ARG;
    if (with_A && g->coeff_mode < 0) return HG_ERR_NO_COEFFS;
    if (A0 && !is_spd(A0, g->gd.d)) return HG_ERR_NOT_SPD;
    if (g->borrowed.load() > 0) return HG_ERR_BUSY;
    hg_ctx* c = g->ctx;
    DeviceGuard dg(c->device);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    g->form = 0;   // primal operator
    g->has_ref = 0;  // reference medium I
    cudaStream_t s = c->stream;
    const int pr = prec == HG_MIXED ? 1 : 0;
    int st;
    if ((st = grid_alloc_common(g))) return st;
    if ((st = grid_alloc_work(g, 0))) return st;
    if (pr == 1 && (st = grid_alloc_work(g, 1))) return st;
    const size_t n = (size_t)g->gd.d * g->gd.M;
    HG_CU(cudaMemcpyAsync(g->work[0].x, u, n * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (pr == 1) { HG_CU(launch_convert(g->work[0].x, 0, g->work[1].x, 1, (long long)n, s)); c->launches++; }
    const double* A0dev = nullptr;
    if (A0) {
        HG_CU(cudaMemcpyAsync(g->d_A0, A0, sizeof(double) * g->gd.d * g->gd.d, cudaMemcpyHostToDevice, s));
        A0dev = g->d_A0;
    }
    if ((st = enqueue_matvec(g, pr, 1, g->work[pr].x, false, with_A != 0, A0dev, A0, INV_OUT,
                             g->work[pr].r, 0, s))) return st;
    if (pr == 1) { HG_CU(launch_convert(g->work[1].r, 1, g->work[0].r, 0, (long long)n, s)); c->launches++; }
    HG_CU(cudaMemcpyAsync(out, g->work[0].r, n * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    HG_CU(cudaStreamSynchronize(s));
    return HG_OK;
}

int hg_spectrum(hg_grid* g, const double* u, double* S_out, int prec, int on_device) {
    if (!g || !u || !S_out || (prec != HG_FP64 && prec != HG_MIXED)) return HG_ERR_ARG;
    if (g->borrowed.load() > 0) return HG_ERR_BUSY;
    hg_ctx* c = g->ctx;
    DeviceGuard dg(c->device);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    g->form = 0;   // primal operator
    g->has_ref = 0;  // reference medium I
    cudaStream_t s = c->stream;
    const int pr = prec == HG_MIXED ? 1 : 0;
    int st;
    if ((st = grid_alloc_common(g))) return st;
    if ((st = grid_alloc_work(g, 0))) return st;
    if (pr == 1 && (st = grid_alloc_work(g, 1))) return st;
    const GridDev& gd = g->gd;
    const size_t n = (size_t)gd.d * gd.M;
    HG_CU(cudaMemcpyAsync(g->work[0].x, u, n * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (pr == 1) { HG_CU(launch_convert(g->work[0].x, 0, g->work[1].x, 1, (long long)n, s)); c->launches++; }
    Work& w = g->work[pr];
    RowFwdArgs fa;
    memset(&fa, 0, sizeof(fa));
    fa.early_stage = 1;
    fa.mode = FWD_APPLY; fa.L = 1; fa.co = coeffs_for(g, pr, false);
    fa.u = w.x; fa.S = w.S; fa.sc = w.sc; fa.partial = g->partial; fa.counter = g->counters + 2;
    const int last = gd.d - 1;
    HG_CU(launch_row_fwd(pr, gd, g->plan[last], g->tw[pr], g->rowcfg[pr], fa, s));
    c->launches++;
    if ((st = enqueue_forward_strided(g, pr, 1, 0, STR_FWD_SCALE, nullptr, s))) return st;
    const long long nc = (long long)gd.d * gd.Ms;
    if (pr == 1) {
        HG_CU(launch_convert_spectrum(w.S, 1, (double*)g->work[0].S, nc, s));
        c->launches++;
    }
    HG_CU(cudaMemcpyAsync(S_out, g->work[0].S, (size_t)nc * 2 * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    HG_CU(cudaStreamSynchronize(s));
    return HG_OK;
}

int hg_num_passes(hg_grid* g) { return g ? (g->gd.d == 2 ? 3 : 5) : -1; }

int hg_num_iter_passes(hg_grid* g, const hg_solve_opts* opts) {
    if (!g) return HG_ERR_ARG;
    hg_solve_opts o;
    if (opts) o = *opts; else hg_default_opts(&o);
    // the conditions of plane_path() that a solve's options decide (the
    // reduction slots always hold a plane launch's CTAs)
    const bool plane = o.prec == HG_MIXED && o.resident != 0 && o.A0[0] == 0.0 && plane_supported(g->gd);
    return plane ? 3 : hg_num_passes(g);
}

int hg_time_pass(hg_grid* g, int prec, int pass, int reps, double* ms_out, char* name_out) {
    if (!g || !ms_out || reps < 1 || (prec != HG_FP64 && prec != HG_MIXED)) return HG_ERR_ARG;
    const int np = hg_num_passes(g);
    if (pass < 0 || pass >= np) return HG_ERR_ARG;
    if (g->coeff_mode < 0) return HG_ERR_NO_COEFFS;
    if (g->borrowed.load() > 0) return HG_ERR_BUSY;
    hg_ctx* c = g->ctx;
    DeviceGuard dg(c->device);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    cudaStream_t s = c->stream;
    const int pr = prec == HG_MIXED ? 1 : 0;
    int st;
    if ((st = timing_state(g, pr, s))) return st;
    char nm[64] = {0};
    if ((st = enqueue_timing_pass(g, pr, pass, nm, s))) return st;   // warm-up
    HG_CU(cudaEventRecord(g->ev0, s));
    for (int i = 0; i < reps; ++i)
        if ((st = enqueue_timing_pass(g, pr, pass, nullptr, s))) return st;
    HG_CU(cudaEventRecord(g->ev1, s));
    HG_CU(cudaEventSynchronize(g->ev1));
    float ms = 0.f;
    HG_CU(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    *ms_out = (double)ms / reps;
    if (name_out) { strncpy(name_out, nm, 63); name_out[63] = 0; }
    return HG_OK;
}

int hg_submit(hg_ctx* c, hg_grid* g, const hg_solve_opts* opts, uint64_t* ticket) {
    if (!c || !g || !ticket || g->ctx != c) return HG_ERR_ARG;
    return sched_submit(c->sched, g, opts, ticket);
}

int hg_poll(hg_ctx* c, uint64_t ticket, hg_result* out, int timeout_us) {
    if (!c) return HG_ERR_ARG;
    return sched_poll(c->sched, ticket, out, timeout_us);
}

int hg_cancel(hg_ctx* c, uint64_t ticket) {
    if (!c) return HG_ERR_ARG;
    return sched_cancel(c->sched, ticket);
}

}  // extern "C"
