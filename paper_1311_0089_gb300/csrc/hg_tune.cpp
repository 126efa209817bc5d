// Launch geometry of the CG passes and its autotuner (hg_get_launch_cfg,
// hg_set_launch_cfg, hg_tune, hg_tune_cache_find).
//
// A pass's geometry is how it tiles the grid over CTAs: the last-axis passes
// stage RB grid rows of LB loads per CTA, a strided pass stages Cl pencils per
// component.  Every geometry the kernels can run gives the same iterates up
// to the rounding of the reductions' partial sums (the CTA partials change,
// the final sums stay FP64 in a fixed order).  The library's default is a
// heuristic (hg_api.cpp: most loads per CTA, then the most rows that keep two
// CTAs per SM); the tuner times the alternatives on the device and keeps the
// fastest, per device, grid shape and precision, optionally cached on disk.
#include "hg.h"
#include "hg_internal.h"
#include "hg_runtime.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
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

constexpr const char* CACHE_TAG = "hg-tune-v2";

// Axes whose FFT plan is read at run time (no compile-time kernel): only
// their radix order is a tunable.
bool runtime_axis(const hg_grid* g, int a) { return !ct_length(g->gd.d, g->gd.N[a]); }

hg_launch_cfg cfg_of(const hg_grid* g, int pr) {
    hg_launch_cfg c;
    memset(&c, 0, sizeof(c));
    c.row_rb = g->rowcfg[pr].RB;
    c.row_lb = g->rowcfg[pr].LB;
    for (int a = 0; a < g->gd.d - 1 && a < 2; ++a) c.lanes[a] = g->strcfg[pr][a].Cl;
    for (int a = 0; a < g->gd.d; ++a)
        if (runtime_axis(g, a))
            for (int k = 0; k < g->plan[a].nstages && k < 8; ++k) c.radix[a][k] = g->plan[a].radix[k];
    return c;
}

bool same_cfg(const hg_launch_cfg& a, const hg_launch_cfg& b) {
    return a.row_rb == b.row_rb && a.row_lb == b.row_lb && a.lanes[0] == b.lanes[0] && a.lanes[1] == b.lanes[1] &&
           memcmp(a.radix, b.radix, sizeof(a.radix)) == 0;
}

// The plan of axis a with the radix order `order` (zero-terminated; all zero:
// the default order), if it is one: a permutation of the length's factors,
// and only for an axis whose plan is read at run time.
bool plan_with_order(const hg_grid* g, int a, const int* order, AxisPlanH& out) {
    AxisPlanH pl{};
    if (!factor(g->gd.N[a], pl)) return false;
    pl.tw_off = g->plan[a].tw_off;
    if (order[0] == 0) {
        out = pl;
        return true;
    }
    if (!runtime_axis(g, a)) return false;
    int n = 0;
    while (n < 8 && order[n] != 0) ++n;
    if (n != pl.nstages) return false;
    for (int r : {3, 5, 7}) {   // the same multiset of radices
        int want = 0, have = 0;
        for (int k = 0; k < n; ++k) {
            want += order[k] == r;
            have += pl.radix[k] == r;
        }
        if (want != have) return false;
    }
    for (int k = 0; k < n; ++k) pl.radix[k] = order[k];
    out = pl;
    return true;
}

size_t csize_of(int pr) { return pr == 0 ? 16 : 8; }

// Row geometry (RB, LB) of grid g and precision pr, if the kernels can run it.
bool row_cfg(const hg_grid* g, int pr, int RB, int LB, RowCfg& out) {
    const GridDev& gd = g->gd;
    const int last = gd.d - 1;
    return make_row_cfg(pr, gd.Nl, gd.d, gd.d, RB, LB, min_radix(g->plan[last]), csize_of(pr), g->ctx->max_smem,
                        gd.rows, out);
}

// Strided geometry (Cl lanes) of axis a.
bool str_cfg(const hg_grid* g, int pr, int a, int Cl, StrCfg& out) {
    const GridDev& gd = g->gd;
    const long long inner = (a == 0) ? gd.Ms / gd.N[0] : gd.H;
    return make_str_cfg(pr, gd.N[a], gd.d, Cl, min_radix(g->plan[a]), csize_of(pr), g->ctx->max_smem, inner, out);
}

void drop_graphs(hg_grid* g) {
    for (int pr = 0; pr < 2; ++pr) {
        if (g->graphs[pr].exec) cudaGraphExecDestroy(g->graphs[pr].exec);
        g->graphs[pr] = GraphCache();
    }
}

// Validates c for g and sets it (caller holds ctx->mu, no work of g in flight).
int apply_cfg(hg_grid* g, int pr, const hg_launch_cfg& c) {
    RowCfg rc{};
    StrCfg sc[2]{};
    AxisPlanH pl[3]{};
    const int d = g->gd.d;
    for (int a = 0; a < 3; ++a) {
        if (a < d) {
            if (!plan_with_order(g, a, c.radix[a], pl[a])) return HG_ERR_ARG;
        } else if (c.radix[a][0] != 0) {
            return HG_ERR_ARG;
        }
    }
    // the tiles' limits depend on the smallest radix only, not on the order
    if (!row_cfg(g, pr, c.row_rb, c.row_lb, rc)) return HG_ERR_ARG;
    const int nstr = d - 1;
    for (int a = 0; a < 2; ++a) {
        if (a < nstr) {
            if (!str_cfg(g, pr, a, c.lanes[a], sc[a])) return HG_ERR_ARG;
        } else if (c.lanes[a] != 0) {
            return HG_ERR_ARG;
        }
    }
    int st;
    // every pass of either precision writes its CTA partials into the same slots
    const long long nbx = std::max(rc.nbx, g->rowcfg[1 - pr].nbx);
    if ((st = grid_ensure_partial(g, nbx))) return st;
    g->rowcfg[pr] = rc;
    for (int a = 0; a < nstr; ++a) g->strcfg[pr][a] = sc[a];
    for (int a = 0; a < d; ++a) g->plan[a] = pl[a];
    drop_graphs(g);
    return HG_OK;
}

// Mean ms of one launch sequence of `passes` (reps repetitions, best of three
// trials) with the grid's current geometry; timing_state() must have run.
int time_passes(hg_grid* g, int pr, const std::vector<int>& passes, int reps, double* ms) {
    cudaStream_t s = g->ctx->stream;
    int st;
    for (int p : passes)
        if ((st = enqueue_timing_pass(g, pr, p, nullptr, s))) return st;   // warm-up
    double best = 1e30;
    for (int trial = 0; trial < 3; ++trial) {
        HG_CU(cudaEventRecord(g->ev0, s));
        for (int i = 0; i < reps; ++i)
            for (int p : passes)
                if ((st = enqueue_timing_pass(g, pr, p, nullptr, s))) return st;
        HG_CU(cudaEventRecord(g->ev1, s));
        HG_CU(cudaEventSynchronize(g->ev1));
        float t = 0.f;
        HG_CU(cudaEventElapsedTime(&t, g->ev0, g->ev1));
        best = std::min(best, (double)t / reps);
    }
    *ms = best;
    return HG_OK;
}

std::string device_key(int device, int* sms) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        *sms = 0;
        return "unknown";
    }
    *sms = prop.multiProcessorCount;
    std::string n(prop.name);
    for (char& ch : n)
        if (ch == ' ' || ch == '\t') ch = '_';
    return n;
}

// Radix order <-> digit string ("357"; "0" for none).
void order_to_str(const int* order, char* out) {
    int n = 0;
    while (n < 8 && order[n] != 0) {
        out[n] = (char)('0' + order[n]);
        ++n;
    }
    if (n == 0) out[n++] = '0';
    out[n] = 0;
}

bool order_from_str(const char* str, int* order) {
    for (int k = 0; k < 8; ++k) order[k] = 0;
    if (strcmp(str, "0") == 0) return true;
    int n = 0;
    for (; str[n]; ++n) {
        if (n >= 8 || (str[n] != '3' && str[n] != '5' && str[n] != '7')) return false;
        order[n] = str[n] - '0';
    }
    return n > 0;
}

int cache_find(const char* path, const std::string& dev, int sms, int pr, int d, const int* N, hg_launch_cfg* out,
               double* ms_out) {
    FILE* f = fopen(path, "r");
    if (!f) return HG_ERR_ARG;
    char line[512];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        char tag[32], name[256], o[3][16];
        int s_sms, s_pr, s_d, n0, n1, n2, rb, lb, l0, l1;
        double ms;
        if (sscanf(line, "%31s %255s %d %d %d %d %d %d %d %d %d %d %lf %15s %15s %15s", tag, name, &s_sms, &s_pr,
                   &s_d, &n0, &n1, &n2, &rb, &lb, &l0, &l1, &ms, o[0], o[1], o[2]) != 16)
            continue;
        if (strcmp(tag, CACHE_TAG) != 0 || dev != name || s_sms != sms || s_pr != pr || s_d != d) continue;
        if (n0 != N[0] || n1 != N[1] || n2 != (d == 3 ? N[2] : 0)) continue;
        hg_launch_cfg c;
        memset(&c, 0, sizeof(c));
        bool ok = true;
        for (int a = 0; a < 3; ++a) ok = ok && order_from_str(o[a], c.radix[a]);
        if (!ok) continue;
        c.row_rb = rb;
        c.row_lb = lb;
        c.lanes[0] = l0;
        c.lanes[1] = l1;
        *out = c;
        if (ms_out) *ms_out = ms;
        found = true;   // later records override earlier ones
    }
    fclose(f);
    return found ? HG_OK : HG_ERR_ARG;
}

void cache_append(const char* path, const std::string& dev, int sms, int pr, int d, const int* N,
                  const hg_launch_cfg& c, double ms) {
    FILE* f = fopen(path, "a");
    if (!f) return;   // a cache that cannot be written only costs a re-tune
    char o[3][16];
    for (int a = 0; a < 3; ++a) order_to_str(c.radix[a], o[a]);
    fprintf(f, "%s %s %d %d %d %d %d %d %d %d %d %d %.6f %s %s %s\n", CACHE_TAG, dev.c_str(), sms, pr, d, N[0],
            N[1], d == 3 ? N[2] : 0, c.row_rb, c.row_lb, c.lanes[0], c.lanes[1], ms, o[0], o[1], o[2]);
    fclose(f);
}

int check_grid(hg_grid* g, int prec) {
    if (!g || (prec != HG_FP64 && prec != HG_MIXED)) return HG_ERR_ARG;
    if (g->borrowed.load() > 0) return HG_ERR_BUSY;
    return HG_OK;
}

}  // namespace

extern "C" {

int hg_get_launch_cfg(hg_grid* g, int prec, hg_launch_cfg* out) {
    if (!g || !out || (prec != HG_FP64 && prec != HG_MIXED)) return HG_ERR_ARG;
    std::lock_guard<std::recursive_mutex> lk(g->ctx->mu);
    *out = cfg_of(g, prec == HG_MIXED ? 1 : 0);
    return HG_OK;
}

int hg_set_launch_cfg(hg_grid* g, int prec, const hg_launch_cfg* cfg) {
    int st = check_grid(g, prec);
    if (st) return st;
    if (!cfg) return HG_ERR_ARG;
    hg_ctx* c = g->ctx;
    cudaSetDevice(c->device);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    if (g->borrowed.load() > 0) return HG_ERR_BUSY;
    HG_CU(cudaStreamSynchronize(c->stream));
    return apply_cfg(g, prec == HG_MIXED ? 1 : 0, *cfg);
}

int hg_tune_cache_find(const char* path, const char* device_name, int sm_count, int prec, int d, const int* N,
                       hg_launch_cfg* out, double* ms_out) {
    if (!path || !device_name || !N || !out || (d != 2 && d != 3) || (prec != HG_FP64 && prec != HG_MIXED))
        return HG_ERR_ARG;
    return cache_find(path, device_name, sm_count, prec == HG_MIXED ? 1 : 0, d, N, out, ms_out);
}

int hg_tune(hg_grid* g, int prec, int reps, const char* cache_path, hg_tune_result* out) {
    int st = check_grid(g, prec);
    if (st) return st;
    if (reps < 1) return HG_ERR_ARG;
    if (g->coeff_mode < 0) return HG_ERR_NO_COEFFS;
    hg_ctx* c = g->ctx;
    cudaSetDevice(c->device);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    if (g->borrowed.load() > 0) return HG_ERR_BUSY;
    const int pr = prec == HG_MIXED ? 1 : 0;
    const GridDev& gd = g->gd;
    const int d = gd.d, np = d == 2 ? 3 : 5;
    hg_tune_result res;
    memset(&res, 0, sizeof(res));
    HG_CU(cudaStreamSynchronize(c->stream));

    // the library's default for this grid (the geometry set at creation may
    // have been replaced by an earlier hg_set_launch_cfg or hg_tune)
    hg_launch_cfg heur;
    memset(&heur, 0, sizeof(heur));
    {
        RowCfg rc{};
        if (!choose_row_cfg(pr, gd.Nl, d, d, min_radix(g->plan[d - 1]), csize_of(pr), c->max_smem, gd.rows, rc))
            return HG_ERR_UNSUPPORTED_SIZE;
        heur.row_rb = rc.RB;
        heur.row_lb = rc.LB;
        for (int a = 0; a < d - 1; ++a) {
            StrCfg sc{};
            const long long inner = (a == 0) ? gd.Ms / gd.N[0] : gd.H;
            const long long outer = (a == 0) ? 1 : gd.N[0];
            if (!choose_str_cfg(pr, gd.N[a], d, min_radix(g->plan[a]), csize_of(pr), c->max_smem, inner, outer, d, sc))
                return HG_ERR_UNSUPPORTED_SIZE;
            heur.lanes[a] = sc.Cl;
        }
        for (int a = 0; a < d; ++a) {
            AxisPlanH pl{};
            if (runtime_axis(g, a) && factor(gd.N[a], pl))
                for (int k = 0; k < pl.nstages && k < 8; ++k) heur.radix[a][k] = pl.radix[k];
        }
    }
    res.heuristic = heur;

    int sms = 0;
    const std::string dev = device_key(c->device, &sms);
    if (cache_path) {
        hg_launch_cfg cached;
        double ms = 0.0;
        if (cache_find(cache_path, dev, sms, pr, d, gd.N, &cached, &ms) == HG_OK &&
            apply_cfg(g, pr, cached) == HG_OK) {
            res.chosen = cached;
            res.ms_chosen = ms;
            res.from_cache = 1;
            if (out) *out = res;
            return HG_OK;
        }
    }

    if ((st = timing_state(g, pr, c->stream))) return st;
    if ((st = apply_cfg(g, pr, heur))) return st;
    hg_launch_cfg best = heur;

    // last-axis passes: every (RB, LB) tile the kernels can run
    {
        const std::vector<int> passes = {0, np - 1};
        double t_heur = 0.0;
        if ((st = time_passes(g, pr, passes, reps, &t_heur))) return st;
        double t_best = t_heur;
        ++res.candidates;
        for (int LB = d; LB >= 1; --LB) {
            for (int RB = 1; RB <= MAX_REAL_ROWS_HOST; ++RB) {
                RowCfg rc{};
                if (!row_cfg(g, pr, RB, LB, rc)) break;
                if (RB == heur.row_rb && LB == heur.row_lb) continue;
                hg_launch_cfg cand = best;
                cand.row_rb = RB;
                cand.row_lb = LB;
                if ((st = apply_cfg(g, pr, cand))) return st;
                double t = 0.0;
                if ((st = time_passes(g, pr, passes, reps, &t))) return st;
                ++res.candidates;
                if (t < t_best && t < 0.97 * t_heur) {
                    t_best = t;
                    best.row_rb = RB;
                    best.row_lb = LB;
                }
            }
        }
        if ((st = apply_cfg(g, pr, best))) return st;
    }
    // strided passes, one axis at a time (axis 0: the projection pass; axis 1
    // in 3D: its forward and inverse passes)
    for (int a = 0; a < d - 1; ++a) {
        std::vector<int> passes;
        if (d == 2) passes = {1};
        else if (a == 0) passes = {2};
        else passes = {1, 3};
        double t_heur = 0.0;
        if ((st = time_passes(g, pr, passes, reps, &t_heur))) return st;
        double t_best = t_heur;
        ++res.candidates;
        const int heur_cl = best.lanes[a];
        for (int Cl = 1; Cl <= 32; Cl *= 2) {
            StrCfg sc{};
            if (!str_cfg(g, pr, a, Cl, sc)) break;
            if (Cl == heur_cl) continue;
            hg_launch_cfg cand = best;
            cand.lanes[a] = Cl;
            if ((st = apply_cfg(g, pr, cand))) return st;
            double t = 0.0;
            if ((st = time_passes(g, pr, passes, reps, &t))) return st;
            ++res.candidates;
            if (t < t_best && t < 0.97 * t_heur) {
                t_best = t;
                best.lanes[a] = Cl;
            }
        }
        if ((st = apply_cfg(g, pr, best))) return st;
    }

    // radix order of every axis whose plan is read at run time: each distinct
    // permutation of its factors (the default order, ascending, first)
    for (int a = 0; a < d; ++a) {
        if (!runtime_axis(g, a) || heur.radix[a][1] == 0) continue;   // one stage: no choice
        std::vector<int> passes;
        if (a == d - 1) passes = {0, np - 1};
        else if (a == 0) passes = {d == 2 ? 1 : 2};
        else passes = {1, 3};
        double t_heur = 0.0;
        if ((st = time_passes(g, pr, passes, reps, &t_heur))) return st;
        double t_best = t_heur;
        ++res.candidates;
        int order[8] = {0}, n = 0;
        while (n < 8 && heur.radix[a][n] != 0) {
            order[n] = heur.radix[a][n];
            ++n;
        }
        int tried = 0;
        while (std::next_permutation(order, order + n) && ++tried <= 24) {
            hg_launch_cfg cand = best;
            for (int k = 0; k < 8; ++k) cand.radix[a][k] = order[k];
            if ((st = apply_cfg(g, pr, cand))) return st;
            double t = 0.0;
            if ((st = time_passes(g, pr, passes, reps, &t))) return st;
            ++res.candidates;
            if (t < t_best && t < 0.97 * t_heur) {
                t_best = t;
                best = cand;
            }
        }
        if ((st = apply_cfg(g, pr, best))) return st;
    }

    // one whole iteration with the default and with the chosen geometry
    std::vector<int> all;
    for (int p = 0; p < np; ++p) all.push_back(p);
    if ((st = apply_cfg(g, pr, heur))) return st;
    if ((st = time_passes(g, pr, all, reps, &res.ms_heuristic))) return st;
    if ((st = apply_cfg(g, pr, best))) return st;
    if (!same_cfg(best, heur)) {
        if ((st = time_passes(g, pr, all, reps, &res.ms_chosen))) return st;
        // the passes were tuned one group at a time: keep the combination only
        // if the whole iteration is faster too
        if (!(res.ms_chosen < res.ms_heuristic)) {
            best = heur;
            res.ms_chosen = res.ms_heuristic;
            if ((st = apply_cfg(g, pr, best))) return st;
        }
    } else {
        res.ms_chosen = res.ms_heuristic;
    }
    res.chosen = best;
    if (cache_path) cache_append(cache_path, dev, sms, pr, d, gd.N, best, res.ms_chosen);
    if (out) *out = res;
    return HG_OK;
}

}  // extern "C"
