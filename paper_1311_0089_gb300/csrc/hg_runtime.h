// Host-side objects behind the opaque hg_ctx / hg_grid handles.
#pragma once
#include "hg.h"
#include "hg_internal.h"

#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <thread>
#include <unordered_map>
#include <vector>

namespace hgrt {
struct Scheduler;
}

struct hg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // private, always idle: CUDA graph capture
    bool own_stream = false;
    size_t budget = 0;
    std::atomic<size_t> used{0};
    std::map<void*, size_t> alloc_sizes;
    std::atomic<long long> launches{0};
    std::atomic<int> ngrids{0};         // live grids (hg_destroy refuses while > 0)
    std::set<hg_grid*> grids;           // live grids (guarded by mu)
    int max_smem = 48 * 1024;
    int nsm = 1;                        // streaming multiprocessors of the device
    std::recursive_mutex mu;            // serialises device work issued by callers
    hgrt::Scheduler* sched = nullptr;   // request scheduler (hg_submit / hg_poll)
};

namespace hgrt {

constexpr int MAX_PROF_CHUNK = 64;   // iterations per graph when a pass is timed

struct Work {
    void* x = nullptr;
    void* r = nullptr;
    void* p = nullptr;
    void* S = nullptr;
    hgk::Scalars* sc = nullptr;
    bool ready = false;
};

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    int chunk = 0;
    int nkern = 0;
    int prof_pass = -1;   // pass bracketed by event records (-1: none)
    int form = 0;         // formulation captured (coefficients and projection)
    int plane = 0;        // 3D plane passes captured
    int has_ref = 0;      // general reference medium captured, and its value
    double ref[9] = {0};
};

}  // namespace hgrt

struct hg_grid {
    hg_ctx* ctx = nullptr;
    hgk::GridDev gd{};
    hgk::AxisPlanH plan[3]{};
    hgk::RowCfg rowcfg[2]{};
    hgk::StrCfg strcfg[2][3]{};
    void* tw[2] = {nullptr, nullptr};
    // coefficients
    int coeff_mode = -1;          // -1 none, 0 phase, 1 packed field
    int n_phases = 0;
    uint8_t* d_phase = nullptr;
    void* d_table[2] = {nullptr, nullptr};
    void* d_field[2] = {nullptr, nullptr};
    // Galerkin scheme with exact integration: this grid is the quadrature grid
    // and band the trial space Z_N (0: GaNi on this grid)
    int band[3] = {0, 0, 0};
    bool exact = false;
    // inverse coefficients A^-1 for the dual formulation (made on first use)
    void* d_table_inv[2] = {nullptr, nullptr};
    void* d_field_inv[2] = {nullptr, nullptr};
    bool inv_ok = false;
    // formulation the next enqueued work uses: 0 primal, 1 dual (coefficients
    // A^-1 and the projection onto J_N); set by every entry point that enqueues
    int form = 0;
    // the FP32 CG iterations of the next enqueued work may run as the 3D plane
    // passes (hg_plane.cu) where the grid allows them; set like `form`
    bool use_plane = true;
    // general reference medium A0 of the next enqueued CG work (0: A0 = I); set
    // like `form`
    int has_ref = 0;
    double ref[9] = {0};
    // eigenvalue bounds c_A, C_A of the coefficients of each formulation
    // (Moulinec-Suquet)
    bool bounds_ok[2] = {false, false};
    double c_A[2] = {0.0, 0.0}, C_A[2] = {0.0, 0.0};
    // solver state
    hgrt::Work work[2];
    double* partial = nullptr;
    long long partial_slots = 0;
    unsigned* counters = nullptr;
    double* d_AH = nullptr;        // 32 doubles: [0, 18) A_H forms, [24, 26) bounds
    double* d_E = nullptr;
    double* d_A0 = nullptr;
    hgk::Scalars* d_sc_aux = nullptr;   // FP64 true residual at exit (scratch scalars)
    hgk::Scalars* h_sc = nullptr;  // pinned: scalars of the last tick [MAXL], then the
                                   // true-residual scalars [MAXL]
    double* h_AH = nullptr;        // pinned: 2 d x d (energy, flux)
    hgrt::GraphCache graphs[2];
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_tick = nullptr;
    cudaEvent_t prof_ev[2 * hgrt::MAX_PROF_CHUNK] = {};   // per-iteration pass brackets
    int last_prec = 0;
    bool counted = false;
    std::atomic<int> borrowed{0};
};

namespace hgrt {
void set_last_cuda_error(cudaError_t e, const char* what);
const char* last_cuda_error();
int dev_alloc(hg_ctx* ctx, void** p, size_t bytes);
void dev_free(hg_ctx* ctx, void* p);
int grid_init_plans(hg_grid* g);
// FFT plan and launch geometry helpers (hg_api.cpp)
bool factor(int n, hgk::AxisPlanH& pl);
int min_radix(const hgk::AxisPlanH& pl);
// make_*: the geometry with the given tile, if the kernels can run it;
// choose_*: the default (heuristic) geometry.
bool make_row_cfg(int prec, int n, int d, int L, int RB, int LB, int minR, size_t csize, int max_smem,
                  long long rows, hgk::RowCfg& cfg);
bool make_str_cfg(int prec, int n, int d, int Cl, int minR, size_t csize, int max_smem, long long inner,
                  hgk::StrCfg& cfg);
bool choose_row_cfg(int prec, int n, int d, int L, int minR, size_t csize, int max_smem,
                    long long rows, hgk::RowCfg& cfg);
bool choose_str_cfg(int prec, int n, int d, int minR, size_t csize, int max_smem,
                    long long inner, long long outer, int L, hgk::StrCfg& cfg);
int grid_alloc_work(hg_grid* g, int prec);
size_t solve_bytes_needed(const hg_grid* g, int prec, long long nbx = 0);
int grid_alloc_common(hg_grid* g);
hgk::CoeffsDev coeffs_for(const hg_grid* g, int prec, bool withA);
int enqueue_forward_strided(hg_grid* g, int prec, int L, int check_status, int gamma_mode,
                            const double* A0, cudaStream_t s, hgk::Scalars* status_sc = nullptr);
// The arguments of one operator application on one grid (d + 1 launches): the
// last-axis forward pass, the strided passes in launch order, the last-axis
// inverse pass.
struct PassArgs {
    hgk::RowFwdArgs fa;
    hgk::StrArgs sa[3];
    int nstr = 0;
    hgk::RowInvArgs ia;
    int plane = 0;      // 1: fa / ia run as the 3D plane passes, sa[0] is the axis-0 pass
};
void cg_iteration_args(hg_grid* g, int prec, int L, PassArgs* pa);
void matvec_args(hg_grid* g, int prec, int L, const void* u, bool unit_loads, bool withA,
                 const double* A0dev, const double* A0host, int inv_mode, void* out, int check_status,
                 hgk::Scalars* status_sc, PassArgs* pa);
int enqueue_cg_iteration(hg_grid* g, int prec, int L, cudaStream_t s, int prof_pass = -1,
                         cudaEvent_t ev_before = nullptr, cudaEvent_t ev_after = nullptr);
int enqueue_matvec(hg_grid* g, int prec, int L, const void* u, bool unit_loads, bool withA,
                   const double* A0dev, const double* A0host, int inv_mode, void* out,
                   int check_status, cudaStream_t s, hgk::Scalars* status_sc = nullptr);
int get_cg_graph(hg_grid* g, int prec, int chunk, cudaGraphExec_t* out, int* nkern, int prof_pass = -1);

// One solve as a resumable state machine: job_begin enqueues the first
// steps; each time the job's tick event has completed, job_advance reads the
// copied scalars and enqueues the next steps, until *done.
struct Job {
    enum Phase { PLAIN = 0, INNER = 1, RESID = 2, FINAL = 3, DONE = 4 };
    hg_grid* g = nullptr;
    hg_solve_opts o{};
    cudaStream_t s = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, tick = nullptr;
    int prec = 0, cg_prec = 0, phase = PLAIN, outer = 0, chunk = 8, result = 0;
    long long launched = 0, launches0 = 0;
    double t0 = 0.0;
    hg_result res{};
    double fixed_alpha = 0.0;   // Moulinec-Suquet: 1 / lambda (0: CG)
    double zscale = 1.0;        // scale of the zero right-hand-side test
    double lambda = 0.0;
    int stall_max = 64;         // inner FP32 solves: iterations without a 4x drop
    bool allow_resident = false;   // inner FP32 solves may run the resident kernel
    int res_ctas = 0;           // CTAs of the last resident launch (0: none)
    int res_drop_cta = -1;      // >= 1: that CTA of the resident launch leaves at once, so
                                // the others' bounded barrier waits run out (error-path test)
    int prof_prev_iters = 0;    // time_pass: iterations done before the chunk in flight
    double prof_ms = 0.0;
    int prof_n = 0;
};
int job_begin(Job& j);
int job_advance(Job& j, bool* done);
void grid_free_work(hg_grid* g);
// Frees the solver state of every grid of ctx that no ticket holds (except
// `keep`); returns the bytes released.  Caller holds ctx->mu.
size_t ctx_reclaim(hg_ctx* ctx, hg_grid* keep);
int solve_impl(hg_grid* g, const hg_solve_opts* o, double* AH_out, hg_result* info, int res_drop_cta = -1);
int validate_solve_opts(const hg_grid* g, hg_solve_opts* o);
int ga_build_field(hg_grid* g, const int* Ntr, const int* P, const uint8_t* phase, const double* table,
                   double* out64, float* out32, cudaStream_t s);
hgk::Weight grid_weight(const hg_grid* g);   // the scalar product of the iteration
// Single-pass timing (hg_time_pass, hg_tune): buffers and steady-state
// scalars, then one launch of pass `pass` with the grid's launch geometry.
int timing_state(hg_grid* g, int pr, cudaStream_t s);
int enqueue_timing_pass(hg_grid* g, int pr, int pass, char* nm, cudaStream_t s);
// Reduction slots for row passes of nbx CTAs per load (reallocated when the
// current buffer is smaller; the caller holds ctx->mu with no work in flight).
int grid_ensure_partial(hg_grid* g, long long nbx);

// Rolling batch (hg_batch.cpp): the scheduler's cross-request batching.
// Requests of one precision step together, check_every CG iterations per
// chunk, one batched launch per pass and grid shape for all of them; members
// join and leave between ticks.
struct Rolling;
struct RollDone {
    uint64_t tag;
    int status;
    hg_result res;
};
Rolling* rolling_create(hg_ctx* ctx, int prec, int chunk);
void rolling_destroy(Rolling* R);
int rolling_chunk(const Rolling* R);
// Members plus chunks not read yet and results not returned yet (0: idle).
int rolling_size(const Rolling* R);
// Row-pass CTAs of the shape's batched launches (reduction slots a member needs).
long long rolling_nbx(Rolling* R, const hg_grid* g);
// Admits g (standard CG, primal, A0 = I, R's precision): allocates its solver
// state and enqueues its right-hand side.  HG_ERR_NO_MEMORY leaves nothing
// allocated beyond what the grid already held.
int rolling_add(Rolling* R, hg_grid* g, const hg_solve_opts& o, uint64_t tag);
// One tick: enqueues the next chunk (check_every iterations of every member),
// reads the scalars of the chunk before it and enqueues the refinement steps
// and A_H they call for; appends to *done the results whose copies have
// completed (waits for them once no member is left).
int rolling_tick(Rolling* R, std::vector<RollDone>* done);
// Drops a member (cancellation); waits for the batch's streams first.
void rolling_remove(Rolling* R, uint64_t tag);

// scheduler (hg_sched.cpp)
Scheduler* sched_create(hg_ctx* ctx);
void sched_destroy(Scheduler* s);
int sched_submit(Scheduler* s, hg_grid* g, const hg_solve_opts* o, uint64_t* ticket);
int sched_poll(Scheduler* s, uint64_t ticket, hg_result* out, int timeout_us);
int sched_cancel(Scheduler* s, uint64_t ticket);
}  // namespace hgrt
