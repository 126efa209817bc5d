// Internal interface between the host runtime (hg_api.cpp) and the CUDA
// kernels (hg_kernels.cu).  Plain structs and pointers only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hgk {

enum { MAXD = 3, MAXL = 3 };

// Composite codelet twiddle table layout (W_R^m for R = 9, 15, 25, 27).
enum { CTW_9 = 0, CTW_15 = 9, CTW_25 = 24, CTW_27 = 49, CTW_TOTAL = 76 };

// Status of one CG system on the device.
enum {
    ST_ACTIVE = 0,
    ST_CONVERGED = 1,
    ST_ZERO_RHS = 2,
    ST_MAXITER = 3,
    ST_BREAKDOWN = 4,
    ST_IDLE = 5,       // not part of this solve (load not requested)
    ST_STAGNATED = 6,  // inner FP32 solve stopped improving (refinement goes on)
    ST_RHS_RECHECK = 7, // FP32 right-hand side too small to tell from zero: the
                        // solve recomputes it in FP64
    ST_TIMEOUT = 8      // a bounded device-side wait (grid barrier of the
                        // resident solver) gave up
};

// Per-system CG scalars kept on the device (written by the last CTA of a
// reduction, read by the following kernels).
struct Scalars {
    double rr;       // (r, r) of the current residual
    double pt;       // (p, A p)
    double alpha;    // rr / pt
    double beta;     // rr_new / rr_old (0 before the first step)
    double bnorm;    // ||b|| of this system
    double aen;      // ||A E|| (zero right-hand-side test)
    double relres;   // last ||r|| / ||b||
    double tol;      // stopping tolerance of this system
    int iters;
    int status;
    int max_iter;
    int total_iters; // accumulated over refinement steps
    float alpha_f;   // alpha and beta rounded to FP32 for the FP32 kernels
    float beta_f;
    double best_rr;  // stagnation test (inner FP32 solves): best (r, r) so far
    int stall;       // iterations since best_rr last fell by 4x
    int stall_max;   // > 0: stop (ST_STAGNATED) after this many such iterations
    double fixed_alpha;  // > 0: Moulinec-Suquet step 1/lambda in place of CG's
                         // alpha, beta = 0, stop on the step just taken
    double zscale;       // zero right-hand-side test: ||b|| <= ZERO_RHS zscale ||A E||
                         // (sqrt(lmax(A0)) / lmin(A0) for a general reference medium)
};

// Scalar product of the iteration: (W u, v) with a constant SPD d x d W
// (the reference medium A0), or the plain one when has = 0.
struct Weight {
    int has;
    double w[9];
    float wf[9];
};

struct GridDev {
    int d;                 // dimension (2 or 3)
    int N[3];              // axis lengths
    int Nl;                // last axis length
    int H;                 // (Nl + 1) / 2
    long long M;           // |N|
    long long rows;        // M / Nl
    long long Ms;          // rows * H (complex half-spectrum entries per component)
    double Y[3];           // cell half sizes
    double invY[3];        // 1 / Y
    double invM;
    float invYf[3];        // FP32 copies for the FP32 kernels
    float invMf;
};

struct AxisPlanH {
    int n;
    int nstages;
    int radix[16];
    int tw_off;
};

struct CoeffsDev {
    int mode;                  // 0 phase map, 1 packed field, 2 identity
    int n_phases;              // mode 0: table entries (<= 16 are staged in shared memory)
    const uint8_t* phase;
    const void* table;         // n_phases x d x d (T)
    const void* field;         // npk x M (T), order 11,22[,33],12[,13,23]
};

// Row (last-axis) pass launch geometry.
// ct = 1: the compile-time kernel for this length is used (256 threads).
struct RowCfg { int RB; int LB; int threads; int smem; long long nbx; int nby; int ct; };
// Strided-axis pass launch geometry.
struct StrCfg { int Cl; int threads; int smem; int ct; };

enum RowFwdMode { FWD_CG = 0, FWD_APPLY = 1 };
enum RowInvMode { INV_CG = 0, INV_RHS = 1, INV_OUT = 2, INV_RESID = 3, INV_PROJ = 4 };
enum StrMode { STR_FWD = 0, STR_INV = 1, STR_GAMMA = 2, STR_FWD_SCALE = 3 };

struct RowFwdArgs {
    int mode;
    int L;                      // systems in this launch (loads)
    CoeffsDev co;
    void* p;                    // FWD_CG: in/out search direction [L][d][M]
    const void* r;              // FWD_CG: residual
    const void* u;              // FWD_APPLY: input field [L][d][M] or null (= 0)
    int has_E;                  // FWD_APPLY: add the loads E (by value, both precisions)
    double Ed[MAXL * MAXD];     //   [L][d]
    float Ef[MAXL * MAXD];
    const double* A0;           // FWD_APPLY: d x d reference medium applied after A, or null
    void* S;                    // out: half spectra [L][d][rows][H]
    Scalars* sc;                // per system
    double* partial;            // reduction scratch [L][nbx]
    unsigned* counter;          // one counter, reset by the last CTA
    int check_status;           // skip systems that are not ACTIVE
    int early_stage;            // 1: twiddle/coefficient staging may precede the wait for
                                //    the previous kernel (tables written only by copies)
};

struct StrArgs {
    int mode;
    int L;
    int axis;
    long long outer, inner;
    int n;
    void* S;
    const Scalars* sc;
    int check_status;
    int has_A0;
    double A0[9];
    int early_stage;            // 1: twiddle/coefficient staging may precede the wait for
                                //    the previous kernel (tables written only by copies)
    int dual;                   // STR_GAMMA projects onto J_N (identity - mean - Gamma)
    int band[3];                // STR_GAMMA: > 0: keep only frequencies |m_a| <= (band_a - 1) / 2
                                // (the trial space of the Galerkin scheme with exact integration)
};

struct RowInvArgs {
    int mode;
    int L;
    const void* S;
    void* x;                    // INV_CG / INV_RHS
    void* r;                    // INV_CG / INV_RHS / INV_RESID
    void* p;                    // INV_CG (read) / INV_RHS (write)
    void* out;                  // INV_OUT
    Scalars* sc;
    double* partial;
    unsigned* counter;
    int check_status;
    int early_stage;            // 1: twiddle/coefficient staging may precede the wait for
                                //    the previous kernel (tables written only by copies)
    Weight W;                   // (r, r) of INV_CG / INV_RHS / INV_RESID in the product (W r, r)
};

// Resident FP32 CG solver for square 2D grids (hg_resident.cu): one
// cooperative launch runs every iteration of the inner FP32 solve, with r and
// p kept in the shared memory of a team of CTAs (one per SM) and grid-wide
// barriers between the row, column and row phases of each iteration.
struct ResArgs {
    GridDev g;
    CoeffsDev co;          // FP32 coefficients: mode 0 (phase map + table) or 1 (packed field)
    int L;                 // systems (loads)
    int units, cunits;     // row units N * L (grid row, load), column units H * L
    int umax, bufp;        // most row units of a CTA; pencils of the transform buffer
    const float* r0;       // initial residual [L][2][M]
    float* x;              // [L][2][M] solution of the inner system (zeroed by the kernel)
    float2* S;             // [L][2][N][H] half spectra (scratch)
    const float2* tw;      // W_N^m, m < N
    Scalars* sc;           // [L] inner scalars: read at start, written at exit
    double* part;          // [2][team][MAXL] CTA partial sums
    unsigned* bar;         // barrier counter, zero at launch
    int* err;              // zero at launch; set when a barrier wait gives up
    int dual, has_A0;
    float A0[4];
    int band[2];
    Weight W;
    int drop_cta;          // >= 0: that CTA leaves at once (exercises the bounded wait)
    unsigned long long wait_ns;   // limit of one barrier wait
};
struct ResCfg { int T; int umax; int bufp; int smem; };
// Whether square grids of side n have a resident kernel.
bool resident_length(int n);
// Team size and shared-memory layout for an n x n grid with L loads; T = 0
// picks the default.  False if the state does not fit on chip.
bool resident_cfg(int n, int L, int T, int nsm, int max_smem, ResCfg& cfg);
cudaError_t launch_resident(int n, const ResArgs& a, const ResCfg& cfg, cudaStream_t s);
cudaError_t configure_resident(int max_smem, const double* ctw);

// Plane passes of the FP32 CG iteration on N0 x N x N grids (hg_plane.cu):
// one CTA per (load, axis-0 plane, component), the axis-1 and axis-2
// transforms in shared memory; the spectrum in the pass kernels' layout.
bool plane_supported(const GridDev& g);
long long plane_units(const GridDev& g);        // CTAs per load (reduction slots)
cudaError_t launch_plane_fwd(const GridDev& g, const void* tw, const RowFwdArgs& a, cudaStream_t s);
cudaError_t launch_plane_inv(const GridDev& g, const void* tw, const RowInvArgs& a, cudaStream_t s);
cudaError_t launch_plane_fwd_batch(const GridDev& g, const void* tw, const RowFwdArgs* items, int P, int L,
                                   cudaStream_t s);
cudaError_t launch_plane_inv_batch(const GridDev& g, const void* tw, const RowInvArgs* items, int P, int L,
                                   cudaStream_t s);
cudaError_t configure_plane(const double* ctw);

// Launchers (prec: 0 = double, 1 = float).  Return cudaGetLastError().
cudaError_t launch_row_fwd(int prec, const GridDev& g, const AxisPlanH& pl, const void* tw,
                           const RowCfg& cfg, const RowFwdArgs& a, cudaStream_t s);
cudaError_t launch_strided(int prec, const GridDev& g, const AxisPlanH& pl, const void* tw,
                           const StrCfg& cfg, const StrArgs& a, cudaStream_t s);
cudaError_t launch_row_inv(int prec, const GridDev& g, const AxisPlanH& pl, const void* tw,
                           const RowCfg& cfg, const RowInvArgs& a, cudaStream_t s);
// Batched forms: P problems of the grid shape g, problem p's arguments at items[p]
// (device memory), L loads each.
cudaError_t launch_row_fwd_batch(int prec, const GridDev& g, const AxisPlanH& pl, const void* tw,
                                 const RowCfg& cfg, const RowFwdArgs* items, int P, int L, cudaStream_t s);
cudaError_t launch_row_inv_batch(int prec, const GridDev& g, const AxisPlanH& pl, const void* tw,
                                 const RowCfg& cfg, const RowInvArgs* items, int P, int L, cudaStream_t s);
cudaError_t launch_strided_batch(int prec, const GridDev& g, const AxisPlanH& pl, const void* tw,
                                 const StrCfg& cfg, const StrArgs* items, int P, int L, int n,
                                 long long inner, long long outer, cudaStream_t s);

// Small helpers.
// fixed_alpha > 0 selects the Moulinec-Suquet update with step fixed_alpha.
cudaError_t launch_init_scalars(Scalars* sc, int L, const int* status_init, double tol,
                                int max_iter, double fixed_alpha, double zscale, cudaStream_t s);
// Mixed precision: r32 = (float) r64, p32 = r32, x32 = 0, inner scalars from
// the outer status (and its fixed step); reduction of (r32, r32).  An inner
// solve stops (STAGNATED) after stall_max iterations without a 4x drop of (r, r).
// r64 = null: r32 = p32 = b and x32 = 0 were written by the FP32 right-hand
// side (INV_RHS) and the outer scalars hold (b, b); only the inner scalars are
// set (one block).
cudaError_t launch_inner_init(const GridDev& g, int L, const double* r64, float* r32, float* p32,
                              float* x32, const Scalars* outer, Scalars* inner, double inner_tol,
                              int inner_max, int stall_max, const Weight& W, double* partial,
                              unsigned* counter, cudaStream_t s);
// bounds[0] = min, bounds[1] = max over the voxels of the eigenvalues of A(x_k)
// (FP64 coefficients co64); both exact up to the eigenvalue formula's rounding
// and independent of the reduction order.
// A(x_k)^-1 of a packed symmetric FP64 field (component-major, order
// 11,22[,33],12[,13,23]) into the same layout, FP64 and FP32.
cudaError_t launch_invert_field(int d, long long M, const double* in, double* out64, float* out32,
                                cudaStream_t s);
// dst[p * MAXL + l] = src[p][l] for p < P (src: device array of P pointers).
cudaError_t launch_gather_scalars(const Scalars* const* src, Scalars* dst, int P, cudaStream_t s);
cudaError_t launch_coeff_bounds(const GridDev& g, const CoeffsDev& co64, double* bounds, cudaStream_t s);
// x64 += x32 for systems whose outer status is ACTIVE; inner iterations are
// added to the outer totals.
cudaError_t launch_outer_update(const GridDev& g, int L, double* x64, const float* x32,
                                Scalars* outer, const Scalars* inner, cudaStream_t s);
// Energy and flux forms of A_H from the FP64 fluctuations.
cudaError_t launch_energy(const GridDev& g, int L, const CoeffsDev& co64, const double* x,
                          unsigned loadmask, double* partial, unsigned* counter, double* out,
                          cudaStream_t s);
cudaError_t launch_convert(const void* src, int src_prec, void* dst, int dst_prec, long long n,
                           cudaStream_t s);
cudaError_t launch_convert_spectrum(const void* src, int src_prec, double* dst, long long ncomplex,
                                    cudaStream_t s);
int row_max_threads();
cudaError_t configure_kernels(int max_smem);
// Lengths with compile-time kernels (per dimension) and the pencils one CTA
// of such a kernel may stage (mirrors CtCaps in fft_device.cuh).
bool ct_length(int d, int n);
int ct_npmax(int prec, int n);
enum { CT_THREADS_HOST = 256 };   // = CT_THREADS
enum { MAX_REAL_ROWS_HOST = 64 };  // = MAX_REAL_ROWS: real rows one row-pass CTA stages
// Most lanes of a compile-time strided tile (the device bounds its per-thread
// loads by it; the host never chooses more).
__host__ __device__ constexpr int ct_max_lanes(int d) { return d == 2 ? 2 : 4; }

// per-precision launchers (hg_kernels_f32.cu, hg_kernels_f64.cu)
cudaError_t launch_row_fwd_f32(const GridDev&, const AxisPlanH&, const void*, const RowCfg&, const RowFwdArgs&, cudaStream_t);
cudaError_t launch_row_fwd_f64(const GridDev&, const AxisPlanH&, const void*, const RowCfg&, const RowFwdArgs&, cudaStream_t);
cudaError_t launch_row_inv_f32(const GridDev&, const AxisPlanH&, const void*, const RowCfg&, const RowInvArgs&, cudaStream_t);
cudaError_t launch_row_inv_f64(const GridDev&, const AxisPlanH&, const void*, const RowCfg&, const RowInvArgs&, cudaStream_t);
cudaError_t launch_strided_f32(const GridDev&, const AxisPlanH&, const void*, const StrCfg&, const StrArgs&, cudaStream_t);
cudaError_t launch_strided_f64(const GridDev&, const AxisPlanH&, const void*, const StrCfg&, const StrArgs&, cudaStream_t);
cudaError_t launch_row_fwd_batch_f32(const GridDev&, const AxisPlanH&, const void*, const RowCfg&, const RowFwdArgs*, int, int, cudaStream_t);
cudaError_t launch_row_fwd_batch_f64(const GridDev&, const AxisPlanH&, const void*, const RowCfg&, const RowFwdArgs*, int, int, cudaStream_t);
cudaError_t launch_row_inv_batch_f32(const GridDev&, const AxisPlanH&, const void*, const RowCfg&, const RowInvArgs*, int, int, cudaStream_t);
cudaError_t launch_row_inv_batch_f64(const GridDev&, const AxisPlanH&, const void*, const RowCfg&, const RowInvArgs*, int, int, cudaStream_t);
cudaError_t launch_strided_batch_f32(const GridDev&, const AxisPlanH&, const void*, const StrCfg&, const StrArgs*, int, int, int, long long, long long, cudaStream_t);
cudaError_t launch_strided_batch_f64(const GridDev&, const AxisPlanH&, const void*, const StrCfg&, const StrArgs*, int, int, int, long long, long long, cudaStream_t);
cudaError_t configure_f32(int max_smem, const double* ctw);
cudaError_t configure_f64(int max_smem, const double* ctw);

}  // namespace hgk
