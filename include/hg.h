/*
 * hg.h -- C ABI of the GB300 FFT-Galerkin homogenization library (libhg.so).
 *
 * The library solves the cell problem of periodic homogenization discretised
 * by trigonometric polynomials with numerical integration (GaNi), following
 * Vondrejc, Zeman & Marek, "An FFT-based Galerkin method for homogenization
 * of periodic media" (arXiv:1311.0089):
 *
 *   G_N A_N e~ = -G_N A_N E            (Sec. 5.2, Eq. final_system, A0 = I)
 *
 * by conjugate gradients (Sec. 5.3, Lemma on CG), where A_N is the pointwise
 * coefficient matrix at the grid points (Sec. 5.1), G_N = F^-1 Gamma_hat F A0
 * (Eq. FFT_matrices) and Gamma_hat(k) = xi xi^T / (A0 xi . xi), zero at k = 0
 * (Sec. 3, Eq. Gamma_hat).  For each macroscopic load E = e_j it returns the
 * fluctuation e~_j and the homogenized matrix
 *
 *   A_H[i][j] = (A_N (E_j + e~_j), E_i + e~_i)    (energy of Eq. forms_def1;
 *                                                   the paper does not define A_H)
 *
 * with the scalar product (u,v) = 1/|N| sum_k u^k . v^k of Sec. 5.1.
 *
 * Conventions common to every call:
 *   - Status codes only (hg_status); nothing aborts, traps or throws.
 *   - Grids: d in {2,3}; every N_a odd (assumption A4, Sec. 4.1), a product
 *     of the primes 3, 5 and 7 (a limit of this library's FFT kernels, not of
 *     the paper), 1 <= N_a <= 1024.
 *   - Arrays are C order, first index slowest.  A field of d components is
 *     stored component-major: u[a * |N| + k] (d x |N| doubles).
 *   - The library owns every device buffer it allocates; coefficient arrays
 *     passed in are copied, the caller keeps ownership of its pointers.
 *   - "on_device" flags say whether a pointer is a device pointer (1) or a
 *     host pointer (0).  Host pointers are copied through the context stream.
 *   - Every call that launches work runs on the context's stream and returns
 *     after that work has completed, unless documented otherwise.
 */
#ifndef HG_H
#define HG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hg_ctx hg_ctx;
typedef struct hg_grid hg_grid;

typedef enum {
    HG_OK = 0,
    HG_PENDING = 1,                 /* hg_poll: the ticket is still running      */
    HG_ERR_ARG = -1,                /* null pointer, bad enum, d not in {2,3}     */
    HG_ERR_UNSUPPORTED_SIZE = -2,   /* even N_a (A4) or prime factor not 3/5/7   */
    HG_ERR_NOT_SPD = -3,            /* a coefficient tensor is not symmetric PD  */
    HG_ERR_NO_MEMORY = -4,          /* device allocation or the ctx budget failed */
    HG_ERR_NOT_CONVERGED = -5,      /* max_iter reached; best iterate is kept     */
    HG_ERR_DEVICE_TIMEOUT = -6,     /* a bounded device-side wait (a grid barrier
                                       of the resident solver) gave up           */
    HG_ERR_BUSY = -7,               /* grid borrowed by a pending ticket          */
    HG_ERR_CUDA = -8,               /* a CUDA runtime call failed                 */
    HG_ERR_CANCELLED = -9,          /* the ticket was cancelled                   */
    HG_ERR_BREAKDOWN = -10,         /* CG breakdown: (p, A p) <= 0 or not finite   */
    HG_ERR_NO_COEFFS = -11,         /* solve requested before hg_set_coeffs*       */
    HG_ERR_TOO_LARGE = -12          /* grid exceeds the fixed scratch of
                                       hg_apply_noalloc                            */
} hg_status;

typedef enum {
    HG_FP64 = 0,    /* every step in FP64 */
    HG_MIXED = 1    /* FP32 FFTs/products/axpys, FP64 dots, FP64 outer residual
                       and A_H (iterative refinement) */
} hg_precision;

typedef enum {
    HG_CG = 0,      /* conjugate gradients on G_N A_N e~ = -G_N A_N E
                       (Eq. final_system, Sec. 5.3 Lemma)                  */
    HG_MS = 1       /* Moulinec-Suquet fixed point (Neumann series of the
                       discrete Lippmann-Schwinger equation, Sec. 5.3
                       comments): e_i = E - Gamma_N (A_N - lambda I) e_{i-1} */
} hg_method;

typedef enum {
    HG_PRIMAL = 0,  /* fields: e = E + e~, e~ in E_N (curl-free), loads E = e_j */
    HG_DUAL = 1     /* fluxes: s = S + s~, s~ in J_N (divergence-free), unit
                       flux loads S = e_j, coefficients A_N^-1; the Helmholtz
                       decomposition R^{dN} = U_N + E_N + J_N of Sec. 5.1
                       (Eq. Helmholtz_discrete) and the dual problem that
                       Sec. 6 announces.  Gives the compliance C_H and
                       A_H = C_H^-1, equal to the primal A_H for GaNi        */
} hg_formulation;

typedef enum {
    HG_COEFF_FULL = 0,    /* |N| x d x d doubles, voxel-major, symmetric      */
    HG_COEFF_PACKED = 1   /* d(d+1)/2 x |N| doubles, component-major; the
                             packed order is (11,22[,33],12[,13,23])          */
} hg_coeff_layout;

typedef struct {
    double tol;          /* HG_CG: stop when ||r_i|| / ||b|| <= tol.  HG_MS: stop
                            when ||e_i - e_{i-1}|| / ||E|| <= tol (HG_MIXED:
                            when the next step, ||r|| / lambda with the FP64
                            residual r, is).  Default 1e-10                    */
    int max_iter;        /* iterations per load (default 10000)                 */
    int prec;            /* hg_precision (default HG_FP64)                      */
    double lambda_ref;   /* A0 = lambda I.  HG_CG does not depend on it (Lemma
                            FD_projection (v)).  HG_MS: the reference medium;
                            <= 0 (default 0) takes (c_A + C_A) / 2, the extreme
                            eigenvalues of A_N over all voxels; a lambda <=
                            C_A / 2, for which the series need not converge,
                            returns HG_ERR_ARG                                 */
    unsigned loads_mask; /* bit j set: solve load E = e_j (default all)        */
    double inner_tol;    /* HG_MIXED: relative tolerance of each FP32 inner solve
                            (default 1e-4)                                      */
    int check_every;     /* iterations between host reads of the convergence
                            flags (default 8); each chunk is one CUDA graph    */
    int max_outer;       /* HG_MIXED: refinement steps (default 30)            */
    int time_pass;       /* >= 0: time this pass with CUDA events inside the
                            captured graphs, in the first iteration of every
                            chunk of check_every iterations (0 = the forward
                            pass, last = the inverse pass (update), in launch
                            order; hg_num_iter_passes passes); results in
                            hg_result.pass_*.  -1 (default): no timing.
                            check_every <= 64.                                 */
    int method;          /* hg_method (default HG_CG).  HG_MS needs the bounds
                            c_A, C_A: the first HG_MS solve after new
                            coefficients computes them on the device and
                            waits for them on the host once                   */
    int formulation;     /* hg_formulation (default HG_PRIMAL); HG_DUAL needs
                            every load in loads_mask and the reference
                            medium A0 = I                                      */
    double A0[9];        /* HG_CG, HG_PRIMAL: a general SPD reference medium
                            (d x d row-major) for Eq. LSD.  The iteration runs
                            on Gamma_N(A0) A_N e~ = -Gamma_N(A0) A_N E in the
                            scalar product (A0 u, v), in which that operator
                            is symmetric positive definite on E_N (Lemma
                            FD_projection (ii)-(iii)); the solution, hence
                            A_H, does not depend on A0, the iteration count
                            does (an anisotropic A0 close to the medium's
                            anisotropy can save many iterations).  A0[0] = 0
                            (default): A0 = lambda_ref I.  Not SPD:
                            HG_ERR_NOT_SPD; with HG_MS or HG_DUAL: HG_ERR_ARG */
    int batch_tiles;     /* hg_solve_batch only.  1 (default): the last-axis
                            passes of each grid shape use the largest row tile
                            (all loads, the most grid rows per CTA) that still
                            gives at least two CTAs per SM over the shape's
                            problems: few large CTAs pay off when many problems
                            share a launch, many small ones for a single
                            problem.  Iterates then equal a single solve's up to
                            the rounding of the CTA partial sums.  0: each shape
                            runs its first grid's launch geometry, and every
                            problem's iterates equal those of its own
                            hg_solve_AH bitwise.                              */
    int resident;        /* HG_MIXED on a square 2D grid of side 15, 27, 45,
                            75, 81, 135, 243, 375 or 729: run each inner FP32
                            solve as
                            ONE cooperative launch whose CTAs (one per SM) keep
                            the residual, the search direction and the iterate
                            of their grid rows in tensor memory for all its
                            iterations, with bounded grid-wide barriers between
                            the row, column and row phases of an iteration
                            (hg_solve_AH only; hg_submit and hg_solve_batch run
                            the pass kernels there).  On N0 x N x N grids with
                            N in {15, 27, 45, 81, 135} and A0 = I, each FP32
                            iteration is the three plane passes (axes 1 and 2
                            transformed in shared memory, one CTA per plane and
                            component), in every entry point.  -1 (default):
                            where they apply and the state fits; 0: never (the
                            pass kernels, check_every iterations per CUDA
                            graph); > 0: as -1, the resident launch with at
                            most that many CTAs.  The iterates equal those of
                            the pass kernels up to the rounding of the partial
                            sums.  time_pass >= 0 times the resident launch
                            (one per inner solve) or a plane pass.  A barrier
                            wait that gives up returns HG_ERR_DEVICE_TIMEOUT. */
} hg_solve_opts;

typedef struct {
    int status;             /* hg_status of the solve                          */
    int d;
    double AH[9];           /* d x d row-major energy form (HG_DUAL: C_H^-1)   */
    double AH_flux[9];      /* d x d mean-flux form <A e_j>_i (check)          */
    int iters[3];           /* iterations per load (HG_MIXED: inner FP32
                               iterations summed over refinement steps)        */
    int outer[3];           /* HG_MIXED: FP64 residual evaluations per load    */
    double rel_res[3];      /* final ||r|| / ||b|| in the scalar product of the
                               iteration (FP64 true residual for
                               HG_MIXED, recursive residual for HG_FP64)       */
    double device_ms;       /* time of the solve on the context stream         */
    double wall_ms;         /* host wall time of the call                      */
    long long launches;     /* kernels launched by this solve                  */
    double pass_ms_total;   /* time_pass >= 0: summed duration of the timed pass
                               over the timed iterations in which a system was
                               active                                          */
    int pass_launches;      /* number of such launches                         */
    double lambda_ref;      /* HG_MS: the lambda used (0 for HG_CG)            */
    double c_A, C_A;        /* HG_MS: smallest and largest eigenvalue of the
                               coefficients the method iterates with (A_N, or
                               A_N^-1 for HG_DUAL) over the voxels             */
    double CH[9];           /* HG_DUAL: compliance C_H[i][j] = (A_N^-1 s_j, s_i)
                               (energy form); AH = C_H^-1, AH_flux = the inverse
                               of the mean-field form <A_N^-1 s_j>_i           */
    double true_rel_res[3]; /* ||b - G_N A_N e~|| / ||b|| recomputed in FP64 from
                               the returned e~ at exit (the paper leaves the
                               stopping rule of Sec. 5.3 open; this is the
                               residual the recursion does not see), in the
                               scalar product of the iteration; 0 for loads
                               not solved or with a zero right-hand side      */
    int resident_ctas;      /* CTAs of the resident FP32 solver (0: not used)  */
} hg_result;

/* Fill opts with the defaults listed above. */
void hg_default_opts(hg_solve_opts* opts);

/* Context: one device, one stream.  cuda_stream = NULL creates an owned
 * non-blocking stream; otherwise the given cudaStream_t is used (borrowed).
 * mem_budget_bytes = 0 means no budget; otherwise device allocations made
 * through this context beyond the budget fail with HG_ERR_NO_MEMORY. */
int hg_create(hg_ctx** out, int device, size_t mem_budget_bytes, void* cuda_stream);
/* Fails with HG_ERR_BUSY while grids created on ctx are still alive. */
int hg_destroy(hg_ctx* ctx);

/* Grid of Sec. 4.1: d axes of N[a] points on the cell prod_a [-Y_a, Y_a]
 * (Y = NULL: all Y_a = 1).  xi(k) = (k_a / Y_a)_a (Sec. 2).  Allocates the
 * plans and twiddle tables; work buffers are allocated on first solve. */
int hg_create_grid(hg_ctx* ctx, int d, const int* N, const double* Y, hg_grid** out);
int hg_destroy_grid(hg_grid* grid);   /* HG_ERR_BUSY if a ticket holds it */

/* Coefficients A(x_k) of Sec. 5.1 (A_N), assumptions A1-A2 (Sec. 3): symmetric
 * positive definite per voxel.  Copied into device memory.  Symmetry and
 * positive definiteness are checked on the host for every voxel (device inputs
 * are staged through host memory for the check); a violation returns
 * HG_ERR_NOT_SPD and leaves the previous coefficients. */
int hg_set_coeffs(hg_grid* grid, const double* A, int layout, int on_device);

/* Coefficients as a phase map: phase[k] in [0, n_phases) per voxel (uint8),
 * table = n_phases x d x d doubles (row-major, each SPD).  1 <= n_phases <= 256. */
int hg_set_coeffs_phase(hg_grid* grid, const uint8_t* phase, int n_phases,
                        const double* table, int on_device);

/* Coefficients for the Galerkin scheme with exact integration (Sec. 4.2, Ga):
 * A constant on the pixels of a grid P (phase: |P| bytes on the host, C order,
 * entries in [0, n_phases); table: n_phases x d x d host doubles, each SPD),
 * trial space Z_N with N = N_trial (odd per axis).  The grid is the quadrature
 * grid M and needs M_a >= 2 N_a - 1 per axis, so that the grid mean of
 * A_M u . v for trial fields u, v is their exact integral (A_M: the Fourier
 * series of A truncated to |l_a| <= N_a - 1, built from the pixels' sinc
 * coefficients).  Solves then restrict the projection Gamma_hat to Z_N and
 * return the Ga A_H, an upper bound on the continuous A_H; an HG_DUAL solve
 * uses (A^-1)_M and returns the matching lower bound.  HG_MS and a general A0
 * are refused on such a grid (HG_ERR_ARG).  Blocks until the fields are built.
 * Errors: HG_ERR_ARG (sizes, phases), HG_ERR_NOT_SPD, HG_ERR_OOM, HG_ERR_BUSY. */
int hg_set_coeffs_exact(hg_grid* grid, const int* N_trial, const int* P, const uint8_t* phase,
                        int n_phases, const double* table);

/* Blocking solve of Eq. final_system for the loads in opts->loads_mask and
 * assembly of A_H (rows/columns of unsolved loads are left 0).  AH_out may be
 * NULL (d*d doubles, row-major); info may be NULL. */
int hg_solve_AH(hg_grid* grid, const hg_solve_opts* opts, double* AH_out, hg_result* info);

/* Batched blocking solve of n problems, each grid with its own shape (d, N,
 * Y) and coefficients.  Problems of one shape form a group: every pass of the
 * iteration is one launch for all problems of the group (the launch's z index
 * picks the problem).  The CG iterations of the whole batch are captured
 * check_every at a time in one CUDA graph with one branch per group, so the
 * groups run concurrently and one graph launch steps every problem; each
 * problem keeps its own convergence status, so converged problems drop out of
 * the launches.  HG_MIXED: each problem's FP64 refinement step runs as soon as
 * its inner FP32 solve stops, beside the next graph launch.  A group runs the
 * strided passes with the launch geometry of its first grid, and the
 * last-axis passes with the row tile opts->batch_tiles selects.
 * results[p] (n entries) is the result of grids[p]; device_ms and wall_ms are
 * those of the whole batch.  Each problem solves its own d loads (those in
 * loads_mask).  Supports HG_CG, HG_PRIMAL, A0 = I, HG_FP64 and HG_MIXED,
 * time_pass = -1 (else HG_ERR_ARG); all grids on one context, each at most
 * once.  Returns the first non-OK status of a problem, or HG_OK. */
int hg_solve_batch(hg_grid* const* grids, int n, const hg_solve_opts* opts, hg_result* results);

/* Copy e~_load of the last solve (d x |N| doubles, component-major); after an
 * HG_DUAL solve, the flux fluctuation s~_load. */
int hg_get_field(hg_grid* grid, int load, double* e_out, int on_device);

/* Asynchronous solve through the context's scheduler (continuous batching:
 * iterations of all admitted requests run together).  The grid is borrowed
 * until the ticket completes or is cancelled.  Admission waits for memory
 * within the context budget. */
int hg_submit(hg_ctx* ctx, hg_grid* grid, const hg_solve_opts* opts, uint64_t* ticket);
/* HG_PENDING while running; otherwise fills *out and releases the ticket.
 * timeout_us = 0 polls once; < 0 waits without limit. */
int hg_poll(hg_ctx* ctx, uint64_t ticket, hg_result* out, int timeout_us);
int hg_cancel(hg_ctx* ctx, uint64_t ticket);

/* ---- operator-level entry points (parity tests and diagnostics) ---------- */

/* out = G_N A_N u (with_A = 1) or out = G_N u (with_A = 0), for one d x |N|
 * field, with G_N = F^-1 Gamma_hat F A0 (Eq. FFT_matrices).  A0 = NULL means
 * I; otherwise a d x d SPD matrix (row-major).  prec = hg_precision: HG_MIXED
 * runs the FP32 kernels (inputs/outputs still FP64 at the boundary). */
int hg_apply(hg_grid* grid, const double* u, double* out, int with_A,
             const double* A0, int prec, int on_device);

/* Forward DFT of Eq. DFT_def (with 1/|N|) of a real d x |N| field, returned as
 * the half spectrum over the last axis: d x (|N|/N_d) x ((N_d+1)/2) complex
 * values, interleaved (re, im) doubles; bin j of an axis holds frequency
 * j or j - N_a (Sec. 4.1); the last axis keeps j = 0..(N_d-1)/2. */
int hg_spectrum(hg_grid* grid, const double* u, double* S_out, int prec, int on_device);

/* out = G_N A_N u for one d x |N| field, like hg_apply(with_A = 1, A0 = NULL,
 * HG_FP64) on a grid with Y = 1, but without allocating any device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they need the operator (plug-ins whose
 * device memory belongs to their host application's allocator, real-time
 * loops in which cudaMalloc/cudaFree and their synchronisation are not
 * allowed).  It needs no hg_ctx or hg_grid.
 *   d, N      : as hg_create_grid (N_a odd, factors 3/5/7, <= 1024).
 *   phase     : device pointer, |N| uint8 phase indices (< n_phases).  The
 *               map is not checked (that would need a read-back): an index
 *               >= n_phases is read as n_phases - 1, never past the table.
 *   table     : device pointer, n_phases x d x d doubles (SPD, not checked).
 *   u, out    : device pointers, d x |N| doubles each (component-major).
 *   cuda_stream: cudaStream_t to enqueue on (NULL = the legacy default stream).
 * Scratch: a fixed 16 MiB static device array per GPU that loads the library,
 * held until process exit; grids whose twiddles, reduction slots and half
 * spectrum (d * |N|/N_d * (N_d+1)/2 complex doubles) do not fit return
 * HG_ERR_TOO_LARGE before any work is enqueued.  The call only enqueues work
 * (out is ready when the stream reaches it).  Every call shares the scratch:
 * calls whose work overlaps on the GPU race; each call clears what must start
 * at zero.  The first call on a device sets up that device (scratch address,
 * kernel attributes, codelet constants): make it before any stream capture. */
int hg_apply_noalloc(int d, const int* N, const uint8_t* phase, int n_phases,
                     const double* table, const double* u, double* out, void* cuda_stream);

/* ---- launch geometry and its autotuner ------------------------------------
 * Not in the paper: the paper gives no kernel.  Each CG iteration runs d + 1
 * passes over the grid (the last-axis forward pass with the A_N p product, the
 * strided passes with the Gamma_hat projection of Eq. Gamma_hat, the last-axis
 * inverse pass with the CG update).  How a pass tiles the grid over CTAs
 * changes its speed, not its result beyond the rounding of the reductions'
 * partial sums. */
typedef struct {
    int row_rb;      /* grid rows (lines along the last axis) staged per CTA by the
                        last-axis passes (forward and inverse share it)          */
    int row_lb;      /* loads staged per CTA by the last-axis passes (1..d)      */
    int lanes[2];    /* pencils per component staged per CTA by the strided pass
                        of axis a (a = 0, and a = 1 in 3D; 0 where unused), a
                        power of two                                             */
    int radix[3][8]; /* order of the radix-3/5/7 Stockham stages of the FFT along
                        axis a, zero-terminated, for the lengths without
                        compile-time kernels (whose plan is read at run time);
                        all zero for the other axes.  hg_set_launch_cfg: all
                        zero = the default order (3s, then 5s, then 7s); a
                        permutation of the length's factors otherwise.  The
                        order is the grid's, shared by both precisions.          */
} hg_launch_cfg;

/* The grid's current geometry for precision prec (HG_FP64 or HG_MIXED, the
 * latter meaning the FP32 kernels). */
int hg_get_launch_cfg(hg_grid* grid, int prec, hg_launch_cfg* out);
/* Sets it.  HG_ERR_ARG if the kernels cannot run that tile (too many pencils
 * for shared memory or registers, lanes not a power of two, more rows than the
 * grid, a radix order that is not a permutation of the axis length's factors
 * or is given for a length with compile-time kernels); HG_ERR_BUSY while a
 * ticket holds the grid.  Drops the grid's cached CUDA graphs. */
int hg_set_launch_cfg(hg_grid* grid, int prec, const hg_launch_cfg* cfg);

typedef struct {
    hg_launch_cfg chosen;      /* geometry set on the grid                        */
    hg_launch_cfg heuristic;   /* the library's default for this grid             */
    double ms_chosen;          /* one CG iteration's passes, ms (timed; or the
                                  cache's record when from_cache)                 */
    double ms_heuristic;       /* same with the default geometry (0 from cache)   */
    int candidates;            /* geometries timed (0 from cache)                 */
    int from_cache;            /* 1: taken from cache_path without timing         */
} hg_tune_result;

/* Autotuner: times every geometry the kernels can run for this grid shape and
 * precision (all rows x loads tiles of the last-axis passes, all lane counts
 * of each strided pass, every distinct radix order of each axis whose length
 * has no compile-time kernel), each over `reps` launches of its passes (CUDA
 * events on the context stream, best of three), on the grid's own
 * coefficients with steady-state CG scalars, and sets the fastest (the
 * default unless another is at least 3% faster: closer timings are within the
 * run-to-run spread; and the default again unless the whole iteration with
 * the chosen combination beats it).  cache_path (NULL: no cache) is a text file of one
 * record per line, "hg-tune-v2 <device> <SMs> <prec> <d> <N0> <N1> <N2> <rb>
 * <lb> <lanes0> <lanes1> <ms> <order0> <order1> <order2>", device = its name
 * with blanks as '_', order_a = the radix order of axis a as digits ("357"),
 * or 0 (the default order, or a length with compile-time kernels): a record
 * for this device, shape and precision is applied without timing (the last
 * such line wins); otherwise the result is appended.  The work buffers are
 * left with meaningless values (every solve starts from its right-hand side).
 * Errors: HG_ERR_ARG, HG_ERR_NO_COEFFS, HG_ERR_BUSY, HG_ERR_CUDA. */
int hg_tune(hg_grid* grid, int prec, int reps, const char* cache_path, hg_tune_result* out);

/* Looks up a record of the cache format above (host only, no device work):
 * HG_OK and *out if found, HG_ERR_ARG if not (or unreadable); *ms_out (may be
 * NULL) receives the recorded time. */
int hg_tune_cache_find(const char* cache_path, const char* device_name, int sm_count, int prec, int d,
                       const int* N, hg_launch_cfg* out, double* ms_out);

/* Error-path check of the resident FP32 solver (not in the paper): an
 * HG_MIXED hg_solve_AH in which CTA drop_cta (>= 1) of the resident launch
 * leaves at once, so the other CTAs' barrier waits run out after their time
 * limit (0.1 s here).  Returns HG_ERR_DEVICE_TIMEOUT when the grid runs the
 * resident solver (the context stays usable; the grid's last result is
 * meaningless), the plain solve's status otherwise; HG_ERR_ARG for
 * drop_cta < 1, HG_FP64, resident = 0 or time_pass >= 0. */
int hg_test_resident_timeout(hg_grid* grid, const hg_solve_opts* opts, int drop_cta, hg_result* info);

/* Kernel launches made through this context so far (all entry points). */
long long hg_launch_count(hg_ctx* ctx);

/* Time `reps` back-to-back launches of one pass of the CG iteration on the
 * grid's current state with CUDA events on the context stream.
 * pass: 0 = first-axis forward pass (A.p product + FFT), 1.. = strided-axis
 * passes in launch order, last = last-axis inverse pass (update).  Writes the
 * mean milliseconds per launch and the pass name (<= 63 chars). */
int hg_time_pass(hg_grid* grid, int prec, int pass, int reps, double* ms_out,
                 char* name_out);
int hg_num_passes(hg_grid* grid);
/* Launches of one CG iteration of a solve of `grid` with `opts` (null: the
 * defaults): the valid range of opts->time_pass.  3 where the FP32 iteration
 * runs as the plane passes (see hg_solve_opts.resident), else the pass
 * kernels' d + 1.  Negative status on a null grid. */
int hg_num_iter_passes(hg_grid* grid, const hg_solve_opts* opts);

const char* hg_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* HG_H */
