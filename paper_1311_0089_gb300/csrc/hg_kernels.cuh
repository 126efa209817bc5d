// CUDA kernels of the FFT-Galerkin CG iteration (sm_103a): shared device
// helpers and the three pass kernels, templated on the precision T, the
// dimension D and the transform length NN of the pass (NN = 0: any length,
// plan read at run time; NN > 0: every index and radix fixed at compile time).
//
// One CG iteration on a d-dimensional grid is d + 1 (2D: 3) kernel launches:
//
//   row_fwd   last-axis pass:  p <- r + beta p;  t = A_N p  (Sec. 5.1, A_N);
//             (p, t) partial sums;  real-to-complex DFT of t along the
//             contiguous axis (two real rows packed in one complex FFT);
//             alpha = (r,r) / (p, A p) by the last CTA.
//   strided   middle axes (3D): forward / inverse DFT along a strided axis.
//   strided   first axis: forward DFT, Fourier projection
//             q_hat = xi (xi . t_hat) / |xi|^2 / |N|   (Eq. Gamma_hat, A0 = I),
//             inverse DFT, all in shared memory.
//   row_inv   last-axis inverse (complex-to-real) DFT giving q = G_N A_N p,
//             then x += alpha p, r -= alpha q, (r, r) partial sums; beta and
//             the convergence test by the last CTA.
//
// alpha uses (p, G A p) = (p, A p): G_N is self-adjoint and p lies in E_N
// (Lemma FD_projection (iii),(v); Sec. 5.3, Eq. CG_identity), so the
// denominator is available before the FFTs and q never goes to memory.
//
// Reductions are deterministic: each CTA writes its partial sums to a slot,
// the last CTA to arrive (atomic ticket) adds the slots in a fixed order.
#pragma once
#include "hg_internal.h"
#include "fft_device.cuh"

namespace hgk {

constexpr int MAXB = 2;     // runtime kernels: butterflies per thread per stage
constexpr int MAXT = 512;   // runtime kernels: threads per CTA (upper bound)
constexpr double ZERO_RHS = 1e-13;
// An FP32 right-hand side carries roundoff of about 1e-7 ||A E||; below this
// ratio it cannot decide the zero test, and the FP64 one is taken.
constexpr double RHS32_RECHECK = 1e-4;

template <typename T> using Cx = typename cplx_t<T>::type;

template <typename T> __device__ __forceinline__ Cx<T> czero();
template <> __device__ __forceinline__ double2 czero<double>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 czero<float>() { return make_float2(0.f, 0.f); }

// ---------------------------------------------------------------------------
// block reductions
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double red[NV][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
        if (lane == 0) red[i][wid] = v[i];
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            v[i] = lane < nw ? red[i][lane] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], off);
        }
    }
    __syncthreads();
}

// Block sum of per-thread partials held in T: warp sums in T (32 terms), then
// the warp sums of the block accumulated exactly as an unevaluated pair
// hi + lo (Knuth's TwoSum, error-free in T), and FP64 across the CTAs of the
// grid (final_sums).  The pair is packed into the CTA's FP64 slot, so an
// FP32 pass issues no FP64 instruction outside its last CTA.  Valid in thread 0.
__device__ __forceinline__ double pack_pair(float hi, float lo) {
    return __longlong_as_double(((long long)__float_as_int(lo) << 32) | (unsigned)__float_as_int(hi));
}
__device__ __forceinline__ double unpack_pair(double v) {
    const long long b = __double_as_longlong(v);
    return (double)__int_as_float((int)(b & 0xffffffffll)) + (double)__int_as_float((int)(b >> 32));
}
template <typename T> struct SlotCodec;
template <> struct SlotCodec<float> {
    __device__ __forceinline__ static double pack(float hi, float lo) { return pack_pair(hi, lo); }
    __device__ __forceinline__ static double unpack(double v) { return unpack_pair(v); }
};
template <> struct SlotCodec<double> {
    __device__ __forceinline__ static double pack(double hi, double lo) { return hi + lo; }
    __device__ __forceinline__ static double unpack(double v) { return v; }
};

template <typename T, int NV>
__device__ __forceinline__ void block_sum_t(const T (&v)[NV], double (&out)[NV]) {
    __shared__ T red[NV][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        T x = v[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) red[i][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            T hi = T(0), lo = T(0);
            for (int w = 0; w < nw; ++w) {
                const T b = red[i][w];
                const T s = hi + b;                 // TwoSum(hi, b)
                const T bb = s - hi;
                const T err = (hi - (s - bb)) + (b - bb);
                hi = s;
                lo += err;
            }
            out[i] = SlotCodec<T>::pack(hi, lo);
        }
    }
    __syncthreads();
}

// Writes `cnt` partials (slot s of this CTA at partial[s * stride + bid]) and
// returns true in the last CTA to finish (of `nblocks`).
__device__ __forceinline__ bool publish(const double* vals, const int* slots, int cnt,
                                        double* partial, long long stride, long long bid,
                                        unsigned* counter, unsigned nblocks) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        for (int i = 0; i < cnt; ++i) partial[slots[i] * stride + bid] = vals[i];
        __threadfence();
        unsigned prev = atomicAdd(counter, 1u);
        last = (prev == nblocks - 1);
    }
    __syncthreads();
    return last;
}

// In the last CTA: sums slot s over `nb` CTAs in a fixed order; result in
// out[s] (valid in every thread).
template <int NV, typename T = double>
__device__ __forceinline__ void final_sums(const double* partial, long long stride, long long nb,
                                           int nslots, double (&out)[NV]) {
    __shared__ double res[NV];
    __threadfence();
    double v[NV];
#pragma unroll
    for (int s = 0; s < NV; ++s) v[s] = 0.0;
    for (long long b = threadIdx.x; b < nb; b += blockDim.x) {
#pragma unroll
        for (int s = 0; s < NV; ++s)
            if (s < nslots) v[s] += SlotCodec<T>::unpack(__ldcg(&partial[s * stride + b]));
    }
    block_sum<NV>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < NV; ++s) res[s] = v[s];
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < NV; ++s) out[s] = res[s];
}

// ---------------------------------------------------------------------------
// coefficients A(x_k) (Sec. 5.1: A_N = diag_k A(x_k))
// ---------------------------------------------------------------------------
// A phase table of at most 16 entries is staged in shared memory (the
// lookup then follows the phase byte load with a shared-memory read).
constexpr int SMEM_PHASES = 16;

template <typename T, int D>
__device__ __forceinline__ const T* stage_table(const CoeffsDev& co, T* s_tab) {
    if (co.mode == 0 && co.n_phases <= SMEM_PHASES) {
        const T* tb = static_cast<const T*>(co.table);
        for (int i = threadIdx.x; i < co.n_phases * D * D; i += blockDim.x) s_tab[i] = tb[i];
        return s_tab;
    }
    return static_cast<const T*>(co.table);
}

template <typename T, int D>
__device__ __forceinline__ void load_coeffs(const CoeffsDev& co, long long k, long long M, T (&a)[D][D],
                                            const T* tab) {
    if (co.mode == 0) {
        // an index past the table (possible only through hg_apply_noalloc,
        // whose phase map is not checked on the host) reads the last entry
        const T* tb = tab + min((int)co.phase[k], co.n_phases - 1) * D * D;
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) a[i][j] = tb[i * D + j];
        return;
    }
    if (co.mode == 1) {
        const T* f = static_cast<const T*>(co.field);
        if (D == 2) {
            a[0][0] = f[k]; a[1][1] = f[M + k]; a[0][1] = a[1][0] = f[2 * M + k];
        } else {
            a[0][0] = f[k]; a[1][1] = f[M + k]; a[D - 1][D - 1] = f[2 * M + k];
            a[0][1] = a[1][0] = f[3 * M + k];
            a[0][D - 1] = a[D - 1][0] = f[4 * M + k];
            a[1][D - 1] = a[D - 1][1] = f[5 * M + k];
        }
    } else {
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) a[i][j] = (i == j) ? T(1) : T(0);
    }
}

__device__ __forceinline__ int freq_of(int j, int n) { return (2 * j <= n - 1) ? j : j - n; }

// 1/x: FP32 correctly rounded reciprocal; FP64 by two Newton-Raphson steps
// y <- y (2 - x y) from the FP32 reciprocal (quadratic convergence: 2^-24 ->
// 2^-48 -> below FP64 rounding), avoiding a full FP64 division.
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) {
    double y = (double)__frcp_rn((float)x);
    y = y * fma(-x, y, 2.0);
    y = y * fma(-x, y, 2.0);
    return y;
}

// Transform of `npen` staged pencils of length n (forward or inverse).
template <typename T, int NN, bool INV>
__device__ __forceinline__ void fft_any(Cx<T>* buf, int npen, int n, const AxisPlanH& pl,
                                        const Cx<T>* __restrict__ twg, const Cx<T>* tws) {
    if constexpr (NN > 0) fft_ct<T, NN, INV>(buf, npen, tws);
    else fft_pencils<T, INV, MAXB>(buf, npen, n, pl, twg);
}

// The compile-time kernels stage their per-stage twiddle tables in shared
// memory after the pencils (fewer than n entries); the runtime kernels read
// the natural table from global memory.
template <typename T, int NN>
__device__ __forceinline__ Cx<T>* stage_twiddles(Cx<T>* smem_after, const AxisPlanH& pl,
                                                 const Cx<T>* __restrict__ twg) {
    if constexpr (NN > 0) {
        fft_ct_twiddles<T, NN>(smem_after, twg + pl.tw_off);
        return smem_after;
    } else {
        return nullptr;
    }
}

template <int NN> struct PassThreads { static constexpr int v = NN > 0 ? CT_THREADS : MAXT; };

// The tile a pass body works on (the CTA's block index in a plain launch) and
// the number of tiles in x and y (the grid of a plain launch).
struct TileIdx {
    int x, y, z, nx, ny;
    __device__ static TileIdx of_block() {
        TileIdx t;
        t.x = blockIdx.x; t.y = blockIdx.y; t.z = blockIdx.z; t.nx = gridDim.x; t.ny = gridDim.y;
        return t;
    }
};
// CTAs per SM the compiler must fit: the FP32 3D strided passes of lengths 45,
// 81 and 135 run 6 (at most 42 registers) where they would take 4 at their
// natural 54, which keeps more tile loads in flight (10-15% faster on 135^3);
// other lengths would spill under that bound.  The FP32 2D passes keep 3 (at
// most 85 registers), the residency their one-wave grids are sized for.
template <typename T, int D, int NN> struct StridedMinBlocks {
    static constexpr int v = (D == 3 && sizeof(T) == 4 && (NN == 45 || NN == 81 || NN == 135)) ? 6
                             : (D == 2 && sizeof(T) == 4 && NN > 0) ? 3 : 1;
};

// Programmatic dependent launch: the pass kernels are launched so that their
// CTAs may start while the previous kernel in the stream finishes.  Work that
// depends on nothing the previous kernel writes (twiddle and coefficient
// staging) runs first; grid_dep_wait() then blocks until the previous grid has
// completed and its memory is visible, before any dependent read.
// grid_dep_launch() lets the next kernel start launching its CTAs.  Both are
// no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Strided-pass transform: interleaved layout for the compile-time kernels.
template <typename T, int D, int NN, bool INV>
__device__ __forceinline__ void fft_str(Cx<T>* buf, int Cl, int lgCl, int n, const AxisPlanH& pl,
                                        const Cx<T>* __restrict__ twg, const Cx<T>* tws) {
    if constexpr (NN > 0) fft_ct_il<T, NN, INV, D>(buf, lgCl, tws);
    else fft_pencils<T, INV, MAXB>(buf, D * Cl, n, pl, twg);
}

__device__ __forceinline__ float weight_of(const Weight& w, int i, float) { return w.wf[i]; }
__device__ __forceinline__ double weight_of(const Weight& w, int i, double) { return w.w[i]; }
__device__ __forceinline__ float load_of(const RowFwdArgs& a, int i, float) { return a.Ef[i]; }
__device__ __forceinline__ double load_of(const RowFwdArgs& a, int i, double) { return a.Ed[i]; }

// CG scalars in the kernel's precision (FP32 copies are written beside the
// FP64 values by the reducing CTA).
__device__ __forceinline__ float beta_of(const Scalars& s, float) { return s.beta_f; }
__device__ __forceinline__ double beta_of(const Scalars& s, double) { return s.beta; }
__device__ __forceinline__ float alpha_of(const Scalars& s, float) { return s.alpha_f; }
__device__ __forceinline__ double alpha_of(const Scalars& s, double) { return s.alpha; }
__device__ __forceinline__ float inv_y(const GridDev& g, int a, float) { return g.invYf[a]; }
__device__ __forceinline__ double inv_y(const GridDev& g, int a, double) { return g.invY[a]; }
__device__ __forceinline__ float inv_m(const GridDev& g, float) { return g.invMf; }
__device__ __forceinline__ double inv_m(const GridDev& g, double) { return g.invM; }
// f / den for the projection: FP32 fast division (2 ulp), FP64 Newton reciprocal
__device__ __forceinline__ float div_proj(float f, float den) { return __fdividef(f, den); }
__device__ __forceinline__ double div_proj(double f, double den) { return f * recip(den); }

// Largest number of real rows a row-pass CTA stages (RB * LB * D).
constexpr int MAX_REAL_ROWS = 64;
// Most lanes (pencils per component) of a compile-time strided tile: 2 in
// 2D, 4 in 3D (ct_max_lanes in hg_internal.h, shared with the host's choice).
static_assert(CT_THREADS == CT_THREADS_HOST, "host launch geometry and device tiling disagree");

// The step of a CG iteration from val = (p, A p) (the last CTA of the forward
// pass, thread 0): alpha = (r, r) / (p, A p) (Sec. 5.3, Eq. CG_identity);
// Moulinec-Suquet takes the fixed step 1 / lambda.
__device__ __forceinline__ void fwd_cg_scalars(Scalars& s, double val) {
    s.pt = val;
    if (s.fixed_alpha > 0.0 && s.rr == 0.0) {
        // Moulinec-Suquet reached the fixed point exactly: the step from r = 0
        // is zero
        s.status = ST_CONVERGED;
        s.alpha = 0.0;
    } else if (!(val > 0.0) || !isfinite(val)) {
        s.status = ST_BREAKDOWN;
        s.alpha = 0.0;
    } else {
        s.alpha = s.fixed_alpha > 0.0 ? s.fixed_alpha : s.rr / val;
    }
    s.alpha_f = (float)s.alpha;
}

// The end of a CG iteration from rr = (r, r) of the updated residual (the last
// CTA of the inverse pass, thread 0): iteration count, relative residual,
// stopping tests, beta = (r, r) / (r, r)_old.
__device__ __forceinline__ void inv_cg_scalars(Scalars& s, double rr) {
    s.iters += 1;
    s.total_iters += 1;
    const double rel = sqrt(rr) / s.bnorm;
    s.relres = rel;
    // Moulinec-Suquet stops on the step just taken, x_{i+1} - x_i = r_i /
    // lambda, i.e. on the residual before this update (the tolerance was
    // rescaled by lambda / ||b|| at the right-hand side)
    const double crit = s.fixed_alpha > 0.0 ? sqrt(s.rr) / s.bnorm : rel;
    if (!isfinite(rr)) s.status = ST_BREAKDOWN;
    else if (crit <= s.tol) s.status = ST_CONVERGED;
    else if (s.iters >= s.max_iter) s.status = ST_MAXITER;
    if (s.stall_max > 0 && s.status == ST_ACTIVE) {
        if (rr < 0.25 * s.best_rr) {
            s.best_rr = rr;
            s.stall = 0;
        } else if (++s.stall >= s.stall_max) {
            s.status = ST_STAGNATED;
        }
    }
    s.beta = s.fixed_alpha > 0.0 ? 0.0 : rr / s.rr;   // MS: p = r
    s.beta_f = (float)s.beta;
    s.rr = rr;
}

// Offset of the half-spectrum row of real row rr (-1: none) for a row tile:
// real row rr = (rowi * nl + li) * D + al holds component al of load l0 + li
// on spatial row row0 + rowi.
template <int D>
__device__ __forceinline__ void row_offsets(long long* s_off, int nreal, int nl, int l0, long long row0,
                                            int nrow, const int* s_act, long long rows, int H) {
    for (int rr = threadIdx.x; rr < nreal; rr += blockDim.x) {
        const int rowi = rr / (nl * D);
        const int li = (rr / D) % nl;
        const int al = rr % D;
        s_off[rr] = (rowi < nrow && s_act[li]) ? ((((long long)(l0 + li) * D + al) * rows + row0 + rowi) * H) : -1;
    }
}

// ---------------------------------------------------------------------------
// last-axis forward pass (prologue + real-to-complex DFT)
// ---------------------------------------------------------------------------
template <typename T, int D, int NN, typename Args = RowFwdArgs>
__device__ __forceinline__ void row_fwd_body(GridDev g, AxisPlanH pl, const Cx<T>* __restrict__ tw,
                                             Args a, int RB, int LB, TileIdx ti) {
    typedef Cx<T> C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int Nl = NN > 0 ? NN : g.Nl;
    const int H = (Nl + 1) >> 1;
    const long long M = g.M, rows = g.rows;
    const long long row0 = (long long)ti.x * RB;
    const int nrow = (int)min((long long)RB, rows - row0);
    const int l0 = ti.y * LB;
    const int nl = min(LB, a.L - l0);
    const int nreal = RB * nl * D;
    const int ncplx = (nreal + 1) >> 1;
    if (!a.early_stage) grid_dep_wait();
    const C* tws = stage_twiddles<T, NN>(buf + ncplx * Nl, pl, tw);

    __shared__ T s_beta[D];
    __shared__ int s_act[D];
    __shared__ T s_tab[SMEM_PHASES * D * D];
    __shared__ long long s_off[MAX_REAL_ROWS];
    const T* tab = stage_table<T, D>(a.co, s_tab);
    if (a.early_stage) grid_dep_wait();
    if (threadIdx.x < nl) {
        const Scalars& s = a.sc[l0 + threadIdx.x];
        s_act[threadIdx.x] = (!a.check_status) || (s.status == ST_ACTIVE);
        s_beta[threadIdx.x] = beta_of(s, T());
    }
    __shared__ int s_any;
    if (threadIdx.x == 0) {
        // a launch in which no system is ACTIVE (the tail of a graph chunk after
        // convergence) does no work; every CTA sees the same statuses, so none
        // of them takes a ticket and the counter stays at zero
        int any = 0;
        for (int l = 0; l < a.L; ++l) any |= (!a.check_status) || (a.sc[l].status == ST_ACTIVE);
        s_any = any;
    }
    __syncthreads();
    if (!s_any) return;
    row_offsets<D>(s_off, nreal, nl, l0, row0, nrow, s_act, rows, H);
    T beta_t[D];
    bool act[D];
#pragma unroll
    for (int li = 0; li < D; ++li) {
        act[li] = li < nl && s_act[li];
        beta_t[li] = li < nl ? s_beta[li] : T(0);
    }

    // tile bases: the RB rows of a tile are contiguous in memory; component
    // (li, al) of the tile starts (li D + al) M after these
    const long long kb = row0 * Nl;
    const bool cg = a.mode == FWD_CG;
    const long long b0 = (long long)l0 * D * M + kb;
    T* const Pt = cg ? static_cast<T*>(a.p) + b0 : nullptr;
    const T* const Rt = cg ? static_cast<const T*>(a.r) + b0 : (a.u ? static_cast<const T*>(a.u) + b0 : nullptr);
    const unsigned Mu = (unsigned)M;
    T Ev[D][D];
#pragma unroll
    for (int li = 0; li < D; ++li)
#pragma unroll
        for (int al = 0; al < D; ++al)
            Ev[li][al] = (a.has_E && li < nl) ? load_of(a, (l0 + li) * D + al, T()) : T(0);
    const uint8_t* phb = a.co.phase ? a.co.phase + kb : nullptr;
    CoeffsDev co = a.co;     // phase map / packed field shifted to the tile
    co.phase = phb;
    if (co.mode == 1) co.field = static_cast<const T*>(a.co.field) + kb;

    // per-thread partial sums in T over this thread's voxels, FP64 above the warp
    T tacc[MAXL] = {T(0), T(0), T(0)};
    const int total = nrow * Nl;
    constexpr int UNR = D == 2 ? 2 : 1;   // loads in flight vs registers (3D is register-bound)
    for (int e0 = threadIdx.x; e0 < RB * Nl; e0 += UNR * blockDim.x) {
        T vv[UNR][D][D];
        T pp[UNR][D][D];
        T am[UNR][D][D];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const int e = e0 + u * blockDim.x;
            const bool valid = e < total;
            if (valid) load_coeffs<T, D>(co, e, M, am[u], tab);
#pragma unroll
            for (int li = 0; li < D; ++li) {
                if (li >= nl) break;
                const bool on = valid && act[li];
#pragma unroll
                for (int al = 0; al < D; ++al) {
                    const size_t o = (size_t)(li * D + al) * Mu + e;
                    vv[u][li][al] = (on && Rt) ? Rt[o] : T(0);
                    pp[u][li][al] = (on && cg) ? Pt[o] : T(0);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e >= RB * Nl) break;
            const bool valid = e < total;
            const int rowi = e / Nl;
            const int i = e - rowi * Nl;
#pragma unroll
            for (int li = 0; li < D; ++li) {
                if (li >= nl) break;
                T t[D];
#pragma unroll
                for (int al = 0; al < D; ++al) t[al] = T(0);
                if (valid && act[li]) {
                    T v[D];
#pragma unroll
                    for (int al = 0; al < D; ++al) {
                        if (cg) {
                            v[al] = vv[u][li][al] + beta_t[li] * pp[u][li][al];
                            Pt[(size_t)(li * D + al) * Mu + e] = v[al];
                        } else {
                            v[al] = vv[u][li][al] + Ev[li][al];
                        }
                    }
#pragma unroll
                    for (int al = 0; al < D; ++al) {
                        T sacc = T(0);
#pragma unroll
                        for (int be = 0; be < D; ++be) sacc += am[u][al][be] * v[be];
                        t[al] = sacc;
                    }
                    if (!cg && a.A0) {
                        T w[D];
#pragma unroll
                        for (int al = 0; al < D; ++al) {
                            T sacc = T(0);
#pragma unroll
                            for (int be = 0; be < D; ++be) sacc += (T)a.A0[al * D + be] * t[be];
                            w[al] = sacc;
                        }
#pragma unroll
                        for (int al = 0; al < D; ++al) t[al] = w[al];
                    }
#pragma unroll
                    for (int al = 0; al < D; ++al) tacc[li] += cg ? v[al] * t[al] : t[al] * t[al];
                }
#pragma unroll
                for (int al = 0; al < D; ++al) {
                    const int rr = (rowi * nl + li) * D + al;
                    C* z = &buf[(rr >> 1) * Nl + i];
                    if (rr & 1) z->y = t[al]; else z->x = t[al];
                }
            }
        }
    }
    if (nreal & 1)
        for (int i = threadIdx.x; i < Nl; i += blockDim.x) buf[(ncplx - 1) * Nl + i].y = T(0);
    __syncthreads();

    fft_any<T, NN, false>(buf, ncplx, Nl, pl, tw, tws);
    grid_dep_launch();

    // Separate the packed pairs: Z = a + i b  ->  A(k) = (Z(k) + conj Z(-k))/2,
    // B(k) = (Z(k) - conj Z(-k)) / 2i, for k = 0..H-1 (Hermitian half).
    C* __restrict__ S = static_cast<C*>(a.S);
    for (int e = threadIdx.x; e < ncplx * H; e += blockDim.x) {
        const int c = e / H;
        const int kk = e - c * H;
        const C z = buf[c * Nl + kk];
        const C zm = buf[c * Nl + (kk ? Nl - kk : 0)];
        const long long o0 = s_off[2 * c];
        const long long o1 = (2 * c + 1 < nreal) ? s_off[2 * c + 1] : -1;
        if (o0 >= 0) {
            C A;
            A.x = T(0.5) * (z.x + zm.x); A.y = T(0.5) * (z.y - zm.y);
            S[o0 + kk] = A;
        }
        if (o1 >= 0) {
            C B;
            B.x = T(0.5) * (z.y + zm.y); B.y = T(0.5) * (zm.x - z.x);
            S[o1 + kk] = B;
        }
    }

    // reductions
    double acc[MAXL];
    block_sum_t<T, MAXL>(tacc, acc);
    const long long nbx = ti.nx;
    const unsigned nblocks = ti.nx * ti.ny;
    int slots[MAXL];
    for (int li = 0; li < nl; ++li) slots[li] = l0 + li;
    const bool last = publish(acc, slots, nl, a.partial, nbx, ti.x, a.counter, nblocks);
    if (!last) return;
    double tot[MAXL];
    final_sums<MAXL, T>(a.partial, nbx, nbx, a.L, tot);
    if (threadIdx.x == 0) {
        for (int l = 0; l < a.L; ++l) {
            Scalars& s = a.sc[l];
            const double val = tot[l] * g.invM;
            if (a.mode == FWD_CG) {
                if (a.check_status && s.status != ST_ACTIVE) continue;
                fwd_cg_scalars(s, val);
            } else {
                s.aen = sqrt(val);
            }
        }
        *a.counter = 0u;
    }
}

template <typename T, int D, int NN>
__global__ void __launch_bounds__(PassThreads<NN>::v) k_row_fwd(GridDev g, AxisPlanH pl,
                                                               const Cx<T>* __restrict__ tw,
                                                               RowFwdArgs a, int RB, int LB) {
    row_fwd_body<T, D, NN>(g, pl, tw, a, RB, LB, TileIdx::of_block());
}


// ---------------------------------------------------------------------------
// strided-axis pass (complex DFT along one axis; Fourier projection on axis 0)
// ---------------------------------------------------------------------------
template <typename T, int D, int NN, typename Args = StrArgs>
__device__ __forceinline__ void strided_body(GridDev g, AxisPlanH pl, const Cx<T>* __restrict__ tw,
                                             Args a, int Cl, TileIdx ti) {
    typedef Cx<T> C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const long long i0 = (long long)ti.x * Cl;
    const long long o = ti.y;
    const int l = ti.z;
    const int n = NN > 0 ? NN : a.n;
    const int inner = (int)a.inner;
    if (!a.early_stage) grid_dep_wait();
    const C* tws = stage_twiddles<T, NN>(buf + D * Cl * n, pl, tw);
    if (a.early_stage) grid_dep_wait();
    if (a.check_status && a.sc[l].status != ST_ACTIVE) return;

    // Cl is a power of two dividing blockDim.x: each thread keeps one lane and
    // walks the (component, position) rows with stride blockDim.x / Cl.
    const int lane = threadIdx.x & (Cl - 1);
    const int rstep = blockDim.x / Cl;
    const bool lane_ok = i0 + lane < inner;
    const int lgCl = 31 - __clz(Cl);
    // shared layout: compile-time kernels interleave the lanes
    // ([component][position][lane]); the runtime kernel keeps pencils contiguous
    auto sidx = [&](int al, int m) -> int {
        return NN > 0 ? (al * n + m) * Cl + lane : (al * Cl + lane) * n + m;
    };
    C* Sb = static_cast<C*>(a.S) + (long long)l * D * g.Ms + o * (long long)n * inner + i0 + lane;
    const long long cstride = g.Ms;
    if constexpr (NN > 0) {
        // Every load of the thread is issued before the first shared-memory
        // store (a store through a generic pointer would otherwise keep the
        // next global load behind it): one memory latency per tile instead of
        // one per few rows.  At most ct_max_lanes(D) lanes, so KL bounds the rows
        // (a bound above the rows actually held costs registers and time).
        constexpr int KL = (D * NN * ct_max_lanes(D) + CT_THREADS - 1) / CT_THREADS;
        C v[KL];
#pragma unroll
        for (int k = 0; k < KL; ++k) {
            const int row = threadIdx.x / Cl + k * rstep;
            const int al = row / n;
            const int m = row - al * n;
            v[k] = (lane_ok && row < D * n) ? Sb[al * cstride + m * inner] : czero<T>();
        }
#pragma unroll
        for (int k = 0; k < KL; ++k) {
            const int row = threadIdx.x / Cl + k * rstep;
            if (row < D * n) {
                const int al = row / n;
                buf[sidx(al, row - al * n)] = v[k];
            }
        }
    } else {
#pragma unroll 4
        for (int row = threadIdx.x / Cl; row < D * n; row += rstep) {
            const int al = row / n;
            const int m = row - al * n;
            C v = czero<T>();
            if (lane_ok) v = Sb[al * cstride + m * inner];
            buf[sidx(al, m)] = v;
        }
    }
    __syncthreads();

    if (a.mode != STR_INV) fft_str<T, D, NN, false>(buf, Cl, lgCl, n, pl, tw, tws);

    if (a.mode == STR_FWD_SCALE) {
        const T sc = inv_m(g, T());
        for (int e = threadIdx.x; e < D * Cl * n; e += blockDim.x) buf[e] = cscale(buf[e], sc);
        __syncthreads();
    } else if (a.mode == STR_GAMMA) {
        // q_hat = xi (xi . t_hat) / (xi . A0 xi) / |N| with t = A0 A u (Eq. Gamma_hat,
        // G = Gamma A0); A0 = I unless has_A0.  Computed in T.
        const int i = (int)i0 + lane;     // < inner < 2^31
        T xi_rest[D];        // the components of xi fixed by this lane
        xi_rest[0] = T(0);
        if (lane_ok) {
            if (D == 2) {
                xi_rest[1] = (T)i * inv_y(g, 1, T());
            } else {
                const int k2 = i % g.H;
                const int k1 = i / g.H;
                xi_rest[1] = (T)freq_of(k1, g.N[1]) * inv_y(g, 1, T());
                xi_rest[D - 1] = (T)k2 * inv_y(g, D - 1, T());
            }
        }
        // Galerkin scheme with exact integration: the trial space is the band
        // |m_a| <= (band_a - 1) / 2 of this grid's frequencies; no output
        // outside it
        bool lane_band = true;
        if (a.band[0] > 0 && lane_ok) {
            if (D == 2) {
                lane_band = i <= (a.band[1] - 1) / 2;
            } else {
                const int f1 = freq_of(i / g.H, g.N[1]);
                lane_band = f1 <= (a.band[1] - 1) / 2 && -f1 <= (a.band[1] - 1) / 2 &&
                            i % g.H <= (a.band[D - 1] - 1) / 2;
            }
        }
        const int mb = a.band[0] > 0 ? (a.band[0] - 1) / 2 : n;
        const T invY0 = inv_y(g, 0, T());
        const T invM = inv_m(g, T());
        // the row's frequency in T, stepped with the row (integers below 2^24
        // are exact in FP32): one integer-to-float conversion per thread, not
        // one per frequency (conversions run on the slow FP64 pipe)
        const int m_first = threadIdx.x / Cl;
        const int half = (n - 1) >> 1;
        const T stepf = (T)rstep, nf = (T)n;
        T mf = (T)m_first;
        for (int m = m_first; m < n && lane_ok; m += rstep, mf += stepf) {
            T xi[D];
            xi[0] = (m <= half ? mf : mf - nf) * invY0;
#pragma unroll
            for (int al = 1; al < D; ++al) xi[al] = xi_rest[al];
            C th[D];
#pragma unroll
            for (int al = 0; al < D; ++al) th[al] = buf[sidx(al, m)];
            T den = T(0);
            C num = czero<T>();
            if (a.has_A0) {
#pragma unroll
                for (int al = 0; al < D; ++al) {
                    T axi = T(0);
#pragma unroll
                    for (int be = 0; be < D; ++be) axi += (T)a.A0[al * D + be] * xi[be];
                    den += xi[al] * axi;
                    num.x += xi[al] * th[al].x;
                    num.y += xi[al] * th[al].y;
                }
            } else {
#pragma unroll
                for (int al = 0; al < D; ++al) {
                    den += xi[al] * xi[al];
                    num.x += xi[al] * th[al].x;
                    num.y += xi[al] * th[al].y;
                }
            }
            const int fm = m <= half ? m : m - n;
            const bool inb = lane_band && fm <= mb && -fm <= mb;
            C s = czero<T>();
            if (den > T(0) && inb) {
                const T f = div_proj(invM, den);
                s.x = num.x * f;
                s.y = num.y * f;
            }
            if (a.dual) {
                // onto J_N: t_hat - xi (xi . t_hat) / |xi|^2 away from k = 0, and
                // nothing of the mean (Eq. Helmholtz_discrete)
#pragma unroll
                for (int al = 0; al < D; ++al) {
                    C q = czero<T>();
                    if (den > T(0) && inb) {
                        q.x = th[al].x * invM - s.x * xi[al];
                        q.y = th[al].y * invM - s.y * xi[al];
                    }
                    buf[sidx(al, m)] = q;
                }
            } else {
#pragma unroll
                for (int al = 0; al < D; ++al) buf[sidx(al, m)] = cscale(s, xi[al]);
            }
        }
        __syncthreads();
        fft_str<T, D, NN, true>(buf, Cl, lgCl, n, pl, tw, tws);
    } else if (a.mode == STR_INV) {
        fft_str<T, D, NN, true>(buf, Cl, lgCl, n, pl, tw, tws);
    }

    grid_dep_launch();
    if (lane_ok) {
#pragma unroll 4
        for (int row = threadIdx.x / Cl; row < D * n; row += rstep) {
            const int al = row / n;
            const int m = row - al * n;
            Sb[al * cstride + m * inner] = buf[sidx(al, m)];
        }
    }
}

template <typename T, int D, int NN>
__global__ void __launch_bounds__(PassThreads<NN>::v, StridedMinBlocks<T, D, NN>::v) k_strided(GridDev g, AxisPlanH pl,
                                                               const Cx<T>* __restrict__ tw,
                                                               StrArgs a, int Cl) {
    strided_body<T, D, NN>(g, pl, tw, a, Cl, TileIdx::of_block());
}


// ---------------------------------------------------------------------------
// last-axis inverse pass (complex-to-real DFT + CG update)
// ---------------------------------------------------------------------------
template <typename T, int D, int NN, typename Args = RowInvArgs>
__device__ __forceinline__ void row_inv_body(GridDev g, AxisPlanH pl, const Cx<T>* __restrict__ tw,
                                             Args a, int RB, int LB, TileIdx ti) {
    typedef Cx<T> C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int Nl = NN > 0 ? NN : g.Nl;
    const int H = (Nl + 1) >> 1;
    const long long M = g.M, rows = g.rows;
    const long long row0 = (long long)ti.x * RB;
    const int nrow = (int)min((long long)RB, rows - row0);
    const int l0 = ti.y * LB;
    const int nl = min(LB, a.L - l0);
    const int nreal = RB * nl * D;
    const int ncplx = (nreal + 1) >> 1;
    if (!a.early_stage) grid_dep_wait();
    const C* tws = stage_twiddles<T, NN>(buf + ncplx * Nl, pl, tw);

    __shared__ T s_alpha[D];
    __shared__ int s_act[D];
    __shared__ long long s_off[MAX_REAL_ROWS];
    __shared__ int s_any;
    if (a.early_stage) grid_dep_wait();
    if (threadIdx.x < nl) {
        const Scalars& s = a.sc[l0 + threadIdx.x];
        s_act[threadIdx.x] = (!a.check_status) || (s.status == ST_ACTIVE);
        s_alpha[threadIdx.x] = alpha_of(s, T());
    }
    if (threadIdx.x == 0) {
        int any = 0;   // see k_row_fwd: a launch with no ACTIVE system does nothing
        for (int l = 0; l < a.L; ++l) any |= (!a.check_status) || (a.sc[l].status == ST_ACTIVE);
        s_any = any;
    }
    __syncthreads();
    if (!s_any) return;
    row_offsets<D>(s_off, nreal, nl, l0, row0, nrow, s_act, rows, H);
    __syncthreads();

    // Rebuild two real rows a, b as one complex row Z = a + i b from their
    // Hermitian half spectra: X(k) for k >= H is conj X(Nl - k).
    const C* __restrict__ S = static_cast<const C*>(a.S);
    // KB elements per thread are loaded before any is stored (see k_strided)
    constexpr int KB = (sizeof(T) == 4 && D == 3) ? 8 : 4;
    for (int e0 = threadIdx.x; e0 < ncplx * Nl; e0 += KB * blockDim.x) {
        C v0[KB], v1[KB];
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            const int e = e0 + u * blockDim.x;
            v0[u] = czero<T>();
            v1[u] = czero<T>();
            if (e < ncplx * Nl) {
                const int c = e / Nl;
                const int kk = e - c * Nl;
                const int ks = kk >= H ? Nl - kk : kk;
                const long long o0 = s_off[2 * c];
                const long long o1 = (2 * c + 1 < nreal) ? s_off[2 * c + 1] : -1;
                if (o0 >= 0) v0[u] = S[o0 + ks];
                if (o1 >= 0) v1[u] = S[o1 + ks];
            }
        }
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < ncplx * Nl) {
                const int c = e / Nl;
                const int kk = e - c * Nl;
                if (kk >= H) { v0[u].y = -v0[u].y; v1[u].y = -v1[u].y; }
                C z;
                z.x = v0[u].x - v1[u].y;
                z.y = v0[u].y + v1[u].x;
                buf[c * Nl + kk] = z;
            }
        }
    }
    __syncthreads();

    fft_any<T, NN, true>(buf, ncplx, Nl, pl, tw, tws);
    grid_dep_launch();

    const long long b0 = (long long)l0 * D * M + row0 * Nl;
    T* const Xt = a.x ? static_cast<T*>(a.x) + b0 : nullptr;
    T* const Rt = a.r ? static_cast<T*>(a.r) + b0 : nullptr;
    T* const Pt = a.p ? static_cast<T*>(a.p) + b0 : nullptr;
    T* const Ot = a.out ? static_cast<T*>(a.out) + b0 : nullptr;
    const unsigned Mu = (unsigned)M;
    T alpha_t[D];
    bool act[D];
#pragma unroll
    for (int li = 0; li < D; ++li) {
        act[li] = li < nl && s_act[li];
        alpha_t[li] = li < nl ? s_alpha[li] : T(0);
    }
    T tacc[MAXL] = {T(0), T(0), T(0)};
    T Wt[D * D];
#pragma unroll
    for (int i = 0; i < D * D; ++i) Wt[i] = weight_of(a.W, i, T());
    constexpr int UNR = D == 2 ? 2 : 1;
    const int total = nrow * Nl;
    const bool cgm = a.mode == INV_CG;
    for (int e0 = threadIdx.x; e0 < total; e0 += UNR * blockDim.x) {
        T xv[UNR][D][D], rv0[UNR][D][D], pv[UNR][D][D];
        if (cgm) {
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const int e = e0 + u * blockDim.x;
                const bool valid = e < total;
#pragma unroll
                for (int li = 0; li < D; ++li) {
                    if (li >= nl) break;
                    const bool on = valid && act[li];
#pragma unroll
                    for (int al = 0; al < D; ++al) {
                        const size_t o = (size_t)(li * D + al) * Mu + e;
                        xv[u][li][al] = on ? Xt[o] : T(0);
                        rv0[u][li][al] = on ? Rt[o] : T(0);
                        pv[u][li][al] = on ? Pt[o] : T(0);
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e >= total) break;
            const int rowi = e / Nl;
            const int i = e - rowi * Nl;
#pragma unroll
            for (int li = 0; li < D; ++li) {
                if (li >= nl) break;
                if (!act[li]) continue;
                T rn[D];
#pragma unroll
                for (int al = 0; al < D; ++al) {
                    const int rr = (rowi * nl + li) * D + al;
                    const C z = buf[(rr >> 1) * Nl + i];
                    const T q = (rr & 1) ? z.y : z.x;
                    const size_t o = (size_t)(li * D + al) * Mu + e;
                    rn[al] = T(0);
                    if (cgm) {
                        Xt[o] = xv[u][li][al] + alpha_t[li] * pv[u][li][al];
                        rn[al] = rv0[u][li][al] - alpha_t[li] * q;
                        Rt[o] = rn[al];
                    } else if (a.mode == INV_RHS) {
                        rn[al] = -q;
                        Rt[o] = rn[al];
                        Pt[o] = rn[al];
                        Xt[o] = T(0);
                    } else if (a.mode == INV_RESID) {
                        rn[al] = -q;
                        Rt[o] = rn[al];
                    } else if (a.mode == INV_PROJ) {
                        Xt[o] = q;             // x <- Gamma x
                    } else {
                        Ot[o] = q;
                    }
                }
                // (r, r) in the scalar product of the iteration, (W r, r)
#pragma unroll
                for (int al = 0; al < D; ++al) {
                    T wr = rn[al];
                    if (a.W.has) {
                        wr = T(0);
#pragma unroll
                        for (int be = 0; be < D; ++be) wr += Wt[al * D + be] * rn[be];
                    }
                    tacc[li] += rn[al] * wr;
                }
            }
        }
    }

    if (a.mode == INV_OUT || a.mode == INV_PROJ) return;
    double acc[MAXL];
    block_sum_t<T, MAXL>(tacc, acc);
    const long long nbx = ti.nx;
    const unsigned nblocks = ti.nx * ti.ny;
    int slots[MAXL];
    for (int li = 0; li < nl; ++li) slots[li] = l0 + li;
    const bool last = publish(acc, slots, nl, a.partial, nbx, ti.x, a.counter, nblocks);
    if (!last) return;
    double tot[MAXL];
    final_sums<MAXL, T>(a.partial, nbx, nbx, a.L, tot);
    if (threadIdx.x == 0) {
        for (int l = 0; l < a.L; ++l) {
            Scalars& s = a.sc[l];
            if (a.check_status && s.status != ST_ACTIVE) continue;
            const double rr = tot[l] * g.invM;
            if (a.mode == INV_CG) {
                inv_cg_scalars(s, rr);
            } else if (a.mode == INV_RHS) {
                s.rr = rr;
                s.bnorm = sqrt(rr);
                s.beta = 0.0;
                s.beta_f = 0.f;
                s.iters = 0;
                s.relres = 1.0;
                // b = -G A E vanishes in exact arithmetic when A E is constant
                // along every direction G keeps (G kills constants, Lemma
                // FD_projection (iv)); ||b|| <= ||A E|| since G is an
                // orthogonal projection (zscale = 1; for a general reference
                // medium ||b||_A0 <= sqrt(lmax) / lmin ||A E|| = zscale ||A E||),
                // so a ratio at roundoff level is zero.
                if (sizeof(T) == 4 && !(s.bnorm > RHS32_RECHECK * s.zscale * s.aen)) {
                    s.status = ST_RHS_RECHECK;
                } else if (!(s.bnorm > ZERO_RHS * s.zscale * s.aen)) {
                    s.status = ST_ZERO_RHS;
                    s.relres = 0.0;
                } else if (s.fixed_alpha > 0.0) {
                    // Moulinec-Suquet: ||e_{i+1} - e_i|| = ||r_i|| / lambda with
                    // ||E|| = 1 for a unit load, so ||e_{i+1} - e_i|| / ||E||
                    // <= tol  <=>  ||r_i|| / ||b|| <= tol lambda / ||b||
                    s.tol = s.tol / (s.fixed_alpha * s.bnorm);
                }
            } else {  // INV_RESID
                s.relres = sqrt(rr) / s.bnorm;
                if (!isfinite(rr)) s.status = ST_BREAKDOWN;
                else if (s.relres <= s.tol) s.status = ST_CONVERGED;
            }
        }
        *a.counter = 0u;
    }
}

template <typename T, int D, int NN>
__global__ void __launch_bounds__(PassThreads<NN>::v) k_row_inv(GridDev g, AxisPlanH pl,
                                                               const Cx<T>* __restrict__ tw,
                                                               RowInvArgs a, int RB, int LB) {
    row_inv_body<T, D, NN>(g, pl, tw, a, RB, LB, TileIdx::of_block());
}


// ---------------------------------------------------------------------------
// batched passes: P problems of one grid shape in one launch
// ---------------------------------------------------------------------------
// The arguments of problem p (its coefficients, vectors, scalars, reduction
// slots and tickets) are items[p] in device memory; the grid's z index picks
// the problem (strided: z = problem * L + load).  Twiddles and launch geometry
// are those of the shared shape.
// The arguments of this CTA's problem, copied once per CTA from the device
// array into shared memory: the pass body then reads them (some fields with
// run-time indices, e.g. the loads E) from shared memory, where a by-value
// copy of a global struct would be a per-thread copy in local memory.
// Items are written by the host before the launch, never by the previous
// kernel, so the copy may precede the programmatic-dependency wait.
template <typename Args>
__device__ __forceinline__ const Args& stage_item(const Args* __restrict__ items, int p) {
    static_assert(sizeof(Args) % 4 == 0 && sizeof(Args) <= 4 * 64 * 32, "item larger than the copy loop");
    __shared__ __align__(16) unsigned char raw[sizeof(Args)];
    const unsigned* src = reinterpret_cast<const unsigned*>(items + p);
    unsigned* dst = reinterpret_cast<unsigned*>(raw);
    for (int i = threadIdx.x; i < (int)(sizeof(Args) / 4); i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
    return *reinterpret_cast<const Args*>(raw);
}

template <typename T, int D, int NN>
__global__ void __launch_bounds__(PassThreads<NN>::v) k_row_fwd_b(GridDev g, AxisPlanH pl,
                                                                 const Cx<T>* __restrict__ tw,
                                                                 const RowFwdArgs* __restrict__ items,
                                                                 int RB, int LB) {
    row_fwd_body<T, D, NN, const RowFwdArgs&>(g, pl, tw, stage_item(items, blockIdx.z), RB, LB,
                                              TileIdx::of_block());
}

template <typename T, int D, int NN>
__global__ void __launch_bounds__(PassThreads<NN>::v) k_row_inv_b(GridDev g, AxisPlanH pl,
                                                                 const Cx<T>* __restrict__ tw,
                                                                 const RowInvArgs* __restrict__ items,
                                                                 int RB, int LB) {
    row_inv_body<T, D, NN, const RowInvArgs&>(g, pl, tw, stage_item(items, blockIdx.z), RB, LB,
                                              TileIdx::of_block());
}

template <typename T, int D, int NN>
__global__ void __launch_bounds__(PassThreads<NN>::v, StridedMinBlocks<T, D, NN>::v)
k_strided_b(GridDev g, AxisPlanH pl, const Cx<T>* __restrict__ tw, const StrArgs* __restrict__ items, int Cl,
            int L) {
    TileIdx ti = TileIdx::of_block();
    ti.z = (int)blockIdx.z % L;
    strided_body<T, D, NN, const StrArgs&>(g, pl, tw, stage_item(items, (int)blockIdx.z / L), Cl, ti);
}

// ---------------------------------------------------------------------------
// per-precision launch dispatch (hg_kernels_f32.cu / hg_kernels_f64.cu)
// ---------------------------------------------------------------------------
// Transform lengths with compile-time kernels; every other length runs the
// runtime-plan kernels.
#define HG_CT_SIZES_2D(X) X(15) X(27) X(45) X(75) X(81) X(135) X(243) X(375) X(729)
#define HG_CT_SIZES_3D(X) X(15) X(27) X(45) X(81) X(135)

// Launch with programmatic stream serialization (see grid_dep_wait).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, int threads, int smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename T>
cudaError_t launch_row_fwd_t(const GridDev& g, const AxisPlanH& pl, const void* tw, const RowCfg& cfg,
                             const RowFwdArgs& a, cudaStream_t s) {
    cudaError_t le = cudaSuccess;
    dim3 grid((unsigned)cfg.nbx, (unsigned)((a.L + cfg.LB - 1) / cfg.LB));
    const Cx<T>* twp = (const Cx<T>*)tw;
#define HG_CASE2(NV) case NV: le = launch_pdl(k_row_fwd<T, 2, NV>, grid, CT_THREADS, cfg.smem, s, g, pl, twp, a, cfg.RB, cfg.LB); break;
#define HG_CASE3(NV) case NV: le = launch_pdl(k_row_fwd<T, 3, NV>, grid, CT_THREADS, cfg.smem, s, g, pl, twp, a, cfg.RB, cfg.LB); break;
    if (g.d == 2) {
        if (cfg.ct) {
            switch (g.Nl) {
                HG_CT_SIZES_2D(HG_CASE2)
                default: return cudaErrorInvalidConfiguration;   // no compile-time kernel
            }
        } else {
            le = launch_pdl(k_row_fwd<T, 2, 0>, grid, cfg.threads, cfg.smem, s, g, pl, twp, a, cfg.RB, cfg.LB);
        }
    } else {
        if (cfg.ct) {
            switch (g.Nl) {
                HG_CT_SIZES_3D(HG_CASE3)
                default: return cudaErrorInvalidConfiguration;   // no compile-time kernel
            }
        } else {
            le = launch_pdl(k_row_fwd<T, 3, 0>, grid, cfg.threads, cfg.smem, s, g, pl, twp, a, cfg.RB, cfg.LB);
        }
    }
#undef HG_CASE2
#undef HG_CASE3
    if (le != cudaSuccess) return le;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_row_inv_t(const GridDev& g, const AxisPlanH& pl, const void* tw, const RowCfg& cfg,
                             const RowInvArgs& a, cudaStream_t s) {
    cudaError_t le = cudaSuccess;
    dim3 grid((unsigned)cfg.nbx, (unsigned)((a.L + cfg.LB - 1) / cfg.LB));
    const Cx<T>* twp = (const Cx<T>*)tw;
#define HG_CASE2(NV) case NV: le = launch_pdl(k_row_inv<T, 2, NV>, grid, CT_THREADS, cfg.smem, s, g, pl, twp, a, cfg.RB, cfg.LB); break;
#define HG_CASE3(NV) case NV: le = launch_pdl(k_row_inv<T, 3, NV>, grid, CT_THREADS, cfg.smem, s, g, pl, twp, a, cfg.RB, cfg.LB); break;
    if (g.d == 2) {
        if (cfg.ct) {
            switch (g.Nl) {
                HG_CT_SIZES_2D(HG_CASE2)
                default: return cudaErrorInvalidConfiguration;   // no compile-time kernel
            }
        } else {
            le = launch_pdl(k_row_inv<T, 2, 0>, grid, cfg.threads, cfg.smem, s, g, pl, twp, a, cfg.RB, cfg.LB);
        }
    } else {
        if (cfg.ct) {
            switch (g.Nl) {
                HG_CT_SIZES_3D(HG_CASE3)
                default: return cudaErrorInvalidConfiguration;   // no compile-time kernel
            }
        } else {
            le = launch_pdl(k_row_inv<T, 3, 0>, grid, cfg.threads, cfg.smem, s, g, pl, twp, a, cfg.RB, cfg.LB);
        }
    }
#undef HG_CASE2
#undef HG_CASE3
    if (le != cudaSuccess) return le;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_strided_t(const GridDev& g, const AxisPlanH& pl, const void* tw, const StrCfg& cfg,
                             const StrArgs& a, cudaStream_t s) {
    cudaError_t le = cudaSuccess;
    dim3 grid((unsigned)((a.inner + cfg.Cl - 1) / cfg.Cl), (unsigned)a.outer, (unsigned)a.L);
    const Cx<T>* twp = (const Cx<T>*)tw;
#define HG_CASE2(NV) case NV: le = launch_pdl(k_strided<T, 2, NV>, grid, CT_THREADS, cfg.smem, s, g, pl, twp, a, cfg.Cl); break;
#define HG_CASE3(NV) case NV: le = launch_pdl(k_strided<T, 3, NV>, grid, CT_THREADS, cfg.smem, s, g, pl, twp, a, cfg.Cl); break;
    if (g.d == 2) {
        if (cfg.ct) {
            switch (a.n) {
                HG_CT_SIZES_2D(HG_CASE2)
                default: return cudaErrorInvalidConfiguration;   // no compile-time kernel
            }
        } else {
            le = launch_pdl(k_strided<T, 2, 0>, grid, cfg.threads, cfg.smem, s, g, pl, twp, a, cfg.Cl);
        }
    } else {
        if (cfg.ct) {
            switch (a.n) {
                HG_CT_SIZES_3D(HG_CASE3)
                default: return cudaErrorInvalidConfiguration;   // no compile-time kernel
            }
        } else {
            le = launch_pdl(k_strided<T, 3, 0>, grid, cfg.threads, cfg.smem, s, g, pl, twp, a, cfg.Cl);
        }
    }
#undef HG_CASE2
#undef HG_CASE3
    if (le != cudaSuccess) return le;
    return cudaGetLastError();
}

// Batched launchers (items in device memory, P problems, L loads each).
#define HG_BATCH_DISPATCH(KERN, GRID, ...)                                                         \
    do {                                                                                          \
        if (g.d == 2) {                                                                           \
            if (ct) {                                                                             \
                switch (len) {                                                                    \
                    HG_CT_SIZES_2D(HG_BCASE2)                                                     \
                    default: return cudaErrorInvalidConfiguration;                                \
                }                                                                                 \
            } else {                                                                              \
                le = launch_pdl(KERN<T, 2, 0>, GRID, threads_rt, smem, s, __VA_ARGS__);            \
            }                                                                                     \
        } else {                                                                                  \
            if (ct) {                                                                             \
                switch (len) {                                                                    \
                    HG_CT_SIZES_3D(HG_BCASE3)                                                     \
                    default: return cudaErrorInvalidConfiguration;                                \
                }                                                                                 \
            } else {                                                                              \
                le = launch_pdl(KERN<T, 3, 0>, GRID, threads_rt, smem, s, __VA_ARGS__);            \
            }                                                                                     \
        }                                                                                         \
    } while (0)

template <typename T>
cudaError_t launch_row_fwd_batch_t(const GridDev& g, const AxisPlanH& pl, const void* tw, const RowCfg& cfg,
                                   const RowFwdArgs* items, int P, int L, cudaStream_t s) {
    cudaError_t le = cudaSuccess;
    dim3 grid((unsigned)cfg.nbx, (unsigned)((L + cfg.LB - 1) / cfg.LB), (unsigned)P);
    const Cx<T>* twp = (const Cx<T>*)tw;
    const int ct = cfg.ct, len = g.Nl, threads_rt = cfg.threads, smem = cfg.smem;
#define HG_BCASE2(NV) case NV: le = launch_pdl(k_row_fwd_b<T, 2, NV>, grid, CT_THREADS, smem, s, g, pl, twp, items, cfg.RB, cfg.LB); break;
#define HG_BCASE3(NV) case NV: le = launch_pdl(k_row_fwd_b<T, 3, NV>, grid, CT_THREADS, smem, s, g, pl, twp, items, cfg.RB, cfg.LB); break;
    HG_BATCH_DISPATCH(k_row_fwd_b, grid, g, pl, twp, items, cfg.RB, cfg.LB);
#undef HG_BCASE2
#undef HG_BCASE3
    if (le != cudaSuccess) return le;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_row_inv_batch_t(const GridDev& g, const AxisPlanH& pl, const void* tw, const RowCfg& cfg,
                                   const RowInvArgs* items, int P, int L, cudaStream_t s) {
    cudaError_t le = cudaSuccess;
    dim3 grid((unsigned)cfg.nbx, (unsigned)((L + cfg.LB - 1) / cfg.LB), (unsigned)P);
    const Cx<T>* twp = (const Cx<T>*)tw;
    const int ct = cfg.ct, len = g.Nl, threads_rt = cfg.threads, smem = cfg.smem;
#define HG_BCASE2(NV) case NV: le = launch_pdl(k_row_inv_b<T, 2, NV>, grid, CT_THREADS, smem, s, g, pl, twp, items, cfg.RB, cfg.LB); break;
#define HG_BCASE3(NV) case NV: le = launch_pdl(k_row_inv_b<T, 3, NV>, grid, CT_THREADS, smem, s, g, pl, twp, items, cfg.RB, cfg.LB); break;
    HG_BATCH_DISPATCH(k_row_inv_b, grid, g, pl, twp, items, cfg.RB, cfg.LB);
#undef HG_BCASE2
#undef HG_BCASE3
    if (le != cudaSuccess) return le;
    return cudaGetLastError();
}

// n, inner, outer: the axis and tiling of this strided pass (as in StrArgs).
template <typename T>
cudaError_t launch_strided_batch_t(const GridDev& g, const AxisPlanH& pl, const void* tw, const StrCfg& cfg,
                                   const StrArgs* items, int P, int L, int n, long long inner,
                                   long long outer, cudaStream_t s) {
    cudaError_t le = cudaSuccess;
    dim3 grid((unsigned)((inner + cfg.Cl - 1) / cfg.Cl), (unsigned)outer, (unsigned)(L * P));
    const Cx<T>* twp = (const Cx<T>*)tw;
    const int ct = cfg.ct, len = n, threads_rt = cfg.threads, smem = cfg.smem;
#define HG_BCASE2(NV) case NV: le = launch_pdl(k_strided_b<T, 2, NV>, grid, CT_THREADS, smem, s, g, pl, twp, items, cfg.Cl, L); break;
#define HG_BCASE3(NV) case NV: le = launch_pdl(k_strided_b<T, 3, NV>, grid, CT_THREADS, smem, s, g, pl, twp, items, cfg.Cl, L); break;
    HG_BATCH_DISPATCH(k_strided_b, grid, g, pl, twp, items, cfg.Cl, L);
#undef HG_BCASE2
#undef HG_BCASE3
    if (le != cudaSuccess) return le;
    return cudaGetLastError();
}
#undef HG_BATCH_DISPATCH

template <typename T>
cudaError_t configure_t(int max_smem, const double* ctw) {
    cudaError_t e = cudaSuccess;
    {
        double2 w64[CTW_TOTAL];
        float2 w32[CTW_TOTAL];
        for (int i = 0; i < CTW_TOTAL; ++i) {
            w64[i] = make_double2(ctw[2 * i], ctw[2 * i + 1]);
            w32[i] = make_float2((float)ctw[2 * i], (float)ctw[2 * i + 1]);
        }
        e = cudaMemcpyToSymbol(c_ctw64, w64, sizeof(w64));
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_ctw32, w32, sizeof(w32));
        if (e != cudaSuccess) return e;
    }
#define HG_SET(...)                                                                                        \
    do {                                                                                                   \
        cudaError_t e2 = cudaFuncSetAttribute(__VA_ARGS__, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem); \
        if (e2 != cudaSuccess) e = e2;                                                                     \
    } while (0)
#define HG_SET2(NV) HG_SET(k_row_fwd<T, 2, NV>); HG_SET(k_row_inv<T, 2, NV>); HG_SET(k_strided<T, 2, NV>); \
    HG_SET(k_row_fwd_b<T, 2, NV>); HG_SET(k_row_inv_b<T, 2, NV>); HG_SET(k_strided_b<T, 2, NV>);
#define HG_SET3(NV) HG_SET(k_row_fwd<T, 3, NV>); HG_SET(k_row_inv<T, 3, NV>); HG_SET(k_strided<T, 3, NV>); \
    HG_SET(k_row_fwd_b<T, 3, NV>); HG_SET(k_row_inv_b<T, 3, NV>); HG_SET(k_strided_b<T, 3, NV>);
    HG_SET2(0) HG_SET3(0)
    HG_CT_SIZES_2D(HG_SET2)
    HG_CT_SIZES_3D(HG_SET3)
#undef HG_SET2
#undef HG_SET3
#undef HG_SET
    return e;
}

}  // namespace hgk
