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
template <int NV>
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
            if (s < nslots) v[s] += __ldcg(&partial[s * stride + b]);
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
template <typename T, int D>
__device__ __forceinline__ void load_coeffs(const CoeffsDev& co, long long k, long long M, T (&a)[D][D]) {
    if (co.mode == 0) {
        const T* tb = static_cast<const T*>(co.table) + (int)co.phase[k] * D * D;
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) a[i][j] = __ldg(&tb[i * D + j]);
    } else if (co.mode == 1) {
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

// Transform of `npen` staged pencils of length n (forward or inverse).
template <typename T, int NN, bool INV>
__device__ __forceinline__ void fft_any(Cx<T>* buf, int npen, int n, const AxisPlanH& pl,
                                        const Cx<T>* __restrict__ twg, const Cx<T>* tws) {
    if constexpr (NN > 0) fft_ct<T, NN, INV>(buf, npen, tws);
    else fft_pencils<T, INV, MAXB>(buf, npen, n, pl, twg);
}

// Twiddles of the compile-time kernels are staged in shared memory after the
// pencils (n entries); the runtime kernels read them from global memory.
template <typename T, int NN>
__device__ __forceinline__ Cx<T>* stage_twiddles(Cx<T>* smem_after, const AxisPlanH& pl,
                                                 const Cx<T>* __restrict__ twg) {
    if constexpr (NN > 0) {
        const Cx<T>* src = twg + pl.tw_off;
        for (int i = threadIdx.x; i < NN; i += blockDim.x) smem_after[i] = src[i];
        return smem_after;
    } else {
        return nullptr;
    }
}

template <int NN> struct PassThreads { static constexpr int v = NN > 0 ? CT_THREADS : MAXT; };

// ---------------------------------------------------------------------------
// last-axis forward pass (prologue + real-to-complex DFT)
// ---------------------------------------------------------------------------
template <typename T, int D, int NN>
__global__ void __launch_bounds__(PassThreads<NN>::v) k_row_fwd(GridDev g, AxisPlanH pl,
                                                               const Cx<T>* __restrict__ tw,
                                                               RowFwdArgs a, int RB, int LB) {
    typedef Cx<T> C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int Nl = NN > 0 ? NN : g.Nl;
    const int H = (Nl + 1) >> 1;
    const long long M = g.M, rows = g.rows;
    const long long row0 = (long long)blockIdx.x * RB;
    const int l0 = blockIdx.y * LB;
    const int nl = min(LB, a.L - l0);
    const int nreal = RB * nl * D;
    const int ncplx = (nreal + 1) >> 1;
    const C* tws = stage_twiddles<T, NN>(buf + ncplx * Nl, pl, tw);

    __shared__ double s_beta[MAXL];
    __shared__ int s_act[MAXL];
    if (threadIdx.x < nl) {
        const Scalars& s = a.sc[l0 + threadIdx.x];
        s_act[threadIdx.x] = (!a.check_status) || (s.status == ST_ACTIVE);
        s_beta[threadIdx.x] = s.beta;
    }
    __syncthreads();

    T* __restrict__ P = static_cast<T*>(a.p);
    const T* __restrict__ R = static_cast<const T*>(a.r);
    const T* __restrict__ U = static_cast<const T*>(a.u);
    double acc[MAXL] = {0.0, 0.0, 0.0};

    for (int e = threadIdx.x; e < RB * Nl; e += blockDim.x) {
        const int rowi = e / Nl;
        const int i = e - rowi * Nl;
        const long long grow = row0 + rowi;
        const bool valid = grow < rows;
        const long long k = grow * Nl + i;
        T am[D][D];
        if (valid) load_coeffs<T, D>(a.co, k, M, am);
#pragma unroll
        for (int li = 0; li < MAXL; ++li) {
            if (li >= nl) break;
            const int l = l0 + li;
            T t[D];
#pragma unroll
            for (int al = 0; al < D; ++al) t[al] = T(0);
            if (valid && s_act[li]) {
                T v[D];
                if (a.mode == FWD_CG) {
                    const T beta = (T)s_beta[li];
#pragma unroll
                    for (int al = 0; al < D; ++al) {
                        const long long idx = ((long long)l * D + al) * M + k;
                        const T pv = R[idx] + beta * P[idx];
                        P[idx] = pv;
                        v[al] = pv;
                    }
                } else {
#pragma unroll
                    for (int al = 0; al < D; ++al) {
                        const long long idx = ((long long)l * D + al) * M + k;
                        v[al] = (U ? U[idx] : T(0)) + (a.E ? (T)a.E[l * D + al] : T(0));
                    }
                }
#pragma unroll
                for (int al = 0; al < D; ++al) {
                    T s = T(0);
#pragma unroll
                    for (int be = 0; be < D; ++be) s += am[al][be] * v[be];
                    t[al] = s;
                }
                if (a.mode == FWD_APPLY && a.A0) {
                    T w[D];
#pragma unroll
                    for (int al = 0; al < D; ++al) {
                        T s = T(0);
#pragma unroll
                        for (int be = 0; be < D; ++be) s += (T)a.A0[al * D + be] * t[be];
                        w[al] = s;
                    }
#pragma unroll
                    for (int al = 0; al < D; ++al) t[al] = w[al];
                }
                double dsum = 0.0;
#pragma unroll
                for (int al = 0; al < D; ++al)
                    dsum += (a.mode == FWD_CG) ? (double)v[al] * (double)t[al] : (double)t[al] * (double)t[al];
                acc[li] += dsum;
            }
#pragma unroll
            for (int al = 0; al < D; ++al) {
                const int rr = (rowi * nl + li) * D + al;
                C* z = &buf[(rr >> 1) * Nl + i];
                if (rr & 1) z->y = t[al]; else z->x = t[al];
            }
        }
    }
    if (nreal & 1)
        for (int i = threadIdx.x; i < Nl; i += blockDim.x) buf[(ncplx - 1) * Nl + i].y = T(0);
    __syncthreads();

    fft_any<T, NN, false>(buf, ncplx, Nl, pl, tw, tws);

    // Separate the packed pairs: Z = a + i b  ->  A(k) = (Z(k) + conj Z(-k))/2,
    // B(k) = (Z(k) - conj Z(-k)) / 2i, for k = 0..H-1 (Hermitian half).
    C* __restrict__ S = static_cast<C*>(a.S);
    for (int e = threadIdx.x; e < ncplx * H; e += blockDim.x) {
        const int c = e / H;
        const int kk = e - c * H;
        const C z = buf[c * Nl + kk];
        const C zm = buf[c * Nl + (kk ? Nl - kk : 0)];
        C A, B;
        A.x = T(0.5) * (z.x + zm.x); A.y = T(0.5) * (z.y - zm.y);
        B.x = T(0.5) * (z.y + zm.y); B.y = T(0.5) * (zm.x - z.x);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int rr = 2 * c + h;
            if (rr >= nreal) break;
            const int rowi = rr / (nl * D);
            const int li = (rr / D) % nl;
            const int al = rr % D;
            const long long grow = row0 + rowi;
            if (grow < rows && s_act[li])
                S[(((long long)(l0 + li) * D + al) * rows + grow) * H + kk] = h ? B : A;
        }
    }

    // reductions
    block_sum<MAXL>(acc);
    const long long nbx = gridDim.x;
    const unsigned nblocks = gridDim.x * gridDim.y;
    int slots[MAXL];
    for (int li = 0; li < nl; ++li) slots[li] = l0 + li;
    const bool last = publish(acc, slots, nl, a.partial, nbx, blockIdx.x, a.counter, nblocks);
    if (!last) return;
    double tot[MAXL];
    final_sums<MAXL>(a.partial, nbx, nbx, a.L, tot);
    if (threadIdx.x == 0) {
        for (int l = 0; l < a.L; ++l) {
            Scalars& s = a.sc[l];
            const double val = tot[l] * g.invM;
            if (a.mode == FWD_CG) {
                if (a.check_status && s.status != ST_ACTIVE) continue;
                s.pt = val;
                if (!(val > 0.0) || !isfinite(val)) {
                    s.status = ST_BREAKDOWN;
                    s.alpha = 0.0;
                } else {
                    s.alpha = s.rr / val;
                }
            } else {
                s.aen = sqrt(val);
            }
        }
        *a.counter = 0u;
    }
}

// ---------------------------------------------------------------------------
// strided-axis pass (complex DFT along one axis; Fourier projection on axis 0)
// ---------------------------------------------------------------------------
template <typename T, int D, int NN>
__global__ void __launch_bounds__(PassThreads<NN>::v) k_strided(GridDev g, AxisPlanH pl,
                                                               const Cx<T>* __restrict__ tw,
                                                               StrArgs a, int Cl) {
    typedef Cx<T> C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const long long i0 = (long long)blockIdx.x * Cl;
    const long long o = blockIdx.y;
    const int l = blockIdx.z;
    if (a.check_status && a.sc[l].status != ST_ACTIVE) return;
    const int n = NN > 0 ? NN : a.n;
    const long long inner = a.inner;
    C* __restrict__ S = static_cast<C*>(a.S);
    const long long cstride = g.Ms;
    const long long base = (long long)l * D * cstride + o * n * inner + i0;
    const C* tws = stage_twiddles<T, NN>(buf + D * Cl * n, pl, tw);

    for (int e = threadIdx.x; e < D * Cl * n; e += blockDim.x) {
        const int lane = e % Cl;
        const int rest = e / Cl;
        const int m = rest % n;
        const int al = rest / n;
        C v = czero<T>();
        if (i0 + lane < inner) v = S[base + al * cstride + (long long)m * inner + lane];
        buf[(al * Cl + lane) * n + m] = v;
    }
    __syncthreads();

    if (a.mode != STR_INV) fft_any<T, NN, false>(buf, D * Cl, n, pl, tw, tws);

    if (a.mode == STR_FWD_SCALE) {
        const T sc = (T)g.invM;
        for (int e = threadIdx.x; e < D * Cl * n; e += blockDim.x) buf[e] = cscale(buf[e], sc);
        __syncthreads();
    } else if (a.mode == STR_GAMMA) {
        // q_hat = xi (xi . t_hat) / (xi . A0 xi) / |N| with t = A0 A u (Eq. Gamma_hat,
        // G = Gamma A0); A0 = I unless has_A0
        for (int e = threadIdx.x; e < Cl * n; e += blockDim.x) {
            const int lane = e % Cl;
            const int m = e / Cl;
            const long long i = i0 + lane;
            if (i >= inner) continue;
            T xi[D];
            xi[0] = (T)((double)freq_of(m, g.N[0]) / g.Y[0]);
            if (D == 2) {
                xi[1] = (T)((double)i / g.Y[1]);
            } else {
                const int k2 = (int)(i % g.H);
                const int k1 = (int)(i / g.H);
                xi[1] = (T)((double)freq_of(k1, g.N[1]) / g.Y[1]);
                xi[D - 1] = (T)((double)k2 / g.Y[2]);
            }
            C th[D];
#pragma unroll
            for (int al = 0; al < D; ++al) th[al] = buf[(al * Cl + lane) * n + m];
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
            C s = czero<T>();
            if (den > T(0)) {
                const T f = (T)g.invM / den;
                s.x = num.x * f;
                s.y = num.y * f;
            }
#pragma unroll
            for (int al = 0; al < D; ++al) buf[(al * Cl + lane) * n + m] = cscale(s, xi[al]);
        }
        __syncthreads();
        fft_any<T, NN, true>(buf, D * Cl, n, pl, tw, tws);
    } else if (a.mode == STR_INV) {
        fft_any<T, NN, true>(buf, D * Cl, n, pl, tw, tws);
    }

    for (int e = threadIdx.x; e < D * Cl * n; e += blockDim.x) {
        const int lane = e % Cl;
        const int rest = e / Cl;
        const int m = rest % n;
        const int al = rest / n;
        if (i0 + lane < inner) S[base + al * cstride + (long long)m * inner + lane] = buf[(al * Cl + lane) * n + m];
    }
}

// ---------------------------------------------------------------------------
// last-axis inverse pass (complex-to-real DFT + CG update)
// ---------------------------------------------------------------------------
template <typename T, int D, int NN>
__global__ void __launch_bounds__(PassThreads<NN>::v) k_row_inv(GridDev g, AxisPlanH pl,
                                                               const Cx<T>* __restrict__ tw,
                                                               RowInvArgs a, int RB, int LB) {
    typedef Cx<T> C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int Nl = NN > 0 ? NN : g.Nl;
    const int H = (Nl + 1) >> 1;
    const long long M = g.M, rows = g.rows;
    const long long row0 = (long long)blockIdx.x * RB;
    const int l0 = blockIdx.y * LB;
    const int nl = min(LB, a.L - l0);
    const int nreal = RB * nl * D;
    const int ncplx = (nreal + 1) >> 1;
    const C* tws = stage_twiddles<T, NN>(buf + ncplx * Nl, pl, tw);

    __shared__ double s_alpha[MAXL];
    __shared__ int s_act[MAXL];
    if (threadIdx.x < nl) {
        const Scalars& s = a.sc[l0 + threadIdx.x];
        s_act[threadIdx.x] = (!a.check_status) || (s.status == ST_ACTIVE);
        s_alpha[threadIdx.x] = s.alpha;
    }
    __syncthreads();

    // Rebuild two real rows a, b as one complex row Z = a + i b from their
    // Hermitian half spectra: X(k) for k >= H is conj X(Nl - k).
    const C* __restrict__ S = static_cast<const C*>(a.S);
    for (int e = threadIdx.x; e < ncplx * Nl; e += blockDim.x) {
        const int c = e / Nl;
        const int kk = e - c * Nl;
        const bool up = kk >= H;
        const int ks = up ? Nl - kk : kk;
        C v[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            v[h] = czero<T>();
            const int rr = 2 * c + h;
            if (rr < nreal) {
                const int rowi = rr / (nl * D);
                const int li = (rr / D) % nl;
                const int al = rr % D;
                const long long grow = row0 + rowi;
                if (grow < rows && s_act[li])
                    v[h] = S[(((long long)(l0 + li) * D + al) * rows + grow) * H + ks];
            }
            if (up) v[h].y = -v[h].y;
        }
        C z;
        z.x = v[0].x - v[1].y;
        z.y = v[0].y + v[1].x;
        buf[c * Nl + kk] = z;
    }
    __syncthreads();

    fft_any<T, NN, true>(buf, ncplx, Nl, pl, tw, tws);

    T* __restrict__ X = static_cast<T*>(a.x);
    T* __restrict__ Rr = static_cast<T*>(a.r);
    T* __restrict__ P = static_cast<T*>(a.p);
    T* __restrict__ O = static_cast<T*>(a.out);
    double acc[MAXL] = {0.0, 0.0, 0.0};
    for (int e = threadIdx.x; e < RB * Nl; e += blockDim.x) {
        const int rowi = e / Nl;
        const int i = e - rowi * Nl;
        const long long grow = row0 + rowi;
        if (grow >= rows) continue;
        const long long k = grow * Nl + i;
#pragma unroll
        for (int li = 0; li < MAXL; ++li) {
            if (li >= nl) break;
            if (!s_act[li]) continue;
            const int l = l0 + li;
            const T alpha = (T)s_alpha[li];
            double dsum = 0.0;
#pragma unroll
            for (int al = 0; al < D; ++al) {
                const int rr = (rowi * nl + li) * D + al;
                const C z = buf[(rr >> 1) * Nl + i];
                const T q = (rr & 1) ? z.y : z.x;
                const long long idx = ((long long)l * D + al) * M + k;
                if (a.mode == INV_CG) {
                    X[idx] += alpha * P[idx];
                    const T rv = Rr[idx] - alpha * q;
                    Rr[idx] = rv;
                    dsum += (double)rv * (double)rv;
                } else if (a.mode == INV_RHS) {
                    const T rv = -q;
                    Rr[idx] = rv;
                    P[idx] = rv;
                    X[idx] = T(0);
                    dsum += (double)rv * (double)rv;
                } else if (a.mode == INV_RESID) {
                    const T rv = -q;
                    Rr[idx] = rv;
                    dsum += (double)rv * (double)rv;
                } else {
                    O[idx] = q;
                }
            }
            acc[li] += dsum;
        }
    }

    if (a.mode == INV_OUT) return;
    block_sum<MAXL>(acc);
    const long long nbx = gridDim.x;
    const unsigned nblocks = gridDim.x * gridDim.y;
    int slots[MAXL];
    for (int li = 0; li < nl; ++li) slots[li] = l0 + li;
    const bool last = publish(acc, slots, nl, a.partial, nbx, blockIdx.x, a.counter, nblocks);
    if (!last) return;
    double tot[MAXL];
    final_sums<MAXL>(a.partial, nbx, nbx, a.L, tot);
    if (threadIdx.x == 0) {
        for (int l = 0; l < a.L; ++l) {
            Scalars& s = a.sc[l];
            if (a.check_status && s.status != ST_ACTIVE) continue;
            const double rr = tot[l] * g.invM;
            if (a.mode == INV_CG) {
                s.iters += 1;
                s.total_iters += 1;
                const double rel = sqrt(rr) / s.bnorm;
                s.relres = rel;
                if (!isfinite(rr)) s.status = ST_BREAKDOWN;
                else if (rel <= s.tol) s.status = ST_CONVERGED;
                else if (s.iters >= s.max_iter) s.status = ST_MAXITER;
                s.beta = rr / s.rr;
                s.rr = rr;
            } else if (a.mode == INV_RHS) {
                s.rr = rr;
                s.bnorm = sqrt(rr);
                s.beta = 0.0;
                s.iters = 0;
                s.relres = 1.0;
                // b = -G A E vanishes in exact arithmetic when A E is constant
                // along every direction G keeps (G kills constants, Lemma
                // FD_projection (iv)); ||b|| <= ||A E|| since G is an
                // orthogonal projection, so a ratio at roundoff level is zero.
                if (!(s.bnorm > ZERO_RHS * s.aen)) {
                    s.status = ST_ZERO_RHS;
                    s.relres = 0.0;
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

// ---------------------------------------------------------------------------
// per-precision launch dispatch (hg_kernels_f32.cu / hg_kernels_f64.cu)
// ---------------------------------------------------------------------------
// Transform lengths with compile-time kernels; every other length runs the
// runtime-plan kernels.
#define HG_CT_SIZES_2D(X) X(15) X(27) X(45) X(75) X(81) X(135) X(243) X(375) X(729)
#define HG_CT_SIZES_3D(X) X(15) X(27) X(45) X(81) X(135)

template <typename T>
cudaError_t launch_row_fwd_t(const GridDev& g, const AxisPlanH& pl, const void* tw, const RowCfg& cfg,
                             const RowFwdArgs& a, cudaStream_t s) {
    dim3 grid((unsigned)cfg.nbx, (unsigned)((a.L + cfg.LB - 1) / cfg.LB));
    const Cx<T>* twp = (const Cx<T>*)tw;
#define HG_CASE2(NV) case NV: k_row_fwd<T, 2, NV><<<grid, CT_THREADS, cfg.smem, s>>>(g, pl, twp, a, cfg.RB, cfg.LB); break;
#define HG_CASE3(NV) case NV: k_row_fwd<T, 3, NV><<<grid, CT_THREADS, cfg.smem, s>>>(g, pl, twp, a, cfg.RB, cfg.LB); break;
    if (g.d == 2) {
        if (cfg.ct) {
            switch (g.Nl) {
                HG_CT_SIZES_2D(HG_CASE2)
                default: return cudaErrorInvalidConfiguration;   // no compile-time kernel
            }
        } else {
            k_row_fwd<T, 2, 0><<<grid, cfg.threads, cfg.smem, s>>>(g, pl, twp, a, cfg.RB, cfg.LB);
        }
    } else {
        if (cfg.ct) {
            switch (g.Nl) {
                HG_CT_SIZES_3D(HG_CASE3)
                default: return cudaErrorInvalidConfiguration;   // no compile-time kernel
            }
        } else {
            k_row_fwd<T, 3, 0><<<grid, cfg.threads, cfg.smem, s>>>(g, pl, twp, a, cfg.RB, cfg.LB);
        }
    }
#undef HG_CASE2
#undef HG_CASE3
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_row_inv_t(const GridDev& g, const AxisPlanH& pl, const void* tw, const RowCfg& cfg,
                             const RowInvArgs& a, cudaStream_t s) {
    dim3 grid((unsigned)cfg.nbx, (unsigned)((a.L + cfg.LB - 1) / cfg.LB));
    const Cx<T>* twp = (const Cx<T>*)tw;
#define HG_CASE2(NV) case NV: k_row_inv<T, 2, NV><<<grid, CT_THREADS, cfg.smem, s>>>(g, pl, twp, a, cfg.RB, cfg.LB); break;
#define HG_CASE3(NV) case NV: k_row_inv<T, 3, NV><<<grid, CT_THREADS, cfg.smem, s>>>(g, pl, twp, a, cfg.RB, cfg.LB); break;
    if (g.d == 2) {
        if (cfg.ct) {
            switch (g.Nl) {
                HG_CT_SIZES_2D(HG_CASE2)
                default: return cudaErrorInvalidConfiguration;   // no compile-time kernel
            }
        } else {
            k_row_inv<T, 2, 0><<<grid, cfg.threads, cfg.smem, s>>>(g, pl, twp, a, cfg.RB, cfg.LB);
        }
    } else {
        if (cfg.ct) {
            switch (g.Nl) {
                HG_CT_SIZES_3D(HG_CASE3)
                default: return cudaErrorInvalidConfiguration;   // no compile-time kernel
            }
        } else {
            k_row_inv<T, 3, 0><<<grid, cfg.threads, cfg.smem, s>>>(g, pl, twp, a, cfg.RB, cfg.LB);
        }
    }
#undef HG_CASE2
#undef HG_CASE3
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_strided_t(const GridDev& g, const AxisPlanH& pl, const void* tw, const StrCfg& cfg,
                             const StrArgs& a, cudaStream_t s) {
    dim3 grid((unsigned)((a.inner + cfg.Cl - 1) / cfg.Cl), (unsigned)a.outer, (unsigned)a.L);
    const Cx<T>* twp = (const Cx<T>*)tw;
#define HG_CASE2(NV) case NV: k_strided<T, 2, NV><<<grid, CT_THREADS, cfg.smem, s>>>(g, pl, twp, a, cfg.Cl); break;
#define HG_CASE3(NV) case NV: k_strided<T, 3, NV><<<grid, CT_THREADS, cfg.smem, s>>>(g, pl, twp, a, cfg.Cl); break;
    if (g.d == 2) {
        if (cfg.ct) {
            switch (a.n) {
                HG_CT_SIZES_2D(HG_CASE2)
                default: return cudaErrorInvalidConfiguration;   // no compile-time kernel
            }
        } else {
            k_strided<T, 2, 0><<<grid, cfg.threads, cfg.smem, s>>>(g, pl, twp, a, cfg.Cl);
        }
    } else {
        if (cfg.ct) {
            switch (a.n) {
                HG_CT_SIZES_3D(HG_CASE3)
                default: return cudaErrorInvalidConfiguration;   // no compile-time kernel
            }
        } else {
            k_strided<T, 3, 0><<<grid, cfg.threads, cfg.smem, s>>>(g, pl, twp, a, cfg.Cl);
        }
    }
#undef HG_CASE2
#undef HG_CASE3
    return cudaGetLastError();
}

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
#define HG_SET2(NV) HG_SET(k_row_fwd<T, 2, NV>); HG_SET(k_row_inv<T, 2, NV>); HG_SET(k_strided<T, 2, NV>);
#define HG_SET3(NV) HG_SET(k_row_fwd<T, 3, NV>); HG_SET(k_row_inv<T, 3, NV>); HG_SET(k_strided<T, 3, NV>);
    HG_SET2(0) HG_SET3(0)
    HG_CT_SIZES_2D(HG_SET2)
    HG_CT_SIZES_3D(HG_SET3)
#undef HG_SET2
#undef HG_SET3
#undef HG_SET
    return e;
}

}  // namespace hgk
