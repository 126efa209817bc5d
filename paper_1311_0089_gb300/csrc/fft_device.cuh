// Device-side mixed-radix (3/5/7) Stockham FFT on pencils staged in shared
// memory.  The DFT convention is Eq. DFT_def (Sec. 4.1): the forward kernel is
// omega^{-km} = exp(-2 pi i k m / N), the inverse exp(+2 pi i k m / N); both are
// unnormalised here (the 1/|N| of the forward transform is folded into the
// Fourier projection by the callers).
//
// A stage of radix R with Ns = product of the radices already applied maps,
// for every butterfly j in [0, N/R) with k = j mod Ns,
//     v_r = x[j + r N/R] * W_N^{r k N/(Ns R)}     (r = 0..R-1, W_N = e^{-2 pi i/N})
//     y   = DFT_R(v)
//     x'[(j / Ns) Ns R + k + r Ns] = y_r
// (the self-sorting Stockham formulation: no bit/digit reversal pass).  The
// stage is done in place: every thread first loads all of its butterflies
// into registers, the block synchronises, then every thread stores.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <type_traits>
#include "hg_internal.h"

namespace hgk {

template <typename T> struct cplx_t;
template <> struct cplx_t<double> { typedef double2 type; };
template <> struct cplx_t<float>  { typedef float2 type; };

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2  cadd(float2 a, float2 b)   { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2  csub(float2 a, float2 b)   { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ float2  cscale(float2 a, float s)   { return make_float2(a.x * s, a.y * s); }
// a * w  (CONJ: a * conj(w))
template <bool CONJ> __device__ __forceinline__ double2 cmulw(double2 a, double2 w) {
    return CONJ ? make_double2(fma(a.x, w.x, a.y * w.y), fma(a.y, w.x, -a.x * w.y))
                : make_double2(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
}
template <bool CONJ> __device__ __forceinline__ float2 cmulw(float2 a, float2 w) {
    return CONJ ? make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y))
                : make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}

// Constants cos/sin(2 pi k / R), written out to 20 digits from their closed
// forms (R = 3: sqrt(3)/2; R = 5: (sqrt(5)-1)/4 etc.).
#define HG_S3   0.86602540378443864676   // sin(2pi/3)
#define HG_C51  0.30901699437494742410   // cos(2pi/5)
#define HG_C52 -0.80901699437494742410   // cos(4pi/5)
#define HG_S51  0.95105651629515357212   // sin(2pi/5)
#define HG_S52  0.58778525229247312917   // sin(4pi/5)
#define HG_C71  0.62348980185873353053   // cos(2pi/7)
#define HG_C72 -0.22252093395631440429   // cos(4pi/7)
#define HG_C73 -0.90096886790241912624   // cos(6pi/7)
#define HG_S71  0.78183148246802980871   // sin(2pi/7)
#define HG_S72  0.97492791218182360702   // sin(4pi/7)
#define HG_S73  0.43388373911755812048   // sin(6pi/7)

// y = x0 + c * (a) - i * s  with s complex: returns (t.x + s.y, t.y - s.x) for
// the forward sign; INV flips the sign of the i-term.
template <bool INV, typename C>
__device__ __forceinline__ void pm_i(C t, C s, C& ym, C& yp) {
    // ym = t - i s, yp = t + i s   (forward);  swapped for the inverse
    C a, b;
    a.x = t.x + s.y; a.y = t.y - s.x;
    b.x = t.x - s.y; b.y = t.y + s.x;
    if (INV) { ym = b; yp = a; } else { ym = a; yp = b; }
}

template <int R, bool INV, typename C> struct Dft;

template <bool INV, typename C> struct Dft<3, INV, C> {
    __device__ __forceinline__ static void run(C* v) {
        typedef decltype(C().x) T;
        C s = cadd(v[1], v[2]);
        C dd = csub(v[1], v[2]);
        C m; m.x = v[0].x - T(0.5) * s.x; m.y = v[0].y - T(0.5) * s.y;
        v[0] = cadd(v[0], s);
        C sd = cscale(dd, T(HG_S3));
        pm_i<INV>(m, sd, v[1], v[2]);
    }
};

template <bool INV, typename C> struct Dft<5, INV, C> {
    __device__ __forceinline__ static void run(C* v) {
        typedef decltype(C().x) T;
        C a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
        C a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
        C x0 = v[0];
        C t1, t2, u1, u2;
        t1.x = x0.x + T(HG_C51) * a1.x + T(HG_C52) * a2.x;
        t1.y = x0.y + T(HG_C51) * a1.y + T(HG_C52) * a2.y;
        t2.x = x0.x + T(HG_C52) * a1.x + T(HG_C51) * a2.x;
        t2.y = x0.y + T(HG_C52) * a1.y + T(HG_C51) * a2.y;
        u1.x = T(HG_S51) * b1.x + T(HG_S52) * b2.x;
        u1.y = T(HG_S51) * b1.y + T(HG_S52) * b2.y;
        u2.x = T(HG_S52) * b1.x - T(HG_S51) * b2.x;
        u2.y = T(HG_S52) * b1.y - T(HG_S51) * b2.y;
        v[0] = cadd(x0, cadd(a1, a2));
        C y1, y4, y2, y3;
        pm_i<INV>(t1, u1, y1, y4);
        pm_i<INV>(t2, u2, y2, y3);
        v[1] = y1; v[2] = y2; v[3] = y3; v[4] = y4;
    }
};

template <bool INV, typename C> struct Dft<7, INV, C> {
    __device__ __forceinline__ static void run(C* v) {
        typedef decltype(C().x) T;
        C a1 = cadd(v[1], v[6]), b1 = csub(v[1], v[6]);
        C a2 = cadd(v[2], v[5]), b2 = csub(v[2], v[5]);
        C a3 = cadd(v[3], v[4]), b3 = csub(v[3], v[4]);
        C x0 = v[0];
        C t1, t2, t3, u1, u2, u3;
        // y_m = x0 + sum_k cos(2 pi m k/7) a_k -/+ i sum_k sin(2 pi m k/7) b_k
        t1.x = x0.x + T(HG_C71) * a1.x + T(HG_C72) * a2.x + T(HG_C73) * a3.x;
        t1.y = x0.y + T(HG_C71) * a1.y + T(HG_C72) * a2.y + T(HG_C73) * a3.y;
        t2.x = x0.x + T(HG_C72) * a1.x + T(HG_C73) * a2.x + T(HG_C71) * a3.x;
        t2.y = x0.y + T(HG_C72) * a1.y + T(HG_C73) * a2.y + T(HG_C71) * a3.y;
        t3.x = x0.x + T(HG_C73) * a1.x + T(HG_C71) * a2.x + T(HG_C72) * a3.x;
        t3.y = x0.y + T(HG_C73) * a1.y + T(HG_C71) * a2.y + T(HG_C72) * a3.y;
        u1.x = T(HG_S71) * b1.x + T(HG_S72) * b2.x + T(HG_S73) * b3.x;
        u1.y = T(HG_S71) * b1.y + T(HG_S72) * b2.y + T(HG_S73) * b3.y;
        u2.x = T(HG_S72) * b1.x - T(HG_S73) * b2.x - T(HG_S71) * b3.x;
        u2.y = T(HG_S72) * b1.y - T(HG_S73) * b2.y - T(HG_S71) * b3.y;
        u3.x = T(HG_S73) * b1.x - T(HG_S71) * b2.x + T(HG_S72) * b3.x;
        u3.y = T(HG_S73) * b1.y - T(HG_S71) * b2.y + T(HG_S72) * b3.y;
        v[0] = cadd(x0, cadd(a1, cadd(a2, a3)));
        C y1, y6, y2, y5, y3, y4;
        pm_i<INV>(t1, u1, y1, y6);
        pm_i<INV>(t2, u2, y2, y5);
        pm_i<INV>(t3, u3, y3, y4);
        v[1] = y1; v[2] = y2; v[3] = y3; v[4] = y4; v[5] = y5; v[6] = y6;
    }
};

// One in-place Stockham stage over `npen` pencils of length n stored at
// buf + p * pstride.  MAXB butterflies per thread at most (host guarantees
// blockDim.x * MAXB >= npen * n / R).
template <typename T, int R, bool INV, int MAXB>
__device__ __forceinline__ void stage(typename cplx_t<T>::type* buf, int npen, int pstride,
                                      int n, int Ns, const typename cplx_t<T>::type* __restrict__ tw) {
    typedef typename cplx_t<T>::type C;
    const int nb = n / R;
    const int total = npen * nb;
    const int twstep = n / (Ns * R);
    C v[MAXB][R];
    int dst[MAXB];
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        int idx = threadIdx.x + b * blockDim.x;
        dst[b] = -1;
        if (idx < total) {
            int pen = idx / nb;
            int j = idx - pen * nb;
            int k = j % Ns;
            const C* src = buf + pen * pstride + j;
#pragma unroll
            for (int r = 0; r < R; ++r) v[b][r] = src[r * nb];
            if (Ns > 1) {
                int step = k * twstep;
#pragma unroll
                for (int r = 1; r < R; ++r) v[b][r] = cmulw<INV>(v[b][r], __ldg(&tw[r * step]));
            }
            Dft<R, INV, C>::run(v[b]);
            dst[b] = pen * pstride + (j - k) * R + k;
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        if (dst[b] >= 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) buf[dst[b] + r * Ns] = v[b][r];
        }
    }
    __syncthreads();
}

// Full transform of npen pencils (forward: INV = false).
template <typename T, bool INV, int MAXB>
__device__ void fft_pencils(typename cplx_t<T>::type* buf, int npen, int pstride,
                            const AxisPlanH& pl, const typename cplx_t<T>::type* __restrict__ twall) {
    const typename cplx_t<T>::type* tw = twall + pl.tw_off;
    int Ns = 1;
    for (int s = 0; s < pl.nstages; ++s) {
        int R = pl.radix[s];
        if (R == 3)      stage<T, 3, INV, MAXB>(buf, npen, pstride, pl.n, Ns, tw);
        else if (R == 5) stage<T, 5, INV, MAXB>(buf, npen, pstride, pl.n, Ns, tw);
        else             stage<T, 7, INV, MAXB>(buf, npen, pstride, pl.n, Ns, tw);
        Ns *= R;
    }
}

}  // namespace hgk

// ===========================================================================
// Compile-time FFT: per-length plans, composite register codelets
// ===========================================================================
namespace hgk {

// W_R^m = exp(-2 pi i m / R) for the composite codelet lengths.  Every
// translation unit holds its own copy; configure_t() fills it per device from
// extended-precision host values.
static __constant__ double2 c_ctw64[CTW_TOTAL];
static __constant__ float2 c_ctw32[CTW_TOTAL];

template <int R> struct CtwOff;
template <> struct CtwOff<9>  { static constexpr int v = CTW_9; };
template <> struct CtwOff<15> { static constexpr int v = CTW_15; };
template <> struct CtwOff<25> { static constexpr int v = CTW_25; };
template <> struct CtwOff<27> { static constexpr int v = CTW_27; };

template <int R, int M> __device__ __forceinline__ double2 ctw(double2) { return c_ctw64[CtwOff<R>::v + (M % R)]; }
template <int R, int M> __device__ __forceinline__ float2 ctw(float2) { return c_ctw32[CtwOff<R>::v + (M % R)]; }

// DFT of length R = R1 * R2 in registers (R1, R2 smaller codelets):
//   n = n1 + R1 n2, k = k1 + R2 k2,  W_R^{nk} = W_R^{n1 k1} W_R1^{n1 k2} W_R2^{n2 k1}
// -> R1 DFTs of length R2 over n2, twiddles W_R^{n1 k1}, R2 DFTs of length R1 over n1.
template <int R1, int R2, bool INV, typename C> struct DftComposite;

template <int R, bool INV, typename C> struct DftAny { };
template <bool INV, typename C> struct DftAny<3, INV, C> { __device__ __forceinline__ static void run(C* v) { Dft<3, INV, C>::run(v); } };
template <bool INV, typename C> struct DftAny<5, INV, C> { __device__ __forceinline__ static void run(C* v) { Dft<5, INV, C>::run(v); } };
template <bool INV, typename C> struct DftAny<7, INV, C> { __device__ __forceinline__ static void run(C* v) { Dft<7, INV, C>::run(v); } };
template <bool INV, typename C> struct DftAny<9, INV, C> { __device__ __forceinline__ static void run(C* v) { DftComposite<3, 3, INV, C>::run(v); } };
template <bool INV, typename C> struct DftAny<15, INV, C> { __device__ __forceinline__ static void run(C* v) { DftComposite<3, 5, INV, C>::run(v); } };
template <bool INV, typename C> struct DftAny<25, INV, C> { __device__ __forceinline__ static void run(C* v) { DftComposite<5, 5, INV, C>::run(v); } };
template <bool INV, typename C> struct DftAny<27, INV, C> { __device__ __forceinline__ static void run(C* v) { DftComposite<3, 9, INV, C>::run(v); } };

template <int R1, int R2, bool INV, typename C> struct DftComposite {
    static constexpr int R = R1 * R2;
    template <int N1, int K1>
    __device__ __forceinline__ static void tw(C (&t)[R1][R2]) {
        if constexpr (N1 > 0 && K1 > 0) t[N1][K1] = cmulw<INV>(t[N1][K1], ctw<R, N1 * K1>(C()));
        if constexpr (K1 + 1 < R2) tw<N1, K1 + 1>(t);
        else if constexpr (N1 + 1 < R1) tw<N1 + 1, 0>(t);
    }
    __device__ __forceinline__ static void run(C* v) {
        C t[R1][R2];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) {
            C col[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) col[n2] = v[n1 + R1 * n2];
            DftAny<R2, INV, C>::run(col);
#pragma unroll
            for (int k1 = 0; k1 < R2; ++k1) t[n1][k1] = col[k1];
        }
        tw<0, 0>(t);
#pragma unroll
        for (int k1 = 0; k1 < R2; ++k1) {
            C row[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) row[n1] = t[n1][k1];
            DftAny<R1, INV, C>::run(row);
#pragma unroll
            for (int k2 = 0; k2 < R1; ++k2) v[k1 + R2 * k2] = row[k2];
        }
    }
};

// Compile-time radix plans per transform length and precision (double:
// smaller codelets, the FP64 path is register- and ALU-bound).
template <typename T, int N> struct CtPlan;
template <int... Rs> struct RadixList {};
#define HG_PLAN(TT, NN, ...) template <> struct CtPlan<TT, NN> { typedef RadixList<__VA_ARGS__> type; static constexpr bool ok = true; };
HG_PLAN(float, 729, 27, 27)
HG_PLAN(float, 375, 15, 25)
HG_PLAN(float, 243, 27, 9)
HG_PLAN(float, 135, 15, 9)
HG_PLAN(float, 81, 9, 9)
HG_PLAN(float, 75, 25, 3)
HG_PLAN(float, 45, 9, 5)
HG_PLAN(float, 27, 27)
HG_PLAN(float, 15, 15)
HG_PLAN(double, 729, 9, 9, 9)
HG_PLAN(double, 375, 15, 5, 5)
HG_PLAN(double, 243, 9, 9, 3)
HG_PLAN(double, 135, 15, 9)
HG_PLAN(double, 81, 9, 9)
HG_PLAN(double, 75, 15, 5)
HG_PLAN(double, 45, 9, 5)
HG_PLAN(double, 27, 9, 3)
HG_PLAN(double, 15, 15)
#undef HG_PLAN

// Threads per CTA of the compile-time kernels and the largest number of
// pencils one CTA stages (bounded by 48 KB of data per CTA and 16 pencils).
constexpr int CT_THREADS = 256;
template <typename T, int N> struct CtCaps {
    static constexpr int csize = (int)sizeof(typename cplx_t<T>::type);
    static constexpr int by_smem = (48 * 1024) / (N * csize);
    static constexpr int npmax = by_smem < 1 ? 1 : (by_smem > 16 ? 16 : by_smem);
};

// One in-place Stockham stage (see the formulation at the top of this file)
// with every size known at compile time.  `tw` is this stage's twiddle table
// in shared memory, laid out [r-1][k] (k = j mod NS): consecutive threads read
// consecutive entries.
//
// Layouts: ILD = 0 -> pencil p occupies buf[p N .. p N + N) (contiguous);
// ILD = D > 0 -> pencil (al, lane), al < D, lane < Cl = 2^lgCl, element j at
// buf[(al N + j) Cl + lane] (interleaved lanes), with the pencil index
// running fastest across threads so that neighbouring threads touch
// neighbouring words.
template <typename T, int N, int R, int NS, bool INV, int NPMAX, int ILD>
__device__ __forceinline__ void stage_ct(typename cplx_t<T>::type* buf, int npen, int lgCl,
                                         const typename cplx_t<T>::type* tw) {
    typedef typename cplx_t<T>::type C;
    constexpr int NB = N / R;
    constexpr int B = (NPMAX * NB + CT_THREADS - 1) / CT_THREADS;
    const int total = npen * NB;
    const int es = ILD > 0 ? (1 << lgCl) : 1;     // element stride
    C v[B][R];
    int dst[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int idx = threadIdx.x + b * CT_THREADS;
        dst[b] = -1;
        if (idx < total) {
            int base, j;
            if constexpr (ILD > 0) {
                const int lane = idx & (es - 1);
                const int t = idx >> lgCl;
                const int al = t % ILD;
                j = t / ILD;
                base = al * N * es + lane;
            } else {
                const int pen = idx / NB;
                j = idx - pen * NB;
                base = pen * N;
            }
            const int k = j % NS;
            const C* src = buf + base + j * es;
#pragma unroll
            for (int r = 0; r < R; ++r) v[b][r] = src[r * NB * es];
            if constexpr (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) v[b][r] = cmulw<INV>(v[b][r], tw[(r - 1) * NS + k]);
            }
            DftAny<R, INV, C>::run(v[b]);
            dst[b] = base + ((j - k) * R + k) * es;
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        if (dst[b] >= 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) buf[dst[b] + r * NS * es] = v[b][r];
        }
    }
    __syncthreads();
}

// Per-stage twiddle tables: stage s (NS > 1) holds W_N^{r k N/(NS R)} at
// [(r-1) NS + k], r = 1..R-1, k < NS; OFF is the running offset.
template <typename T, int N, bool INV, int NPMAX, int NS, int OFF, int... Rs> struct CtStages;
template <typename T, int N, bool INV, int NPMAX, int NS, int OFF> struct CtStages<T, N, INV, NPMAX, NS, OFF> {
    static constexpr int tw_size = OFF;
    template <int ILD>
    __device__ __forceinline__ static void run(typename cplx_t<T>::type*, int, int, const typename cplx_t<T>::type*) {}
    __device__ __forceinline__ static void build(typename cplx_t<T>::type*, const typename cplx_t<T>::type*) {}
};
template <typename T, int N, bool INV, int NPMAX, int NS, int OFF, int R, int... Rs>
struct CtStages<T, N, INV, NPMAX, NS, OFF, R, Rs...> {
    static constexpr int here = NS > 1 ? (R - 1) * NS : 0;
    typedef CtStages<T, N, INV, NPMAX, NS * R, OFF + here, Rs...> Next;
    static constexpr int tw_size = Next::tw_size;
    template <int ILD>
    __device__ __forceinline__ static void run(typename cplx_t<T>::type* buf, int npen, int lgCl,
                                               const typename cplx_t<T>::type* twst) {
        stage_ct<T, N, R, NS, INV, NPMAX, ILD>(buf, npen, lgCl, twst + OFF);
        Next::template run<ILD>(buf, npen, lgCl, twst);
    }
    // twst[OFF + (r-1) NS + k] = tw_nat[r k N/(NS R)]
    __device__ __forceinline__ static void build(typename cplx_t<T>::type* twst,
                                                 const typename cplx_t<T>::type* __restrict__ tw_nat) {
        if constexpr (NS > 1) {
            constexpr int TWS = N / (NS * R);
            for (int idx = threadIdx.x; idx < here; idx += blockDim.x) {
                const int r = idx / NS + 1;
                const int k = idx - (r - 1) * NS;
                twst[OFF + idx] = tw_nat[r * k * TWS];
            }
        }
        Next::build(twst, tw_nat);
    }
};

template <typename T, int N, bool INV, typename L> struct CtRun;
template <typename T, int N, bool INV, int... Rs> struct CtRun<T, N, INV, RadixList<Rs...>> {
    typedef CtStages<T, N, INV, CtCaps<T, N>::npmax, 1, 0, Rs...> S;
    template <int ILD>
    __device__ __forceinline__ static void run(typename cplx_t<T>::type* buf, int npen, int lgCl,
                                               const typename cplx_t<T>::type* twst) {
        S::template run<ILD>(buf, npen, lgCl, twst);
    }
};

// npen pencils of length N, contiguous (stride N) at buf; twst = the
// per-stage twiddle tables built by fft_ct_twiddles.
template <typename T, int N, bool INV>
__device__ __forceinline__ void fft_ct(typename cplx_t<T>::type* buf, int npen,
                                       const typename cplx_t<T>::type* twst) {
    CtRun<T, N, INV, typename CtPlan<T, N>::type>::template run<0>(buf, npen, 0, twst);
}

// Interleaved layout: D components x 2^lgCl lanes (see stage_ct).
template <typename T, int N, bool INV, int D>
__device__ __forceinline__ void fft_ct_il(typename cplx_t<T>::type* buf, int lgCl,
                                          const typename cplx_t<T>::type* twst) {
    CtRun<T, N, INV, typename CtPlan<T, N>::type>::template run<D>(buf, D << lgCl, lgCl, twst);
}

template <typename T, int N>
__device__ __forceinline__ void fft_ct_twiddles(typename cplx_t<T>::type* twst,
                                                const typename cplx_t<T>::type* __restrict__ tw_nat) {
    CtRun<T, N, false, typename CtPlan<T, N>::type>::S::build(twst, tw_nat);
}

}  // namespace hgk
