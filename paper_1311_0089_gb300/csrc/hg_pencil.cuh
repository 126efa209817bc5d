// Pencil transforms of the single-kernel FP32 paths (the resident 2D solver,
// the 3D plane passes): inverse unnormalised DFTs of whole pencils held in
// shared memory, by out-of-place Stockham stages.  The forward DFT is
// conj(IDFT(conj x)).
#pragma once
#include "hg_kernels.cuh"

namespace hgk {

constexpr int PEN_THREADS = 512;

// FFT plans (FP32, length N): the fewest stages whose butterflies (register
// codelets up to radix 27) fit a thread's 128 registers in the out-of-place
// stages.
template <int N> struct ResPlan;
template <> struct ResPlan<729> { typedef RadixList<27, 27> type; };
template <> struct ResPlan<375> { typedef RadixList<15, 25> type; };
template <> struct ResPlan<243> { typedef RadixList<27, 9> type; };
template <> struct ResPlan<135> { typedef RadixList<15, 9> type; };
template <> struct ResPlan<81> { typedef RadixList<9, 9> type; };
template <> struct ResPlan<75> { typedef RadixList<15, 5> type; };
template <> struct ResPlan<45> { typedef RadixList<9, 5> type; };
template <> struct ResPlan<27> { typedef RadixList<9, 3> type; };
template <> struct ResPlan<15> { typedef RadixList<15> type; };
#define HG_RES_SIZES(X) X(729) X(375) X(243) X(135) X(81) X(75) X(45) X(27) X(15)

// One inverse Stockham stage (the formulation of fft_device.cuh), out of
// place: npen contiguous pencils of length N from src to dst.  Each thread
// takes its butterflies one after the other (one butterfly's registers at a
// time), and one block barrier ends the stage.  tw: this stage's table,
// [r-1][k], k < NS.
template <int N, int R, int NS>
__device__ __forceinline__ void rstage(const float2* __restrict__ src, float2* __restrict__ dst, int npen,
                                       const float2* __restrict__ tw) {
    constexpr int NB = N / R;
    const int total = npen * NB;
#pragma unroll 1
    for (int idx = threadIdx.x; idx < total; idx += PEN_THREADS) {
        const int pen = idx / NB;
        const int j = idx - pen * NB;
        const int k = j % NS;
        const float2* sp = src + pen * N + j;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = sp[r * NB];
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmulw<true>(v[r], tw[(r - 1) * NS + k]);
        }
        DftAny<R, true, float2>::run(v);
        float2* dp = dst + pen * N + (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dp[r * NS] = v[r];
    }
    __syncthreads();
}

template <int N, int NS, int OFF, int... Rs> struct RStages;
template <int N, int NS, int OFF> struct RStages<N, NS, OFF> {
    static constexpr int tw_size = OFF;
    __device__ __forceinline__ static float2* run(float2* a, float2*, int, const float2*) { return a; }
    __device__ __forceinline__ static void build(float2*, const float2*) {}
};
template <int N, int NS, int OFF, int R, int... Rs>
struct RStages<N, NS, OFF, R, Rs...> {
    static constexpr int here = NS > 1 ? (R - 1) * NS : 0;
    typedef RStages<N, NS * R, OFF + here, Rs...> Next;
    static constexpr int tw_size = Next::tw_size;
    // stages alternate between the two buffers; returns the one with the result
    __device__ __forceinline__ static float2* run(float2* a, float2* b, int npen, const float2* tws) {
        rstage<N, R, NS>(a, b, npen, tws + OFF);
        return Next::run(b, a, npen, tws);
    }
    // tws[OFF + (r-1) NS + k] = W_N^{r k N / (NS R)}
    __device__ __forceinline__ static void build(float2* tws, const float2* __restrict__ tw_nat) {
        if constexpr (NS > 1) {
            constexpr int TWS = N / (NS * R);
            for (int i = threadIdx.x; i < here; i += blockDim.x) {
                const int r = i / NS + 1;
                const int k = i - (r - 1) * NS;
                tws[OFF + i] = tw_nat[r * k * TWS];
            }
        }
        Next::build(tws, tw_nat);
    }
};
template <int N, typename L> struct RRun;
template <int N, int... Rs> struct RRun<N, RadixList<Rs...>> {
    typedef RStages<N, 1, 0, Rs...> S;
};
template <int N> struct ResTw {
    typedef typename RRun<N, typename ResPlan<N>::type>::S S;
    static constexpr int size = S::tw_size;
};

// Inverse (unnormalised) DFT of npen contiguous pencils (npen the same in
// every thread) held in buf; alt is the second buffer of the out-of-place
// stages.  Returns the buffer holding the result (buf or alt).  The caller has
// synchronised the block after writing buf.  Not inlined: the solver's state
// is saved once around the call instead of spilling inside the butterflies.
// The forward DFT is taken as conj(IDFT(conj x)) (conjugation is exact), with
// the conjugations folded into the loops that fill and read the buffers: one
// transform instantiation keeps the kernel's register allocation free of
// spills, where separate forward and inverse ones did not.
template <int N>
__device__ __noinline__ float2* rifft(float2* buf, float2* alt, int npen, const float2* tws) {
    if (npen <= 0) return buf;
    return ResTw<N>::S::run(buf, alt, npen, tws);
}

}  // namespace hgk
