// Resident FP32 conjugate-gradient solver for square 2D grids (sm_103a).
//
// The inner FP32 solve of the mixed-precision path (CG on Eq. final_system,
// Sec. 5.3 Lemma; the operator K = G_N A_N of Eq. FFT_matrices with Gamma_hat
// of Eq. Gamma_hat) as ONE cooperative launch that runs every iteration.  A
// team of CTAs, one per SM, splits the grid into row units (grid row m, load
// l): each CTA keeps r, p, x and s = K p of its row units in tensor memory
// (TMEM, 256 KB per SM, which this path does not otherwise use) for the whole
// solve, so they never travel to HBM; shared memory holds the transforms.
// The iteration is CG in the form of Chronopoulos and Gear (the same iterates
// in exact arithmetic, with w = K r computed in place of K p), so that both
// dot products of an iteration come from one reduction and an iteration is
// two phases of row work and one of column work separated by two grid-wide
// barriers:
//
//   A  (rows)     t = A_N r (Sec. 5.1);  (r, r) and (A r, r) partial sums
//                 ((K r, r) = (A r, r) for r in E_N, Lemma FD_projection);
//                 forward DFT of t along the contiguous axis (the two
//                 components packed as one complex row); half spectra -> S.
//   B  (columns)  the stopping tests on r and the step scalars beta, alpha
//                 from the team's sums; forward DFT along axis 0,
//                 q_hat = Gamma_hat t_hat / |N|, inverse DFT along axis 0, for
//                 the CTA's column units.
//   C  (rows)     the CTA's rows of S by bulk async copies (one mbarrier);
//                 inverse DFT along the contiguous axis -> w = K r;
//                 p = r + beta p, s = w + beta s, x += alpha p, r -= alpha s.
//
// Every CTA sums the team's partial sums itself in one fixed order, so all
// CTAs take the same decisions (step sizes, convergence) without another
// exchange, and the result does not depend on timing.
//
// Waits are bounded: a grid barrier wait that exceeds its limit sets an error
// flag, the other CTAs see it in their own waits, every CTA releases its TMEM
// and returns, and CTA 0 marks the systems ST_TIMEOUT, which the host reports
// as HG_ERR_DEVICE_TIMEOUT.
#include "hg_pencil.cuh"

#include <algorithm>
#include <cstdint>

namespace hgk {

constexpr int RES_THREADS = PEN_THREADS;

// ---------------------------------------------------------------------------
// tensor memory (TMEM) as per-thread storage, bulk async copies, mbarriers
// ---------------------------------------------------------------------------
// r, p, x and s = K p of a thread's voxels live in TMEM (256 KB per SM,
// otherwise unused on this path): warp w reaches TMEM lanes 32 (w mod 4) ..
// + 31, and warps w, w + 4, w + 8, w + 12 use disjoint column groups of 128.
// Slot s of a thread (voxel e = tid + 512 s of its CTA) keeps (r0, r1, p0, p1)
// in columns 4 s .. 4 s + 3, (x0, x1) in columns 64 + 2 s, 64 + 2 s + 1 and
// (s0, s1) in columns 96 + 2 s, 96 + 2 s + 1.
constexpr int RES_SLOTS = 16;                 // slots per thread (multiple of 4)
constexpr int RES_XCOL = 4 * RES_SLOTS;       // first x column of a group
constexpr int RES_SCOL = RES_XCOL + 2 * RES_SLOTS;   // first s column of a group
constexpr int RES_TMEM_COLS = 512;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void tm_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tm_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tm_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tm_st16(uint32_t taddr, const float (&v)[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15, %16};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
                 "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                 "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                 "r"(__float_as_uint(v[15]))
                 : "memory");
}
__device__ __forceinline__ void tm_st8(uint32_t taddr, const float (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// 1-D bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// ---------------------------------------------------------------------------
// bounded grid-wide barrier of the team
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Arrival: every thread's earlier writes are ordered before the counter
// increment (block barrier, then a device-scope fence by thread 0).
__device__ __forceinline__ void team_arrive(unsigned* bar) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
    }
}
// Wait until `target` arrivals; false (in every thread) if the wait gave up
// (time limit, or another CTA's error flag).  At most 2^24 polls as well.
__device__ __forceinline__ bool team_wait(unsigned* bar, unsigned target, int* err,
                                          unsigned long long limit_ns) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long t0 = global_ns();
        unsigned polls = 0;
        while (ld_acquire_u32(bar) < target) {
            ++polls;
            if ((polls & 31u) == 0u) {
                if (*(volatile int*)err != 0 || global_ns() - t0 > limit_ns || polls > (1u << 24)) {
                    ok = 0;
                    atomicExch(err, 1);
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Sum over the team of the two slots of partial array `arr` (pair-packed FP32
// sums hi + lo), in one fixed order in every CTA: lane i adds CTAs i, i + 32,
// ... (all loads issued first), then a fixed shuffle tree.  The additions are
// float-float (Knuth's TwoSum in FP32, the rounding error carried in a second
// float), so the sum keeps about 48 bits where a plain FP32 sum keeps 24, with
// no FP64 instruction until the one conversion at the end.  out[0..1]
// (shared), valid after a block barrier.  T <= 32 * RES_SUM_PER_LANE.
constexpr int RES_SUM_PER_LANE = 8;
__device__ __forceinline__ void ff_add(float& s, float& e, float hi, float lo) {
    const float t = s + hi;                  // TwoSum(s, hi)
    const float bb = t - s;
    const float err = (s - (t - bb)) + (hi - bb);
    s = t;
    e += err + lo;
}
// Split in two so that the loads can be issued early (team_load) and their
// latency overlap other work before the sums are needed (team_reduce).  Warp k
// (k < 4) sums slot k of the CTAs' partials.
struct TeamPart {
    long long w[RES_SUM_PER_LANE];
};
__device__ __forceinline__ void team_load(const double* part, int k, int T, TeamPart& tp) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < RES_SUM_PER_LANE; ++i) {
        const int c = lane + 32 * i;
        tp.w[i] = c < T ? __ldcg(reinterpret_cast<const long long*>(part + (size_t)c * 4 + k)) : 0ll;
    }
}
__device__ __forceinline__ void team_reduce(const TeamPart& tp, double* out) {
    const int lane = threadIdx.x & 31;
    float s0 = 0.f, e0 = 0.f;
#pragma unroll
    for (int i = 0; i < RES_SUM_PER_LANE; ++i)
        ff_add(s0, e0, __int_as_float((int)(tp.w[i] & 0xffffffffll)), __int_as_float((int)(tp.w[i] >> 32)));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float a0 = __shfl_down_sync(0xffffffffu, s0, off), b0 = __shfl_down_sync(0xffffffffu, e0, off);
        ff_add(s0, e0, a0, b0);
    }
    if (lane == 0) *out = (double)s0 + (double)e0;
}

// CTA sum of four per-thread FP32 partials: warp sums in FP32 (32 terms),
// then thread v < 4 adds the 16 warp sums of value v as a float-float pair
// (TwoSum) and writes it, pair-packed, to part[v] (global memory).
__device__ __forceinline__ void block_sum4(const float (&v)[4], double* part) {
    __shared__ float red[4][RES_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float x = v[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) red[i][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        float hi = 0.f, lo = 0.f;
#pragma unroll
        for (int w = 0; w < RES_THREADS / 32; ++w) ff_add(hi, lo, red[threadIdx.x][w], 0.f);
        part[threadIdx.x] = pack_pair(hi, lo);
    }
}

// FP64 1/x and sqrt(x) by Newton-Raphson from FP32 seeds (two steps each:
// 2^-24 -> 2^-48 -> FP64 rounding), a few FMAs on the slow FP64 pipe instead
// of the full division and square-root sequences.
__device__ __forceinline__ double rcp_d(double x) {
    const double ax = fabs(x);
    if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / x;     // outside the FP32 seed's range
    double y = (double)__frcp_rn((float)x);
    y = y * fma(-x, y, 2.0);
    y = y * fma(-x, y, 2.0);
    return y;
}
__device__ __forceinline__ double sqrt_d(double x) {
    if (!(x > 1e-30 && x < 1e30)) return sqrt(x);      // zero, tiny, huge, NaN
    double y = (double)rsqrtf((float)x);       // 1/sqrt(x)
    y = y * fma(-0.5 * x * y, y, 1.5);
    y = y * fma(-0.5 * x * y, y, 1.5);
    return x * y;
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(RES_THREADS, 1) k_cg_resident(ResArgs a) {
    typedef float2 C;
    constexpr int H = (N + 1) / 2;
    constexpr int HP = (H + 1) & ~1;          // padded spectrum row (16-byte multiple)
    constexpr int L = 2;
    constexpr int KB = 16;                    // column loads a thread issues before storing them
    const int T = gridDim.x, c = blockIdx.x, tid = threadIdx.x;
    const size_t M = (size_t)N * N;
    const int u0 = (int)((long long)c * a.units / T);
    const int nu = (int)((long long)(c + 1) * a.units / T) - u0;
    const int v0 = (int)((long long)c * a.cunits / T);
    const int nv = (int)((long long)(c + 1) * a.cunits / T) - v0;
    const int ne = nu * N;                                  // voxels of the CTA's row units
    const int nslot = (ne + RES_THREADS - 1) / RES_THREADS; // <= RES_SLOTS (host-checked)

    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* stage = reinterpret_cast<C*>(smem_raw);                  // [umax][2][HP] spectrum rows (bulk copies)
    C* buf = stage + (size_t)a.umax * 2 * HP;                   // [bufp][N] transforms
    C* buf2 = buf + (size_t)a.bufp * N;                         // [bufp][N] their second buffer
    C* tws = buf2 + (size_t)a.bufp * N;                         // stage twiddles
    unsigned char* ph_s = reinterpret_cast<unsigned char*>(tws + ResTw<N>::size);   // [umax][N]

    __shared__ float s_tab[SMEM_PHASES * 4];
    __shared__ Scalars s_sc[L];
    __shared__ float s_alpha[L], s_beta[L];
    __shared__ int s_act[L];
    __shared__ double s_red[4];
    __shared__ double s_ib2[L];          // 1 / ||b||^2 of each system (the step scalars are
                                         // formed in FP32 from quantities normalised by it)
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) uint64_t s_mbar;

    if (a.drop_cta == c) return;

    // ---- set-up: TMEM, twiddles, coefficients, r = r0, p = s = x = 0 ----
    const int warp = tid >> 5;
    if (warp == 0) tm_alloc(&s_taddr, RES_TMEM_COLS);
    if (tid == 0) mbar_init(&s_mbar, 1);
    ResTw<N>::S::build(tws, a.tw);
    const bool tab_smem = a.co.mode == 0 && a.co.n_phases <= SMEM_PHASES;
    if (tab_smem) {
        const float* tb = static_cast<const float*>(a.co.table);
        for (int i = tid; i < a.co.n_phases * 4; i += RES_THREADS) s_tab[i] = tb[i];
    }
    const float* tab = tab_smem ? s_tab : static_cast<const float*>(a.co.table);
    const float* fld = static_cast<const float*>(a.co.field);
    const int nph1 = a.co.n_phases - 1;
    if (a.co.mode == 0)
        for (int e = tid; e < ne; e += RES_THREADS) {
            const int j = e / N, k = e - j * N;
            ph_s[e] = a.co.phase[(size_t)((u0 + j) >> 1) * N + k];
        }
    if (tid < L) {
        s_sc[tid] = a.sc[tid];
        const double bn = a.sc[tid].bnorm;
        s_ib2[tid] = bn > 0.0 ? 1.0 / (bn * bn) : 0.0;
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    // this thread's TMEM: lane quarter of its warp, column group of its warp quarter
    const uint32_t tbase = s_taddr + ((uint32_t)(32 * (warp & 3)) << 16) + 128u * (uint32_t)(warp >> 2);
    for (int s0 = 0; s0 < nslot; s0 += 4) {
        float rp[16], zz[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = tid + (s0 + i) * RES_THREADS;
            float r0 = 0.f, r1 = 0.f;
            if (e < ne) {
                const int j = e / N, k = e - j * N;
                const int u = u0 + j, m = u >> 1, l = u & 1;
                const size_t o = (size_t)(l * 2) * M + (size_t)m * N + k;
                r0 = a.r0[o];
                r1 = a.r0[o + M];
            }
            rp[4 * i] = r0; rp[4 * i + 1] = r1; rp[4 * i + 2] = 0.f; rp[4 * i + 3] = 0.f;
            zz[2 * i] = 0.f; zz[2 * i + 1] = 0.f;
        }
        tm_st16(tbase + 4 * s0, rp);
        tm_st8(tbase + RES_XCOL + 2 * s0, zz);
        tm_st8(tbase + RES_SCOL + 2 * s0, zz);
    }
    tm_wait_st();

    const float invY0 = a.g.invYf[0], invY1 = a.g.invYf[1], invM = a.g.invMf;
    const double invMd = a.g.invM;
    const int mb0 = a.band[0] > 0 ? (a.band[0] - 1) / 2 : N;
    const int mb1 = a.band[0] > 0 ? (a.band[1] - 1) / 2 : N;
    unsigned seq = 0, mphase = 0;
    bool ok = true;

    // CG in the form of Chronopoulos and Gear (the iterates of Sec. 5.3's CG in
    // exact arithmetic, with w = K r in place of q = K p): both dot products of
    // an iteration, gamma = (r, r) and delta = (K r, r) = (A r, r) (r in E_N,
    // Lemma FD_projection), come from the same reduction, so beta = gamma /
    // gamma_old and alpha = gamma / (delta - beta gamma / alpha_old) are known
    // before the last phase, which updates p = r + beta p, s = w + beta s
    // (s = K p), x += alpha p, r -= alpha s: two grid barriers per iteration.
    for (;;) {
        if (tid < L) s_act[tid] = s_sc[tid].status == ST_ACTIVE;
        __syncthreads();
        if (!(s_act[0] | s_act[1])) break;

        // ---- phase A: t = A r; (r, r), (A r, r); row DFT of t -> S ----
        {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};       // (r, r) loads 0, 1; (A r, r) loads 0, 1
            const int act0 = s_act[0], act1 = s_act[1];
            const bool wgt = a.W.has != 0;
            const float w00 = a.W.wf[0], w01 = a.W.wf[1], w10 = a.W.wf[2], w11 = a.W.wf[3];
            for (int s0 = 0; s0 < nslot; s0 += 4) {
                float rp[16];
                tm_ld16(tbase + 4 * s0, rp);
                tm_wait_ld();
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int e = tid + (s0 + i) * RES_THREADS;
                    if (e >= ne) continue;
                    const int j = e / N, k = e - j * N;
                    const int u = u0 + j, l = u & 1;
                    C t = make_float2(0.f, 0.f);
                    if (l == 0 ? act0 : act1) {
                        const float r0 = rp[4 * i], r1 = rp[4 * i + 1];
                        float a00, a01, a10, a11;
                        if (a.co.mode == 0) {
                            const float* tb = tab + min((int)ph_s[e], nph1) * 4;
                            a00 = tb[0]; a01 = tb[1]; a10 = tb[2]; a11 = tb[3];
                        } else {
                            const size_t mk = (size_t)(u >> 1) * N + k;
                            a00 = __ldg(fld + mk); a11 = __ldg(fld + M + mk); a01 = a10 = __ldg(fld + 2 * M + mk);
                        }
                        t.x = a00 * r0 + a01 * r1;
                        t.y = a10 * r0 + a11 * r1;
                        // (r, r) in the scalar product of the iteration, (W r, r)
                        float wr0 = r0, wr1 = r1;
                        if (wgt) {
                            wr0 = w00 * r0 + w01 * r1;
                            wr1 = w10 * r0 + w11 * r1;
                        }
                        const float g = r0 * wr0 + r1 * wr1;
                        const float dl = r0 * t.x + r1 * t.y;
                        if (l == 0) { acc[0] += g; acc[2] += dl; } else { acc[1] += g; acc[3] += dl; }
                    }
                    buf[e] = make_float2(t.x, -t.y);        // conj(t0 + i t1)
                }
            }
            __syncthreads();
            const C* yb = rifft<N>(buf, buf2, nu, tws);     // conj(DFT(t0 + i t1))
            // Z = t0 + i t1:  T0(k) = (Z(k) + conj Z(-k)) / 2,  T1(k) = (Z(k) - conj Z(-k)) / 2i,
            // with Z(k) = conj yb[k]
            for (int e = tid; e < nu * H; e += RES_THREADS) {
                const int j = e / H, k = e - j * H;
                const int u = u0 + j, m = u >> 1, l = u & 1;
                if (!s_act[l]) continue;
                const C y = yb[j * N + k], ym = yb[j * N + (k ? N - k : 0)];
                C A, B;
                A.x = 0.5f * (y.x + ym.x); A.y = 0.5f * (ym.y - y.y);
                B.x = -0.5f * (y.y + ym.y); B.y = 0.5f * (ym.x - y.x);
                const size_t o = ((size_t)(l * 2) * N + m) * HP + k;
                a.S[o] = A;
                a.S[o + (size_t)N * HP] = B;
            }
            block_sum4(acc, a.part + (size_t)c * 4);
        }
        team_arrive(a.bar);
        if (!(ok = team_wait(a.bar, ++seq * (unsigned)T, a.err, a.wait_ns))) break;

        // ---- phase B: the step scalars; column DFT, Gamma_hat, inverse column DFT ----
        {
            // the team's partials: loaded now (warps 0..3, one sum each), summed
            // after the column loads
            TeamPart tp;
            if (tid < 128) team_load(a.part, warp, T, tp);
            const int ntot = nv * 2 * N;
            for (int i0 = tid; i0 < ntot; i0 += KB * RES_THREADS) {
                C val[KB];
                int dst[KB];
#pragma unroll
                for (int q = 0; q < KB; ++q) {
                    const int idx = i0 + q * RES_THREADS;
                    dst[q] = -1;
                    val[q] = make_float2(0.f, 0.f);
                    if (idx < ntot) {
                        const int j = idx % nv, t2 = idx / nv;
                        const int cc = t2 & 1, m = t2 >> 1;
                        const int v = v0 + j, l = v / H, k = v - l * H;
                        dst[q] = (j * 2 + cc) * N + m;
                        if (s_act[l]) val[q] = __ldcg(&a.S[((size_t)(l * 2 + cc) * N + m) * HP + k]);
                    }
                }
#pragma unroll
                for (int q = 0; q < KB; ++q)
                    if (dst[q] >= 0) buf[dst[q]] = make_float2(val[q].x, -val[q].y);   // conjugated
            }
            if (tid < 128) team_reduce(tp, &s_red[warp]);
            __syncthreads();
            // stopping tests on r_i (the iterate x_i is final when they hold), then
            // beta_i, alpha_i (Moulinec-Suquet: beta = 0, alpha = 1 / lambda)
            if (tid == 0 || tid == 32) {
                const int l = tid >> 5;
                if (s_act[l]) {
                    Scalars sc = s_sc[l];
                    const double ib2 = s_ib2[l];
                    const double g = s_red[l] * invMd;          // gamma = (r, r)
                    const double dl = s_red[2 + l] * invMd;     // delta = (A r, r)
                    // the decisions and steps in FP32 on quantities normalised by
                    // ||b||^2 (O(1), no FP32 under- or overflow), a few FP64 products
                    const float gn = (float)(g * ib2);
                    const float dn = (float)(dl * ib2);
                    const float gn_old = (float)(sc.rr * ib2);
                    if (sc.iters > 0) {
                        const float rel = sqrtf(gn);
                        sc.relres = rel;
                        // Moulinec-Suquet stops on the step just taken, x_i - x_{i-1} =
                        // r_{i-1} / lambda (the tolerance was rescaled at the right-hand side)
                        const float crit = sc.fixed_alpha > 0.0 ? sqrtf(gn_old) : rel;
                        if (!isfinite(g)) sc.status = ST_BREAKDOWN;
                        else if ((double)crit <= sc.tol) sc.status = ST_CONVERGED;
                        else if (sc.iters >= sc.max_iter) sc.status = ST_MAXITER;
                        if (sc.stall_max > 0 && sc.status == ST_ACTIVE) {
                            if (g < 0.25 * sc.best_rr) {
                                sc.best_rr = g;
                                sc.stall = 0;
                            } else if (++sc.stall >= sc.stall_max) {
                                sc.status = ST_STAGNATED;
                            }
                        }
                    }
                    if (sc.status == ST_ACTIVE) {
                        float beta = 0.f, alpha = 0.f, den = dn;
                        if (sc.fixed_alpha > 0.0) {
                            alpha = (float)sc.fixed_alpha;
                            if (g == 0.0) sc.status = ST_CONVERGED;   // the fixed point, exactly
                        } else {
                            if (sc.iters > 0) {
                                beta = gn / gn_old;
                                den = dn - beta * gn / sc.alpha_f;
                            }
                            if (!(den > 0.f) || !isfinite(den)) sc.status = ST_BREAKDOWN;
                            else alpha = gn / den;
                        }
                        if (sc.status == ST_ACTIVE) {
                            sc.iters += 1;
                            sc.total_iters += 1;
                        }
                        sc.pt = ib2 > 0.0 ? (double)den / ib2 : 0.0;
                        sc.beta = beta;
                        sc.alpha = sc.fixed_alpha > 0.0 ? sc.fixed_alpha : (double)alpha;
                        sc.beta_f = beta;
                        sc.alpha_f = alpha;
                    }
                    sc.rr = g;
                    s_alpha[l] = sc.alpha_f;
                    s_beta[l] = sc.beta_f;
                    s_act[l] = sc.status == ST_ACTIVE;
                    s_sc[l] = sc;
                }
            }
            __syncthreads();
            if (!(s_act[0] | s_act[1])) break;     // every system has stopped at x_i
            C* th = rifft<N>(buf, buf2, 2 * nv, tws);       // conj(t_hat)
            // q_hat = xi (xi . t_hat) / (xi . A0 xi) / |N|   (dual: onto J_N)
            for (int e = tid; e < nv * N; e += RES_THREADS) {
                const int j = e / N, mr = e - j * N;
                const int v = v0 + j, l = v / H, k = v - l * H;
                if (!s_act[l]) continue;
                C* b0 = th + (j * 2) * N + mr;
                C* b1 = b0 + N;
                const C th0 = make_float2(b0->x, -b0->y), th1 = make_float2(b1->x, -b1->y);
                const int fm = 2 * mr <= N - 1 ? mr : mr - N;
                const float xi0 = (float)fm * invY0, xi1 = (float)k * invY1;
                float den;
                if (a.has_A0) {
                    den = xi0 * (a.A0[0] * xi0 + a.A0[1] * xi1) + xi1 * (a.A0[2] * xi0 + a.A0[3] * xi1);
                } else {
                    den = xi0 * xi0 + xi1 * xi1;
                }
                const bool inb = fm <= mb0 && -fm <= mb0 && k <= mb1;
                C s = make_float2(0.f, 0.f);
                const bool keep = den > 0.f && inb;
                if (keep) {
                    const float f = __fdividef(invM, den);
                    s.x = (xi0 * th0.x + xi1 * th1.x) * f;
                    s.y = (xi0 * th0.y + xi1 * th1.y) * f;
                }
                if (a.dual) {
                    *b0 = keep ? make_float2(th0.x * invM - s.x * xi0, th0.y * invM - s.y * xi0) : make_float2(0.f, 0.f);
                    *b1 = keep ? make_float2(th1.x * invM - s.x * xi1, th1.y * invM - s.y * xi1) : make_float2(0.f, 0.f);
                } else {
                    *b0 = make_float2(s.x * xi0, s.y * xi0);
                    *b1 = make_float2(s.x * xi1, s.y * xi1);
                }
            }
            __syncthreads();
            const C* qb = rifft<N>(th, th == buf ? buf2 : buf, 2 * nv, tws);
            for (int idx = tid; idx < ntot; idx += RES_THREADS) {
                const int j = idx % nv, t2 = idx / nv;
                const int cc = t2 & 1, m = t2 >> 1;
                const int v = v0 + j, l = v / H, k = v - l * H;
                if (s_act[l]) a.S[((size_t)(l * 2 + cc) * N + m) * HP + k] = qb[(j * 2 + cc) * N + m];
            }
        }
        team_arrive(a.bar);
        if (!(ok = team_wait(a.bar, ++seq * (unsigned)T, a.err, a.wait_ns))) break;

        // ---- phase C: row inverse DFT -> w = K r; p, s, x, r updates ----
        {
            // the CTA's spectrum rows: one bulk copy per row, on the mbarrier
            if (tid == 0) {
                asm volatile("fence.proxy.async.global;" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&s_mbar, (uint32_t)(nu * 2 * HP * sizeof(C)));
                for (int j = 0; j < nu; ++j) {
                    const int u = u0 + j, m = u >> 1, l = u & 1;
                    for (int cc = 0; cc < 2; ++cc)
                        bulk_g2s(stage + (size_t)(j * 2 + cc) * HP, a.S + ((size_t)(l * 2 + cc) * N + m) * HP,
                                 (uint32_t)(HP * sizeof(C)), &s_mbar);
                }
            }
            {
                int got = 0;
                for (int it = 0; it < (1 << 24); ++it)
                    if (mbar_try_wait(&s_mbar, mphase)) { got = 1; break; }
                mphase ^= 1u;
                if (!__syncthreads_and(got)) {
                    // the copies never completed: the kernel cannot continue
                    if (tid == 0) atomicExch(a.err, 1);
                    ok = false;
                    break;
                }
            }
            // Z = a + i b from the half spectra of the pair (X(k) = conj X(N - k) for k >= H)
            for (int e = tid; e < ne; e += RES_THREADS) {
                const int j = e / N, kk = e - j * N;
                const int ks = kk >= H ? N - kk : kk;
                C w0 = stage[(j * 2) * HP + ks], w1 = stage[(j * 2 + 1) * HP + ks];
                if (kk >= H) { w0.y = -w0.y; w1.y = -w1.y; }
                buf[e] = make_float2(w0.x - w1.y, w0.y + w1.x);
            }
            __syncthreads();
            const C* wr = rifft<N>(buf, buf2, nu, tws);     // w = K r
            const float al0 = s_alpha[0], al1 = s_alpha[1];
            const float be0 = s_beta[0], be1 = s_beta[1];
            const int act0 = s_act[0], act1 = s_act[1];
            for (int s0 = 0; s0 < nslot; s0 += 4) {
                float rp[16], xx[8], ss[8];
                tm_ld16(tbase + 4 * s0, rp);
                tm_ld8(tbase + RES_XCOL + 2 * s0, xx);
                tm_ld8(tbase + RES_SCOL + 2 * s0, ss);
                tm_wait_ld();
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int e = tid + (s0 + i) * RES_THREADS;
                    if (e >= ne) continue;
                    const int j = e / N;
                    const int l = (u0 + j) & 1;
                    if (!(l == 0 ? act0 : act1)) continue;
                    const float al = l == 0 ? al0 : al1;
                    const float be = l == 0 ? be0 : be1;
                    const C w = wr[e];
                    const float p0 = rp[4 * i] + be * rp[4 * i + 2];
                    const float p1 = rp[4 * i + 1] + be * rp[4 * i + 3];
                    const float s0v = w.x + be * ss[2 * i];
                    const float s1v = w.y + be * ss[2 * i + 1];
                    rp[4 * i + 2] = p0;
                    rp[4 * i + 3] = p1;
                    ss[2 * i] = s0v;
                    ss[2 * i + 1] = s1v;
                    xx[2 * i] += al * p0;
                    xx[2 * i + 1] += al * p1;
                    rp[4 * i] -= al * s0v;
                    rp[4 * i + 1] -= al * s1v;
                }
                tm_st16(tbase + 4 * s0, rp);
                tm_st8(tbase + RES_XCOL + 2 * s0, xx);
                tm_st8(tbase + RES_SCOL + 2 * s0, ss);
            }
            tm_wait_st();
        }
    }

    // x of the inner system back to global memory; scalars (CTA 0)
    if (ok) {
        for (int s0 = 0; s0 < nslot; s0 += 4) {
            float xx[8];
            tm_ld8(tbase + RES_XCOL + 2 * s0, xx);
            tm_wait_ld();
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int e = tid + (s0 + i) * RES_THREADS;
                if (e >= ne) continue;
                const int j = e / N, k = e - j * N;
                const int u = u0 + j, m = u >> 1, l = u & 1;
                const size_t o = (size_t)(l * 2) * M + (size_t)m * N + k;
                a.x[o] = xx[2 * i];
                a.x[o + M] = xx[2 * i + 1];
            }
        }
    }
    if (c == 0 && tid < L) {
        Scalars s = s_sc[tid];
        if (!ok) s.status = ST_TIMEOUT;
        a.sc[tid] = s;
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (warp == 0) tm_dealloc(s_taddr, RES_TMEM_COLS);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
bool resident_length(int n) {
    switch (n) {
#define HG_RES_CASE(NV) case NV: return true;
        HG_RES_SIZES(HG_RES_CASE)
#undef HG_RES_CASE
        default: return false;
    }
}

static int res_tw_size(int n) {
    switch (n) {
#define HG_RES_CASE(NV) case NV: return ResTw<NV>::size;
        HG_RES_SIZES(HG_RES_CASE)
#undef HG_RES_CASE
        default: return 0;
    }
}

bool resident_cfg(int n, int L, int T, int nsm, int max_smem, ResCfg& cfg) {
    if (!resident_length(n) || L != 2 || nsm < 1) return false;
    const int H = (n + 1) / 2;
    const int HP = (H + 1) & ~1;
    const int units = n * L, cunits = H * L;
    if (T <= 0) T = std::min(nsm, std::max(1, units / 4));
    T = std::min(T, std::min(nsm, std::min(units, cunits)));
    T = std::min(T, 32 * RES_SUM_PER_LANE);
    if (T < 1) return false;
    const int umax = (units + T - 1) / T;
    const int vmax = (cunits + T - 1) / T;
    // r, p and x of a thread's voxels fit its TMEM slots
    if ((umax * n + RES_THREADS - 1) / RES_THREADS > RES_SLOTS) return false;
    const int bufp = std::max(umax, 2 * vmax);
    size_t smem = (size_t)umax * 2 * HP * sizeof(float2)      // spectrum rows (bulk copies)
                  + (size_t)2 * bufp * n * sizeof(float2)     // transform buffers
                  + (size_t)res_tw_size(n) * sizeof(float2)   // stage twiddles
                  + (size_t)umax * n;                         // phase bytes
    smem = (smem + 15) & ~(size_t)15;
    if (smem > (size_t)max_smem) return false;
    // every CTA takes all of its SM's TMEM columns: ask for more than half the
    // shared memory so that no two CTAs of the launch share an SM (a second
    // one's allocation would wait for the first to leave)
    smem = std::max(smem, (size_t)max_smem / 2 + 1024);
    if (smem > (size_t)max_smem) return false;
    cfg.T = T;
    cfg.umax = umax;
    cfg.bufp = bufp;
    cfg.smem = (int)smem;
    return true;
}

template <int N>
static cudaError_t launch_res_t(const ResArgs& a, const ResCfg& cfg, cudaStream_t s) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)cfg.T);
    lc.blockDim = dim3(RES_THREADS);
    lc.dynamicSmemBytes = (size_t)cfg.smem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, k_cg_resident<N>, a);
}

cudaError_t launch_resident(int n, const ResArgs& a, const ResCfg& cfg, cudaStream_t s) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (n) {
#define HG_RES_CASE(NV) case NV: e = launch_res_t<NV>(a, cfg, s); break;
        HG_RES_SIZES(HG_RES_CASE)
#undef HG_RES_CASE
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t configure_resident(int max_smem, const double* ctw) {
    float2 w32[CTW_TOTAL];
    for (int i = 0; i < CTW_TOTAL; ++i) w32[i] = make_float2((float)ctw[2 * i], (float)ctw[2 * i + 1]);
    cudaError_t e = cudaMemcpyToSymbol(c_ctw32, w32, sizeof(w32));
    if (e != cudaSuccess) return e;
#define HG_RES_CASE(NV)                                                                              \
    {                                                                                                \
        cudaError_t e2 = cudaFuncSetAttribute(k_cg_resident<NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                              max_smem);                                             \
        if (e2 != cudaSuccess) e = e2;                                                               \
    }
    HG_RES_SIZES(HG_RES_CASE)
#undef HG_RES_CASE
    return e;
}

}  // namespace hgk
