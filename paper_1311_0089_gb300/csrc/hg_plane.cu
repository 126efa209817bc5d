// Plane passes of the FP32 CG iteration on 3D grids (sm_103a).
//
// One iteration of CG on Eq. final_system (Sec. 5.3) on an N0 x N x N grid is
// three launches instead of the pass kernels' five:
//
//   plane_fwd  one CTA per (load l, axis-0 plane i0, component al):
//              v = r + beta p for the plane's voxels (all d components, the
//              search direction of this iteration), t_al = (A_N v)_al
//              (Sec. 5.1), the partial sum of (v, A v);  the 2D DFT of the
//              plane of t_al in shared memory: real-to-complex along axis 2
//              (two grid rows packed in one complex row), then along axis 1;
//              the plane's spectrum -> S ([k1][k2], the pass kernels'
//              layout);  alpha by the last CTA.
//   strided    axis 0: DFT, Gamma_hat (Eq. Gamma_hat), inverse DFT (the pass
//              kernel).
//   plane_inv  one CTA per (l, i0, al): inverse DFT along axis 1, then
//              complex-to-real along axis 2 -> q = (G_N A_N v)_al on the
//              plane; x += alpha v, r -= alpha q, p = v;  the partial sum of
//              (r, r);  beta and the convergence test by the last CTA.
//
// The axis-1 transforms never leave shared memory, which removes the two
// axis-1 passes (each a read and a write of the whole spectrum).  The search
// direction is formed in both plane passes from r and the previous p and
// stored by plane_inv, because the three CTAs of a plane read every
// component of r and p: none of them may overwrite p while the others read it.
// Between iterations r, p and x hold what the pass kernels leave (p the
// direction of the last iteration), so the two schedules are interchangeable.
//
// Shared memory: the plane U, H rows of W = N + 1 complex entries (the packed
// row pairs of the axis-2 transform; read with stride H, the half spectra
// X_i1(k2) at U[i1 H + k2]), and a group buffer of G pencils: each transform
// runs its out-of-place stages group by group through it and ends in U.
// About 112 KB for N = 135 (two groups of 34 pencils), so that two CTAs share
// an SM and the loads of one overlap the transforms of the other.
#include "hg_pencil.cuh"

namespace hgk {

constexpr int PLANE_D = 3;
// Threads and CTAs per SM of a plane launch (measured per length): N >= 81
// two CTAs of 512 threads; smaller planes four CTAs of 256 (64 registers
// either way)
template <int N> struct PlaneCfg {
    static constexpr int threads = N >= 81 ? 512 : 256;
    static constexpr int blocks = N >= 81 ? 2 : 4;
};
constexpr int PLANE_ALT_BYTES = 36720;   // group buffer budget (two groups of 34 pencils at N = 135)

template <typename Lst> struct Plan2;
template <int R1> struct Plan2<RadixList<R1>> { static constexpr int r1 = R1, r2 = 1, nst = 1; };
template <int R1, int R2> struct Plan2<RadixList<R1, R2>> { static constexpr int r1 = R1, r2 = R2, nst = 2; };

template <int N> struct PlaneGeo {
    typedef Plan2<typename ResPlan<N>::type> P;
    static constexpr int H = (N + 1) / 2;
    static constexpr int W = 2 * H;                    // row stride of U (N + 1)
    static constexpr int NP = N * H;                   // a component's plane spectrum
    static constexpr int UCX = H * W;
    static constexpr int NG = (NP * 8 + PLANE_ALT_BYTES - 1) / PLANE_ALT_BYTES;   // groups per transform
    static constexpr int G = (H + NG - 1) / NG;        // pencils per group
    static constexpr int bytes = (UCX + G * N + ResTw<N>::size) * (int)sizeof(float2);
};

// One inverse Stockham stage over npen pencils of length N: element m of
// pencil p at src[p sps + m ses] -> dst[p dps + m des] (the stage's output
// order).  PEN_FAST: consecutive threads take consecutive pencils (strided
// pencils); else consecutive butterflies of one pencil.  tw: [r-1][k], k < NS.
template <int N, int R, int NS, bool PEN_FAST, int TH = PlaneCfg<N>::threads>
__device__ __forceinline__ void pstage(const float2* __restrict__ src, int sps, int ses, float2* __restrict__ dst,
                                       int dps, int des, int npen, const float2* __restrict__ tw) {
    constexpr int NB = N / R;
    const int total = npen * NB;
#pragma unroll 1
    for (int idx = threadIdx.x; idx < total; idx += TH) {
        int pen, j;
        if (PEN_FAST) { j = idx / npen; pen = idx - j * npen; }
        else { pen = idx / NB; j = idx - pen * NB; }
        const int k = j % NS;
        const float2* sp = src + pen * sps + j * ses;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = sp[r * NB * ses];
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmulw<true>(v[r], tw[(r - 1) * NS + k]);
        }
        DftAny<R, true, float2>::run(v);
        float2* dp = dst + pen * dps + ((j - k) * R + k) * des;
#pragma unroll
        for (int r = 0; r < R; ++r) dp[r * NS * des] = v[r];
    }
    __syncthreads();
}

// Inverse (unnormalised) DFT of npen pencils of U (element m of pencil p at
// U[p ps + m es]), in place: groups of G pencils through alt.  The caller has
// synchronised the block after writing U.  Not inlined (register allocation
// of the surrounding kernel).
template <int N, bool PEN_FAST>
__device__ __noinline__ void plane_ifft(float2* U, int ps, int es, int npen, float2* alt, const float2* tws) {
    typedef PlaneGeo<N> Q;
    for (int g0 = 0; g0 < npen; g0 += Q::G) {
        const int ng = min(Q::G, npen - g0);
        float2* Ug = U + g0 * ps;
        pstage<N, Q::P::r1, 1, PEN_FAST>(Ug, ps, es, alt, N, 1, ng, tws);
        if constexpr (Q::P::nst == 2) {
            pstage<N, Q::P::r2, Q::P::r1, PEN_FAST>(alt, N, 1, Ug, ps, es, ng, tws);
        } else {
            for (int i = threadIdx.x; i < ng * N; i += PlaneCfg<N>::threads) {
                const int pn = i / N, m = i - pn * N;
                Ug[pn * ps + m * es] = alt[i];
            }
            __syncthreads();
        }
    }
}

// L2 prefetch hints for the 128-byte lines that hold [p, p + bytes): line i
// (from the one holding p) by the CTA i mod nparts == part of the nparts that
// share the range, spread over the block's threads.  Every hinted address
// lies inside the range or on the line of its first byte.
__device__ __forceinline__ void l2_prefetch(const void* p, int bytes, int part, int nparts) {
    const unsigned long long a = reinterpret_cast<unsigned long long>(p);
    const unsigned long long a0 = a & ~127ull;
    const int nl = (int)((a + (unsigned long long)bytes - a0 + 127) >> 7);
    for (int i = part + (int)threadIdx.x * nparts; i < nl; i += (int)blockDim.x * nparts) {
        const unsigned long long q = i == 0 ? a : a0 + ((unsigned long long)i << 7);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
    }
}

__device__ __forceinline__ float pick3(const float (&v)[PLANE_D], int al) {
    return al == 0 ? v[0] : (al == 1 ? v[1] : v[2]);
}

// ---------------------------------------------------------------------------
// plane_fwd
// ---------------------------------------------------------------------------
template <int N, typename Args>
__device__ __forceinline__ void plane_fwd_body(const GridDev& g, const float2* __restrict__ tw_nat, Args a,
                                               TileIdx ti) {
    typedef PlaneGeo<N> Q;
    constexpr int H = Q::H, W = Q::W, NP = Q::NP, NN2 = N * N, PT = PlaneCfg<N>::threads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* U = reinterpret_cast<float2*>(smem_raw);
    float2* alt = U + Q::UCX;
    float2* tws = alt + Q::G * N;
    __shared__ float s_tab[SMEM_PHASES * 9];
    __shared__ int s_any, s_act;
    __shared__ float s_beta;
    const int tid = threadIdx.x;
    const int i0 = ti.x / PLANE_D, al = ti.x - PLANE_D * i0, l = ti.y;
    const long long M = g.M;

    if (!a.early_stage) grid_dep_wait();
    ResTw<N>::S::build(tws, tw_nat);
    const float* tab = stage_table<float, PLANE_D>(a.co, s_tab);
    if (a.early_stage) grid_dep_wait();
    if (tid == 0) {
        // a launch in which no system is ACTIVE does no work (no CTA takes a
        // ticket); otherwise every CTA publishes, inactive loads with zeros
        int any = 0;
        for (int k = 0; k < a.L; ++k) any |= (!a.check_status) || (a.sc[k].status == ST_ACTIVE);
        s_any = any;
        s_act = (!a.check_status) || (a.sc[l].status == ST_ACTIVE);
        s_beta = a.sc[l].beta_f;
    }
    __syncthreads();
    if (!s_any) return;
    const bool act = s_act;
    float tacc = 0.f;
    if (act) {
        // v = r + beta p (all components), t_al = (A v)_al; the plane of t_al
        // packed as rows j = i1 / 2 of t(2j, .) + i t(2j + 1, .), stored
        // conjugated (forward DFT = conj(IDFT(conj)))
        const float beta = s_beta;
        const long long pl0 = (long long)i0 * NN2;
        const float* R0 = static_cast<const float*>(a.r) + (long long)l * PLANE_D * M + pl0;
        const float* P0 = static_cast<const float*>(a.p) + (long long)l * PLANE_D * M + pl0;
        CoeffsDev co = a.co;
        if (co.phase) co.phase += pl0;
        if (co.mode == 1) co.field = static_cast<const float*>(a.co.field) + pl0;
        // the plane's r and p (shared by the three CTAs of the plane: a third
        // each) and its coefficients into L2 ahead of the batched loads below
        // (135^3: plane_fwd 169 -> 164 us; at N <= 81 the hints cost 0.5-1.5%
        // of the solve)
        if constexpr (N >= 135) {
            for (int be = 0; be < PLANE_D; ++be) {
                l2_prefetch(R0 + be * M, NN2 * 4, al, PLANE_D);
                l2_prefetch(P0 + be * M, NN2 * 4, al, PLANE_D);
            }
            if (co.mode == 0) l2_prefetch(co.phase, NN2, al, PLANE_D);
        }
        // the global loads of UV voxels (6 UV floats and the phase bytes or
        // field entries) are all issued before any of them is used; the table
        // lookups follow
        constexpr int UV = 4;
        const int mode = co.mode;
        const float* fld = static_cast<const float*>(co.field);
        const int code = al == 0 ? 0x430 : (al == 1 ? 0x513 : 0x254);   // packed 11,22,33,12,13,23
        const long long o0 = (long long)(code & 15) * M, o1 = (long long)((code >> 4) & 15) * M,
                        o2 = (long long)((code >> 8) & 15) * M;
        const int nph1 = co.n_phases - 1;
        for (int e0 = tid; e0 < NN2; e0 += UV * PT) {
            float rv[UV][PLANE_D], pv[UV][PLANE_D], fv[UV][PLANE_D];
            int ph[UV];
#pragma unroll
            for (int u = 0; u < UV; ++u) {
                const int e = min(e0 + u * PT, NN2 - 1);   // (a clamped index is loaded, not used)
                ph[u] = 0;
                fv[u][0] = fv[u][1] = fv[u][2] = 0.f;
                if (mode == 0) {
                    ph[u] = co.phase[e];
                } else if (mode == 1) {
                    fv[u][0] = __ldg(fld + o0 + e);
                    fv[u][1] = __ldg(fld + o1 + e);
                    fv[u][2] = __ldg(fld + o2 + e);
                }
#pragma unroll
                for (int be = 0; be < PLANE_D; ++be) {
                    rv[u][be] = __ldcg(R0 + be * M + e);
                    pv[u][be] = __ldcg(P0 + be * M + e);
                }
            }
#pragma unroll
            for (int u = 0; u < UV; ++u) {
                const int e = e0 + u * PT;
                if (e >= NN2) break;
                float ar[PLANE_D];
                if (mode == 0) {
                    const float* tb = tab + min(ph[u], nph1) * 9 + al * 3;
                    ar[0] = tb[0]; ar[1] = tb[1]; ar[2] = tb[2];
                } else if (mode == 1) {
                    ar[0] = fv[u][0]; ar[1] = fv[u][1]; ar[2] = fv[u][2];
                } else {
                    ar[0] = al == 0 ? 1.f : 0.f;
                    ar[1] = al == 1 ? 1.f : 0.f;
                    ar[2] = al == 2 ? 1.f : 0.f;
                }
                float v[PLANE_D];
#pragma unroll
                for (int be = 0; be < PLANE_D; ++be) v[be] = rv[u][be] + beta * pv[u][be];
                const float t = ar[0] * v[0] + ar[1] * v[1] + ar[2] * v[2];
                tacc += pick3(v, al) * t;
                const int i1 = e / N, i2 = e - i1 * N;
                float* z = reinterpret_cast<float*>(&U[(i1 >> 1) * W + i2]);
                if (i1 & 1) z[1] = -t; else z[0] = t;
            }
        }
        // N is odd: the last packed row holds one grid row
        for (int i2 = tid; i2 < N; i2 += PT) U[(H - 1) * W + i2].y = 0.f;
    }
    __syncthreads();
    if (act) {
        // axis 2 over the H packed rows: Y = IDFT(conj Z), DFT(Z) = conj(Y)
        plane_ifft<N, false>(U, W, 1, H, alt, tws);
        // split each pair in place: row j becomes conj X_2j(k2), k2 < H, then
        // conj X_2j+1(k2), i.e. conj X_i1(k2) at U[i1 H + k2]
        constexpr int RCH = (4 * PT) / H > 0 ? (4 * PT) / H : 1;
        for (int j0 = 0; j0 < H; j0 += RCH) {
            const int nit = min(RCH, H - j0) * H;
            float2 xe[4], xo[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int it = tid + q * PT;
                if (it < nit) {
                    const int j = j0 + it / H, k = it % H;
                    const float2 y1 = U[j * W + k];
                    const float2 y2 = U[j * W + (k ? N - k : 0)];
                    xe[q] = make_float2(0.5f * (y1.x + y2.x), 0.5f * (y1.y - y2.y));
                    xo[q] = make_float2(-0.5f * (y1.y + y2.y), 0.5f * (y1.x - y2.x));
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int it = tid + q * PT;
                if (it < nit) {
                    const int j = j0 + it / H, k = it % H;
                    U[j * W + k] = xe[q];
                    if (2 * j + 1 < N) U[j * W + H + k] = xo[q];
                }
            }
            __syncthreads();
        }
        // axis 1: pencils k2 (stride 1), elements i1 (stride H); the plane's
        // spectrum is the conjugate of the result, at U[k1 H + k2]
        plane_ifft<N, true>(U, 1, H, H, alt, tws);
        grid_dep_launch();
        float2* Sp = static_cast<float2*>(a.S) + ((long long)(l * PLANE_D + al) * g.N[0] + i0) * NP;
        if constexpr (NP % 2 == 0) {
            // an even plane size keeps every plane 16-byte aligned: two entries at a time
            const float4* U4 = reinterpret_cast<const float4*>(U);
            float4* S4 = reinterpret_cast<float4*>(Sp);
            for (int i = tid; i < NP / 2; i += PT) {
                const float4 q = U4[i];
                S4[i] = make_float4(q.x, -q.y, q.z, -q.w);
            }
        } else {
            for (int i = tid; i < NP; i += PT) {
                const float2 q = U[i];
                Sp[i] = make_float2(q.x, -q.y);
            }
        }
    }

    // (v, A v): float-float block sum, FP64 across the CTAs; alpha by the last
    double acc[1];
    const float tv[1] = {tacc};
    block_sum_t<float, 1>(tv, acc);
    const int slot = l;
    const bool last = publish(acc, &slot, 1, a.partial, ti.nx, ti.x, a.counter, (unsigned)(ti.nx * ti.ny));
    if (!last) return;
    double tot[MAXL];
    final_sums<MAXL, float>(a.partial, ti.nx, ti.nx, a.L, tot);
    if (tid == 0) {
        for (int k = 0; k < a.L; ++k) {
            Scalars& s = a.sc[k];
            if (a.check_status && s.status != ST_ACTIVE) continue;
            fwd_cg_scalars(s, tot[k] * g.invM);
        }
        *a.counter = 0u;
    }
}

// ---------------------------------------------------------------------------
// plane_inv
// ---------------------------------------------------------------------------
template <int N, typename Args>
__device__ __forceinline__ void plane_inv_body(const GridDev& g, const float2* __restrict__ tw_nat, Args a,
                                               TileIdx ti) {
    typedef PlaneGeo<N> Q;
    constexpr int H = Q::H, W = Q::W, NP = Q::NP, NN2 = N * N, PT = PlaneCfg<N>::threads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* U = reinterpret_cast<float2*>(smem_raw);
    float2* alt = U + Q::UCX;
    float2* tws = alt + Q::G * N;
    __shared__ int s_any, s_act;
    __shared__ float s_alpha, s_beta;
    const int tid = threadIdx.x;
    const int i0 = ti.x / PLANE_D, al = ti.x - PLANE_D * i0, l = ti.y;
    const long long M = g.M;

    if (!a.early_stage) grid_dep_wait();
    ResTw<N>::S::build(tws, tw_nat);
    if (a.early_stage) grid_dep_wait();
    if (tid == 0) {
        int any = 0;   // see plane_fwd
        for (int k = 0; k < a.L; ++k) any |= (!a.check_status) || (a.sc[k].status == ST_ACTIVE);
        s_any = any;
        s_act = (!a.check_status) || (a.sc[l].status == ST_ACTIVE);
        s_alpha = a.sc[l].alpha_f;
        s_beta = a.sc[l].beta_f;
    }
    __syncthreads();
    if (!s_any) return;
    const bool act = s_act;
    float tacc = 0.f;
    if (act) {
        // the plane's spectrum [k1][k2] -> U[k1 H + k2]
        const float2* Sp = static_cast<const float2*>(a.S) + ((long long)(l * PLANE_D + al) * g.N[0] + i0) * NP;
        if constexpr (N >= 135) l2_prefetch(Sp, NP * 8, 0, 1);
        if constexpr (NP % 2 == 0) {
            // an even plane size keeps every plane 16-byte aligned: two entries at a time
            constexpr int KB = 3, NP2 = NP / 2;
            const float4* S4 = reinterpret_cast<const float4*>(Sp);
            float4* U4 = reinterpret_cast<float4*>(U);
            for (int i0s = tid; i0s < NP2; i0s += KB * PT) {
                float4 v[KB];
#pragma unroll
                for (int u = 0; u < KB; ++u) v[u] = __ldcg(S4 + min(i0s + u * PT, NP2 - 1));
#pragma unroll
                for (int u = 0; u < KB; ++u) {
                    const int i = i0s + u * PT;
                    if (i < NP2) U4[i] = v[u];
                }
            }
        } else {
            constexpr int KB = 6;
            for (int i0s = tid; i0s < NP; i0s += KB * PT) {
                float2 v[KB];
#pragma unroll
                for (int u = 0; u < KB; ++u) v[u] = __ldcg(Sp + min(i0s + u * PT, NP - 1));
#pragma unroll
                for (int u = 0; u < KB; ++u) {
                    const int i = i0s + u * PT;
                    if (i < NP) U[i] = v[u];
                }
            }
        }
        __syncthreads();
        // axis 1: U[i1 H + k2] = X_i1(k2), the half spectra of the grid rows
        plane_ifft<N, true>(U, 1, H, H, alt, tws);
        // x, r and p of the plane into L2 for the update (after the first
        // transform: hints issued at the start of the kernel were evicted
        // before use, DRAM reads 355 -> 439 MB; here plane_inv 166 -> 146 us
        // at the same DRAM traffic, with the spectrum plane's hints above)
        if constexpr (N >= 135) {
            const long long pbase = ((long long)(l * PLANE_D + al)) * M + (long long)i0 * NN2;
            l2_prefetch(static_cast<const float*>(a.x) + pbase, NN2 * 4, 0, 1);
            l2_prefetch(static_cast<const float*>(a.r) + pbase, NN2 * 4, 0, 1);
            l2_prefetch(static_cast<const float*>(a.p) + pbase, NN2 * 4, 0, 1);
        }
        // rows 2j, 2j + 1 as one complex row Z = X_2j + i X_2j+1 over all k2
        // (X(k2) = conj X(N - k2) for k2 >= H), in place: row j of U (stride W)
        // holds X_2j then X_2j+1, and receives Z_j
        constexpr int RCH = (4 * PT) / H > 0 ? (4 * PT) / H : 1;
        for (int j0 = 0; j0 < H; j0 += RCH) {
            const int nit = min(RCH, H - j0) * H;
            float2 xe[4], xo[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int it = tid + q * PT;
                if (it < nit) {
                    const int j = j0 + it / H, k = it % H;
                    xe[q] = U[j * W + k];
                    xo[q] = 2 * j + 1 < N ? U[j * W + H + k] : make_float2(0.f, 0.f);
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int it = tid + q * PT;
                if (it < nit) {
                    const int j = j0 + it / H, k = it % H;
                    // Z(k) = Xe + i Xo;  Z(N - k) = conj(Xe) + i conj(Xo)
                    U[j * W + k] = make_float2(xe[q].x - xo[q].y, xe[q].y + xo[q].x);
                    if (k) U[j * W + N - k] = make_float2(xe[q].x + xo[q].y, xo[q].x - xe[q].y);
                }
            }
            __syncthreads();
        }
        // axis 2 over the rows: q(2j, i2) + i q(2j + 1, i2) at U[j W + i2]
        plane_ifft<N, false>(U, W, 1, H, alt, tws);
        grid_dep_launch();
        const float alpha = s_alpha, beta = s_beta;
        const long long base = ((long long)(l * PLANE_D + al)) * M + (long long)i0 * NN2;
        float* X = static_cast<float*>(a.x) + base;
        float* R = static_cast<float*>(a.r) + base;
        float* P = static_cast<float*>(a.p) + base;
        // one voxel: x += alpha v, r -= alpha q, p = v (v = r + beta p)
        auto upd = [&](int e, float& xv, float& rv, float& pv) {
            const int i1 = e / N, i2 = e - i1 * N;
            const float2 qz = U[(i1 >> 1) * W + i2];
            const float q = (i1 & 1) ? qz.y : qz.x;
            const float v = rv + beta * pv;
            xv = xv + alpha * v;
            rv = rv - alpha * q;
            pv = v;
            tacc += rv * rv;
        };
        // x, r and p of the plane start at the same offset from their (aligned)
        // buffers: the voxels up to a 16-byte boundary one by one, then groups
        // of four as float4, then the rest one by one
        const int head = (int)((4 - (base & 3)) & 3);
        if (tid < head && tid < NN2) {
            float xv = X[tid], rv = R[tid], pv = P[tid];
            upd(tid, xv, rv, pv);
            X[tid] = xv; R[tid] = rv; P[tid] = pv;
        }
        const int n4 = (NN2 - head) >> 2;
        float4* X4 = reinterpret_cast<float4*>(X + head);
        float4* R4 = reinterpret_cast<float4*>(R + head);
        float4* P4 = reinterpret_cast<float4*>(P + head);
        constexpr int UV4 = 2;
        for (int g0 = tid; g0 < n4; g0 += UV4 * PT) {
            float4 xv[UV4], rv[UV4], pv[UV4];
#pragma unroll
            for (int u = 0; u < UV4; ++u) {
                const int gq = min(g0 + u * PT, n4 - 1);   // (a clamped index is loaded, not used)
                xv[u] = __ldcg(X4 + gq);
                rv[u] = __ldcg(R4 + gq);
                pv[u] = __ldcg(P4 + gq);
            }
#pragma unroll
            for (int u = 0; u < UV4; ++u) {
                const int gq = g0 + u * PT;
                if (gq >= n4) break;
                const int e = head + 4 * gq;
                upd(e, xv[u].x, rv[u].x, pv[u].x);
                upd(e + 1, xv[u].y, rv[u].y, pv[u].y);
                upd(e + 2, xv[u].z, rv[u].z, pv[u].z);
                upd(e + 3, xv[u].w, rv[u].w, pv[u].w);
                X4[gq] = xv[u];
                R4[gq] = rv[u];
                P4[gq] = pv[u];
            }
        }
        for (int e = head + 4 * n4 + tid; e < NN2; e += PT) {
            float xv = X[e], rv = R[e], pv = P[e];
            upd(e, xv, rv, pv);
            X[e] = xv; R[e] = rv; P[e] = pv;
        }
    }

    double acc[1];
    const float tv[1] = {tacc};
    block_sum_t<float, 1>(tv, acc);
    const int slot = l;
    const bool last = publish(acc, &slot, 1, a.partial, ti.nx, ti.x, a.counter, (unsigned)(ti.nx * ti.ny));
    if (!last) return;
    double tot[MAXL];
    final_sums<MAXL, float>(a.partial, ti.nx, ti.nx, a.L, tot);
    if (tid == 0) {
        for (int k = 0; k < a.L; ++k) {
            Scalars& s = a.sc[k];
            if (a.check_status && s.status != ST_ACTIVE) continue;
            inv_cg_scalars(s, tot[k] * g.invM);
        }
        *a.counter = 0u;
    }
}

template <int N>
__global__ void __launch_bounds__(PlaneCfg<N>::threads, PlaneCfg<N>::blocks) k_plane_fwd(GridDev g, const float2* __restrict__ tw,
                                                                RowFwdArgs a) {
    plane_fwd_body<N>(g, tw, a, TileIdx::of_block());
}
template <int N>
__global__ void __launch_bounds__(PlaneCfg<N>::threads, PlaneCfg<N>::blocks) k_plane_inv(GridDev g, const float2* __restrict__ tw,
                                                                RowInvArgs a) {
    plane_inv_body<N>(g, tw, a, TileIdx::of_block());
}
// batched: grid z = problem (the arguments of problem z from items)
template <int N>
__global__ void __launch_bounds__(PlaneCfg<N>::threads, PlaneCfg<N>::blocks) k_plane_fwd_b(GridDev g, const float2* __restrict__ tw,
                                                                  const RowFwdArgs* __restrict__ items) {
    plane_fwd_body<N, const RowFwdArgs&>(g, tw, stage_item(items, blockIdx.z), TileIdx::of_block());
}
template <int N>
__global__ void __launch_bounds__(PlaneCfg<N>::threads, PlaneCfg<N>::blocks) k_plane_inv_b(GridDev g, const float2* __restrict__ tw,
                                                                  const RowInvArgs* __restrict__ items) {
    plane_inv_body<N, const RowInvArgs&>(g, tw, stage_item(items, blockIdx.z), TileIdx::of_block());
}

#define HG_PLANE_SIZES(X) X(15) X(27) X(45) X(81) X(135)

bool plane_supported(const GridDev& g) {
    if (g.d != 3 || g.N[1] != g.N[2]) return false;
    switch (g.N[2]) {
#define HG_PC(NV) case NV:
        HG_PLANE_SIZES(HG_PC)
#undef HG_PC
        return true;
        default: return false;
    }
}

// Reduction slots a plane launch needs per load.
long long plane_units(const GridDev& g) { return (long long)g.N[0] * PLANE_D; }

// Plane launches: grid (N0 d, L[, P]), PlaneCfg threads.
cudaError_t launch_plane_fwd(const GridDev& g, const void* tw, const RowFwdArgs& a, cudaStream_t s) {
    const dim3 grid((unsigned)plane_units(g), (unsigned)a.L);
    const float2* twp = static_cast<const float2*>(tw);
    cudaError_t le = cudaErrorInvalidConfiguration;
    switch (g.N[2]) {
#define HG_PC(NV) case NV: le = launch_pdl(k_plane_fwd<NV>, grid, PlaneCfg<NV>::threads, PlaneGeo<NV>::bytes, s, g, twp, a); break;
        HG_PLANE_SIZES(HG_PC)
#undef HG_PC
        default: break;
    }
    return le != cudaSuccess ? le : cudaGetLastError();
}

cudaError_t launch_plane_inv(const GridDev& g, const void* tw, const RowInvArgs& a, cudaStream_t s) {
    const dim3 grid((unsigned)plane_units(g), (unsigned)a.L);
    const float2* twp = static_cast<const float2*>(tw);
    cudaError_t le = cudaErrorInvalidConfiguration;
    switch (g.N[2]) {
#define HG_PC(NV) case NV: le = launch_pdl(k_plane_inv<NV>, grid, PlaneCfg<NV>::threads, PlaneGeo<NV>::bytes, s, g, twp, a); break;
        HG_PLANE_SIZES(HG_PC)
#undef HG_PC
        default: break;
    }
    return le != cudaSuccess ? le : cudaGetLastError();
}

cudaError_t launch_plane_fwd_batch(const GridDev& g, const void* tw, const RowFwdArgs* items, int P, int L,
                                   cudaStream_t s) {
    const dim3 grid((unsigned)plane_units(g), (unsigned)L, (unsigned)P);
    const float2* twp = static_cast<const float2*>(tw);
    cudaError_t le = cudaErrorInvalidConfiguration;
    switch (g.N[2]) {
#define HG_PC(NV) case NV: le = launch_pdl(k_plane_fwd_b<NV>, grid, PlaneCfg<NV>::threads, PlaneGeo<NV>::bytes, s, g, twp, items); break;
        HG_PLANE_SIZES(HG_PC)
#undef HG_PC
        default: break;
    }
    return le != cudaSuccess ? le : cudaGetLastError();
}

cudaError_t launch_plane_inv_batch(const GridDev& g, const void* tw, const RowInvArgs* items, int P, int L,
                                   cudaStream_t s) {
    const dim3 grid((unsigned)plane_units(g), (unsigned)L, (unsigned)P);
    const float2* twp = static_cast<const float2*>(tw);
    cudaError_t le = cudaErrorInvalidConfiguration;
    switch (g.N[2]) {
#define HG_PC(NV) case NV: le = launch_pdl(k_plane_inv_b<NV>, grid, PlaneCfg<NV>::threads, PlaneGeo<NV>::bytes, s, g, twp, items); break;
        HG_PLANE_SIZES(HG_PC)
#undef HG_PC
        default: break;
    }
    return le != cudaSuccess ? le : cudaGetLastError();
}

// ctw: the composite codelets' twiddles (constant memory is per translation
// unit: this one's copy is written here).
cudaError_t configure_plane(const double* ctw) {
    float2 w32[CTW_TOTAL];
    for (int i = 0; i < CTW_TOTAL; ++i) w32[i] = make_float2((float)ctw[2 * i], (float)ctw[2 * i + 1]);
    cudaError_t e = cudaMemcpyToSymbol(c_ctw32, w32, sizeof(w32));
    if (e != cudaSuccess) return e;
#define HG_PC(NV)                                                                                        \
    for (const void* f : {(const void*)k_plane_fwd<NV>, (const void*)k_plane_inv<NV>,                   \
                          (const void*)k_plane_fwd_b<NV>, (const void*)k_plane_inv_b<NV>}) {             \
        const cudaError_t e2 =                                                                           \
            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, PlaneGeo<NV>::bytes);   \
        if (e2 != cudaSuccess) e = e2;                                                                   \
    }
    HG_PLANE_SIZES(HG_PC)
#undef HG_PC
    return e;
}

}  // namespace hgk
