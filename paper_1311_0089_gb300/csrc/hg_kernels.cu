// CUDA helper kernels of the CG solve (scalars, mixed-precision refinement,
// homogenized matrix, conversions) and the precision dispatch of the pass
// kernels (hg_kernels.cuh, instantiated in hg_kernels_f32.cu / _f64.cu).
#include "hg_kernels.cuh"

namespace hgk {

// ---------------------------------------------------------------------------
// helpers: scalars init, mixed-precision refinement, A_H, conversions
// ---------------------------------------------------------------------------
__global__ void k_init_scalars(Scalars* sc, int L, int s0, int s1, int s2, double tol, int max_iter,
                               double fixed_alpha, double zscale) {
    const int l = threadIdx.x;
    if (l >= L) return;
    Scalars s;
    s.rr = 0; s.pt = 0; s.alpha = 0; s.beta = 0; s.bnorm = 0; s.aen = 0; s.relres = 1.0;
    s.alpha_f = 0.f; s.beta_f = 0.f; s.best_rr = 0.0; s.stall = 0; s.stall_max = 0;
    s.fixed_alpha = fixed_alpha;
    s.zscale = zscale;
    s.tol = tol; s.iters = 0; s.max_iter = max_iter; s.total_iters = 0;
    s.status = (l == 0) ? s0 : (l == 1) ? s1 : s2;
    sc[l] = s;
}

template <int D>
__global__ void __launch_bounds__(256) k_inner_init(GridDev g, int L, const double* __restrict__ r64,
                                                    float* __restrict__ r32, float* __restrict__ p32,
                                                    float* __restrict__ x32, const Scalars* __restrict__ outer,
                                                    Scalars* inner, double inner_tol, int inner_max,
                                                    int stall_max, Weight W, double* partial,
                                                    unsigned* counter) {
    const long long M = g.M;
    const long long n = (long long)L * M;
    double acc[MAXL] = {0.0, 0.0, 0.0};
    bool act[MAXL];
    for (int l = 0; l < MAXL; ++l) act[l] = (l < L) && outer[l].status == ST_ACTIVE;
    double tot[MAXL];
    if (r64) {
        // one voxel of one load per step: the D components together for (W r, r)
        for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
             idx += (long long)gridDim.x * blockDim.x) {
            const int l = (int)(idx / M);
            if (!act[l]) continue;
            const long long k = idx - (long long)l * M;
            double v[D];
#pragma unroll
            for (int al = 0; al < D; ++al) {
                const long long o = ((long long)l * D + al) * M + k;
                const float f = (float)r64[o];
                r32[o] = f;
                p32[o] = f;
                x32[o] = 0.f;
                v[al] = (double)f;
            }
            double q = 0.0;
#pragma unroll
            for (int al = 0; al < D; ++al) {
                double wv = v[al];
                if (W.has) {
                    wv = 0.0;
#pragma unroll
                    for (int be = 0; be < D; ++be) wv += W.w[al * D + be] * v[be];
                }
                q += v[al] * wv;
            }
            if (l == 0) acc[0] += q; else if (l == 1) acc[1] += q; else acc[2] += q;
        }
        block_sum<MAXL>(acc);
        int slots[MAXL] = {0, 1, 2};
        const bool last = publish(acc, slots, L, partial, gridDim.x, blockIdx.x, counter, gridDim.x);
        if (!last) return;
        final_sums<MAXL>(partial, gridDim.x, gridDim.x, L, tot);
    } else {
        for (int l = 0; l < MAXL; ++l) tot[l] = l < L ? outer[l].rr : 0.0;   // (b, b), normalised
    }
    if (threadIdx.x == 0) {
        for (int l = 0; l < L; ++l) {
            Scalars s;
            // inner target: reduce the current FP64 residual just enough to reach
            // the outer tolerance (half of it), never looser than 0.5 nor tighter
            // than inner_tol
            const double need = 0.5 * outer[l].tol / fmax(outer[l].relres, 1e-300);
            const double itol = fmin(0.5, fmax(inner_tol, need));
            s.rr = r64 ? tot[l] * g.invM : tot[l]; s.pt = 0; s.alpha = 0; s.beta = 0; s.alpha_f = 0.f; s.beta_f = 0.f;
            // an inner FP32 solve that stops improving ends; the FP64
            // refinement decides whether another inner solve is needed
            s.best_rr = s.rr; s.stall = 0; s.stall_max = stall_max;
            s.fixed_alpha = outer[l].fixed_alpha;
            s.zscale = outer[l].zscale;
            s.bnorm = sqrt(s.rr); s.aen = 0; s.relres = 1.0; s.tol = itol;
            s.iters = 0; s.max_iter = inner_max; s.total_iters = 0;
            s.status = act[l] ? (s.rr > 0.0 ? ST_ACTIVE : ST_CONVERGED)
                              : (outer[l].status == ST_RHS_RECHECK ? ST_RHS_RECHECK : ST_IDLE);
            inner[l] = s;
        }
        if (r64) *counter = 0u;
    }
}

template <int D>
__global__ void __launch_bounds__(256) k_outer_update(GridDev g, int L, double* __restrict__ x64,
                                                      const float* __restrict__ x32, Scalars* outer,
                                                      const Scalars* __restrict__ inner) {
    const long long M = g.M;
    const long long n = (long long)L * D * M;
    bool act[MAXL];
    for (int l = 0; l < MAXL; ++l) act[l] = (l < L) && outer[l].status == ST_ACTIVE;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(idx / (D * M));
        if (act[l]) x64[idx] += (double)x32[idx];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int l = 0; l < L; ++l)
            if (act[l]) { outer[l].iters += 1; outer[l].total_iters += inner[l].iters; }
    }
}

template <int D>
__global__ void __launch_bounds__(256) k_energy(GridDev g, int L, CoeffsDev co, const double* __restrict__ x,
                                                unsigned mask, double* partial, unsigned* counter,
                                                double* out) {
    constexpr int NV = 2 * D * D;
    const long long M = g.M;
    double acc[NV];
#pragma unroll
    for (int s = 0; s < NV; ++s) acc[s] = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < M;
         k += (long long)gridDim.x * blockDim.x) {
        double am[D][D];
        load_coeffs<double, D>(co, k, M, am, static_cast<const double*>(co.table));
        double e[D][D], f[D][D];   // e[j] = E_j + x_j ; f[j] = A e[j]
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const bool on = (j < L) && ((mask >> j) & 1u);
#pragma unroll
            for (int al = 0; al < D; ++al)
                e[j][al] = on ? ((al == j ? 1.0 : 0.0) + x[((long long)j * D + al) * M + k]) : 0.0;
#pragma unroll
            for (int al = 0; al < D; ++al) {
                double s = 0.0;
#pragma unroll
                for (int be = 0; be < D; ++be) s += am[al][be] * e[j][be];
                f[j][al] = s;
            }
        }
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                double s = 0.0;
#pragma unroll
                for (int al = 0; al < D; ++al) s += f[j][al] * e[i][al];
                acc[i * D + j] += s;
                acc[D * D + i * D + j] += f[j][i];
            }
    }
    block_sum<NV>(acc);
    int slots[NV];
    for (int s = 0; s < NV; ++s) slots[s] = s;
    const bool last = publish(acc, slots, NV, partial, gridDim.x, blockIdx.x, counter, gridDim.x);
    if (!last) return;
    double tot[NV];
    final_sums<NV>(partial, gridDim.x, gridDim.x, NV, tot);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NV; ++s) out[s] = tot[s] * g.invM;
        *counter = 0u;
    }
}

// Eigenvalues of a symmetric D x D matrix by cyclic Jacobi rotations (Golub
// and Van Loan, Matrix Computations, Sec. 8.5): each rotation in the (p, q)
// plane zeroes a_pq; the diagonal converges to the eigenvalues with absolute
// error of order eps ||A||, also for nearly equal eigenvalues.
template <int D>
__device__ __forceinline__ void sym_eig_jacobi(double (&a)[D][D], double (&ev)[D]) {
    for (int sweep = 0; sweep < 12; ++sweep) {
        double off = 0.0, dia = 0.0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            dia += fabs(a[i][i]);
#pragma unroll
            for (int j = i + 1; j < D; ++j) off += fabs(a[i][j]);
        }
        if (off <= 1e-18 * dia) break;
#pragma unroll
        for (int p = 0; p < D - 1; ++p) {
#pragma unroll
            for (int q = p + 1; q < D; ++q) {
                const double apq = a[p][q];
                if (apq == 0.0) continue;
                // tan of the rotation angle: the smaller root of t^2 + 2 theta t - 1 = 0
                const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0);
                const double sn = t * c;
                a[p][p] -= t * apq;
                a[q][q] += t * apq;
                a[p][q] = a[q][p] = 0.0;
#pragma unroll
                for (int r = 0; r < D; ++r) {
                    if (r == p || r == q) continue;
                    const double arp = a[r][p], arq = a[r][q];
                    a[r][p] = a[p][r] = c * arp - sn * arq;
                    a[r][q] = a[q][r] = sn * arp + c * arq;
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < D; ++i) ev[i] = a[i][i];
}

// min and max eigenvalue of A(x_k) over all voxels.  Eigenvalues of SPD
// matrices are positive, so their FP64 bit patterns order like the values
// and the grid-wide min/max are integer atomics (order-independent).
template <int D>
__global__ void __launch_bounds__(256) k_coeff_bounds(GridDev g, CoeffsDev co,
                                                      unsigned long long* bounds) {
    const long long M = g.M;
    double lo = INFINITY, hi = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < M;
         k += (long long)gridDim.x * blockDim.x) {
        double am[D][D], ev[D];
        load_coeffs<double, D>(co, k, M, am, static_cast<const double*>(co.table));
        sym_eig_jacobi<D>(am, ev);
#pragma unroll
        for (int i = 0; i < D; ++i) { lo = fmin(lo, ev[i]); hi = fmax(hi, ev[i]); }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&bounds[0], (unsigned long long)__double_as_longlong(fmax(lo, 0.0)));
        atomicMax(&bounds[1], (unsigned long long)__double_as_longlong(fmax(hi, 0.0)));
    }
}

// Inverse of a symmetric positive definite matrix as its adjugate over its
// determinant (cofactor expansion), per voxel of a packed field.
template <int D>
__global__ void __launch_bounds__(256) k_invert_field(long long M, const double* __restrict__ in,
                                                      double* __restrict__ out64, float* __restrict__ out32) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < M;
         k += (long long)gridDim.x * blockDim.x) {
        if (D == 2) {
            const double a = in[k], b = in[M + k], c = in[2 * M + k];   // a11, a22, a12
            const double det = a * b - c * c;
            const double r[3] = {b / det, a / det, -c / det};
            for (int q = 0; q < 3; ++q) { out64[q * M + k] = r[q]; out32[q * M + k] = (float)r[q]; }
        } else {
            const double a = in[k], b = in[M + k], c = in[2 * M + k];            // a11, a22, a33
            const double d = in[3 * M + k], e = in[4 * M + k], f = in[5 * M + k];  // a12, a13, a23
            const double c11 = b * c - f * f, c22 = a * c - e * e, c33 = a * b - d * d;
            const double c12 = e * f - d * c, c13 = d * f - b * e, c23 = d * e - a * f;
            const double det = a * c11 + d * c12 + e * c13;
            const double r[6] = {c11 / det, c22 / det, c33 / det, c12 / det, c13 / det, c23 / det};
            for (int q = 0; q < 6; ++q) { out64[q * M + k] = r[q]; out32[q * M + k] = (float)r[q]; }
        }
    }
}

// dst[p * MAXL + l] = src[p][l]: the scalars of P problems in one buffer.
__global__ void k_gather_scalars(const Scalars* const* __restrict__ src, Scalars* dst, int P) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P * MAXL) dst[i] = src[i / MAXL][i % MAXL];
}

template <typename S, typename Dd>
__global__ void k_convert(const S* __restrict__ src, Dd* __restrict__ dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = (Dd)src[i];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int g_sm_count = 0;

static int sm_count() {
    if (g_sm_count == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count <= 0) g_sm_count = 1;
    }
    return g_sm_count;
}

int row_max_threads() { return MAXT; }

bool ct_length(int d, int n) {
    switch (n) {
        case 15: case 27: case 45: case 81: case 135: return true;
        case 75: case 243: case 375: case 729: return d == 2;
        default: return false;
    }
}

int ct_npmax(int prec, int n) {
    const int csize = prec == 0 ? 16 : 8;
    int v = (48 * 1024) / (n * csize);
    return v < 1 ? 1 : (v > 16 ? 16 : v);
}

cudaError_t configure_kernels(int max_smem) {
    // W_R^m = exp(-2 pi i m / R) for the composite codelets, extended precision
    double ctw[2 * CTW_TOTAL];
    const int Rs[4] = {9, 15, 25, 27};
    const int off[4] = {CTW_9, CTW_15, CTW_25, CTW_27};
    for (int q = 0; q < 4; ++q)
        for (int m = 0; m < Rs[q]; ++m) {
            const long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)m / (long double)Rs[q];
            ctw[2 * (off[q] + m)] = (double)cosl(ang);
            ctw[2 * (off[q] + m) + 1] = (double)sinl(ang);
        }
    cudaError_t e = configure_f64(max_smem, ctw);
    cudaError_t e2 = configure_f32(max_smem, ctw);
    cudaError_t e3 = configure_resident(max_smem, ctw);
    cudaError_t e4 = configure_plane(ctw);
    return e != cudaSuccess ? e : (e2 != cudaSuccess ? e2 : (e3 != cudaSuccess ? e3 : e4));
}

cudaError_t launch_row_fwd(int prec, const GridDev& g, const AxisPlanH& pl, const void* tw,
                           const RowCfg& cfg, const RowFwdArgs& a, cudaStream_t s) {
    return prec == 0 ? launch_row_fwd_f64(g, pl, tw, cfg, a, s) : launch_row_fwd_f32(g, pl, tw, cfg, a, s);
}

cudaError_t launch_strided(int prec, const GridDev& g, const AxisPlanH& pl, const void* tw,
                           const StrCfg& cfg, const StrArgs& a, cudaStream_t s) {
    return prec == 0 ? launch_strided_f64(g, pl, tw, cfg, a, s) : launch_strided_f32(g, pl, tw, cfg, a, s);
}

cudaError_t launch_row_inv(int prec, const GridDev& g, const AxisPlanH& pl, const void* tw,
                           const RowCfg& cfg, const RowInvArgs& a, cudaStream_t s) {
    return prec == 0 ? launch_row_inv_f64(g, pl, tw, cfg, a, s) : launch_row_inv_f32(g, pl, tw, cfg, a, s);
}

cudaError_t launch_row_fwd_batch(int prec, const GridDev& g, const AxisPlanH& pl, const void* tw,
                                 const RowCfg& cfg, const RowFwdArgs* items, int P, int L, cudaStream_t s) {
    return prec == 0 ? launch_row_fwd_batch_f64(g, pl, tw, cfg, items, P, L, s)
                     : launch_row_fwd_batch_f32(g, pl, tw, cfg, items, P, L, s);
}

cudaError_t launch_row_inv_batch(int prec, const GridDev& g, const AxisPlanH& pl, const void* tw,
                                 const RowCfg& cfg, const RowInvArgs* items, int P, int L, cudaStream_t s) {
    return prec == 0 ? launch_row_inv_batch_f64(g, pl, tw, cfg, items, P, L, s)
                     : launch_row_inv_batch_f32(g, pl, tw, cfg, items, P, L, s);
}

cudaError_t launch_strided_batch(int prec, const GridDev& g, const AxisPlanH& pl, const void* tw,
                                 const StrCfg& cfg, const StrArgs* items, int P, int L, int n,
                                 long long inner, long long outer, cudaStream_t s) {
    return prec == 0 ? launch_strided_batch_f64(g, pl, tw, cfg, items, P, L, n, inner, outer, s)
                     : launch_strided_batch_f32(g, pl, tw, cfg, items, P, L, n, inner, outer, s);
}

cudaError_t launch_init_scalars(Scalars* sc, int L, const int* st, double tol, int max_iter,
                                double fixed_alpha, double zscale, cudaStream_t s) {
    k_init_scalars<<<1, 32, 0, s>>>(sc, L, st[0], L > 1 ? st[1] : ST_IDLE, L > 2 ? st[2] : ST_IDLE,
                                    tol, max_iter, fixed_alpha, zscale);
    return cudaGetLastError();
}

static unsigned elem_grid(long long n) {
    long long b = (n + 255) / 256;
    long long cap = 4LL * sm_count();
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

cudaError_t launch_inner_init(const GridDev& g, int L, const double* r64, float* r32, float* p32,
                              float* x32, const Scalars* outer, Scalars* inner, double inner_tol,
                              int inner_max, int stall_max, const Weight& W, double* partial,
                              unsigned* counter, cudaStream_t s) {
    unsigned nb = r64 ? elem_grid((long long)L * g.M) : 1u;
    if (g.d == 2)
        k_inner_init<2><<<nb, 256, 0, s>>>(g, L, r64, r32, p32, x32, outer, inner, inner_tol, inner_max,
                                           stall_max, W, partial, counter);
    else
        k_inner_init<3><<<nb, 256, 0, s>>>(g, L, r64, r32, p32, x32, outer, inner, inner_tol, inner_max,
                                           stall_max, W, partial, counter);
    return cudaGetLastError();
}

cudaError_t launch_outer_update(const GridDev& g, int L, double* x64, const float* x32,
                                Scalars* outer, const Scalars* inner, cudaStream_t s) {
    unsigned nb = elem_grid((long long)L * g.d * g.M);
    if (g.d == 2) k_outer_update<2><<<nb, 256, 0, s>>>(g, L, x64, x32, outer, inner);
    else          k_outer_update<3><<<nb, 256, 0, s>>>(g, L, x64, x32, outer, inner);
    return cudaGetLastError();
}

cudaError_t launch_energy(const GridDev& g, int L, const CoeffsDev& co64, const double* x,
                          unsigned loadmask, double* partial, unsigned* counter, double* out,
                          cudaStream_t s) {
    unsigned nb = elem_grid(g.M);
    if (g.d == 2) k_energy<2><<<nb, 256, 0, s>>>(g, L, co64, x, loadmask, partial, counter, out);
    else          k_energy<3><<<nb, 256, 0, s>>>(g, L, co64, x, loadmask, partial, counter, out);
    return cudaGetLastError();
}

cudaError_t launch_invert_field(int d, long long M, const double* in, double* out64, float* out32,
                                cudaStream_t s) {
    const unsigned nb = elem_grid(M);
    if (d == 2) k_invert_field<2><<<nb, 256, 0, s>>>(M, in, out64, out32);
    else        k_invert_field<3><<<nb, 256, 0, s>>>(M, in, out64, out32);
    return cudaGetLastError();
}

cudaError_t launch_coeff_bounds(const GridDev& g, const CoeffsDev& co64, double* bounds, cudaStream_t s) {
    unsigned long long* b = reinterpret_cast<unsigned long long*>(bounds);
    cudaError_t e = cudaMemsetAsync(b, 0xff, sizeof(unsigned long long), s);   // min: above every value
    if (e == cudaSuccess) e = cudaMemsetAsync(b + 1, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    unsigned nb = elem_grid(g.M);
    if (g.d == 2) k_coeff_bounds<2><<<nb, 256, 0, s>>>(g, co64, b);
    else          k_coeff_bounds<3><<<nb, 256, 0, s>>>(g, co64, b);
    return cudaGetLastError();
}

cudaError_t launch_gather_scalars(const Scalars* const* src, Scalars* dst, int P, cudaStream_t s) {
    const int n = P * MAXL;
    k_gather_scalars<<<(n + 127) / 128, 128, 0, s>>>(src, dst, P);
    return cudaGetLastError();
}

cudaError_t launch_convert(const void* src, int sp, void* dst, int dp, long long n, cudaStream_t s) {
    unsigned nb = elem_grid(n);
    if (sp == 0 && dp == 1) k_convert<double, float><<<nb, 256, 0, s>>>((const double*)src, (float*)dst, n);
    else if (sp == 1 && dp == 0) k_convert<float, double><<<nb, 256, 0, s>>>((const float*)src, (double*)dst, n);
    else if (sp == 0 && dp == 0) k_convert<double, double><<<nb, 256, 0, s>>>((const double*)src, (double*)dst, n);
    else k_convert<float, float><<<nb, 256, 0, s>>>((const float*)src, (float*)dst, n);
    return cudaGetLastError();
}

cudaError_t launch_convert_spectrum(const void* src, int sp, double* dst, long long ncomplex,
                                    cudaStream_t s) {
    return launch_convert(src, sp, dst, 0, 2 * ncomplex, s);
}

}  // namespace hgk
