// Coefficients of the Galerkin scheme with exact integration (Sec. 4.2, Ga)
// for A constant on the pixels of a grid P.
//
// The trial space is the trigonometric polynomials of Z_N.  The product of two
// of them has frequencies below 2N - 1, so on a grid M with M_a >= 2 N_a - 1
// the grid mean of A_M u . v, with A_M the Fourier series of A truncated to
// |l_a| <= N_a - 1, is the exact integral of A u . v.  The CG of the GaNi
// kernels on the grid M, with the projection limited to the trial band
// (StrArgs.band), then solves Ga, and the grid energy gives its A_H.
//
// A pixel of the grid P contributes exp(-i pi xi(l) . x) integrated over its
// box, i.e. its centre value times prod_a sinc(l_a / P_a).  Per axis, the
// truncated series of a unit pixel k evaluated at the point j of the grid M is
//   W[j][k] = (1 / P) (1 + 2 sum_{l=1}^{N-1} sinc(l / P) cos(2 pi l (j / M - k / P))),
// real since the sum is symmetric in l; A_M is the pixel field multiplied by W
// along every axis.
#include "hg.h"
#include "hg_internal.h"
#include "hg_runtime.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

using namespace hgk;
using namespace hgrt;

namespace {

constexpr double kPi = 3.14159265358979323846;

__global__ void k_ga_axis_weights(int M, int P, int N, double* W) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)M * P) return;
    const int j = (int)(idx / P), k = (int)(idx % P);
    const long long MP = (long long)M * P;
    const long long base = (long long)j * P - (long long)k * M;   // (j/M - k/P) MP
    double acc = 1.0;
    for (int l = 1; l < N; ++l) {
        long long r = ((long long)l * base) % MP;                  // reduce the angle exactly
        if (r < 0) r += MP;
        const double c = cospi(2.0 * (double)r / (double)MP);
        const double t = (double)l / (double)P;
        acc += 2.0 * (sinpi(t) / (kPi * t)) * c;
    }
    W[idx] = acc / (double)P;
}

// out[k] = table[phase[k]][i][j]: one component of the pixel field.
__global__ void k_ga_pixel_component(long long n, const uint8_t* __restrict__ phase,
                                     const double* __restrict__ table, int d, int i, int j,
                                     double* __restrict__ out) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = table[(int)phase[k] * d * d + i * d + j];
}

// in viewed as (pre, K, post), W as (Mo, K): out (pre, Mo, post) = W along K.
__global__ void k_ga_mode_product(long long pre, int K, long long post, int Mo, const double* __restrict__ W,
                                  const double* __restrict__ in, double* __restrict__ out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = pre * Mo * post;
    if (idx >= total) return;
    const long long a = idx / (Mo * post);
    const long long rem = idx - a * Mo * post;
    const int jj = (int)(rem / post);
    const long long c = rem - (long long)jj * post;
    const double* w = W + (long long)jj * K;
    const double* x = in + a * K * post + c;
    double acc = 0.0;
    for (int k = 0; k < K; ++k) acc += w[k] * x[k * post];
    out[idx] = acc;
}

unsigned blocks_for(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

namespace hgrt {

// A_M (or, for `table` holding inverses, (A^-1)_M) as a packed symmetric field
// on the grid of g: FP64 into out64, FP32 into out32 (d(d+1)/2 x |M| each).
// phase (device, |P| bytes) and table (device, n_phases x d x d) describe the
// pixels; Ntr is the trial band.
int ga_build_field(hg_grid* g, const int* Ntr, const int* P, const uint8_t* phase, const double* table,
                   double* out64, float* out32, cudaStream_t s) {
    hg_ctx* c = g->ctx;
    const int d = g->gd.d;
    const int npk = d * (d + 1) / 2;
    static const int pi2[3][2] = {{0, 0}, {1, 1}, {0, 1}};
    static const int pi3[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    long long Pt = 1, Mt = 1, maxsz = 1;
    for (int a = 0; a < d; ++a) { Pt *= P[a]; Mt *= g->gd.N[a]; }
    // the largest intermediate: axes 0..a on M, the rest on P
    for (int a = 0; a <= d; ++a) {
        long long sz = 1;
        for (int b = 0; b < d; ++b) sz *= (b < a ? g->gd.N[b] : P[b]);
        maxsz = std::max(maxsz, sz);
    }
    double* W[3] = {nullptr, nullptr, nullptr};
    double* buf[2] = {nullptr, nullptr};
    int st = HG_OK;
    auto fail = [&](int code) {
        for (int a = 0; a < 3; ++a) dev_free(c, W[a]);
        for (int b = 0; b < 2; ++b) dev_free(c, buf[b]);
        return code;
    };
    for (int a = 0; a < d; ++a) {
        if ((st = dev_alloc(c, (void**)&W[a], sizeof(double) * (size_t)g->gd.N[a] * P[a]))) return fail(st);
        k_ga_axis_weights<<<blocks_for((long long)g->gd.N[a] * P[a]), 256, 0, s>>>(g->gd.N[a], P[a], Ntr[a], W[a]);
        c->launches++;
    }
    for (int b = 0; b < 2; ++b)
        if ((st = dev_alloc(c, (void**)&buf[b], sizeof(double) * (size_t)maxsz))) return fail(st);
    for (int q = 0; q < npk; ++q) {
        const int i = d == 2 ? pi2[q][0] : pi3[q][0];
        const int j = d == 2 ? pi2[q][1] : pi3[q][1];
        k_ga_pixel_component<<<blocks_for(Pt), 256, 0, s>>>(Pt, phase, table, d, i, j, buf[0]);
        c->launches++;
        // W along each axis in turn: (M_0..M_{a-1}, P_a, P_{a+1}..) -> (.., M_a, ..)
        int cur = 0;
        for (int a = 0; a < d; ++a) {
            long long pre = 1, post = 1;
            for (int b = 0; b < a; ++b) pre *= g->gd.N[b];
            for (int b = a + 1; b < d; ++b) post *= P[b];
            double* dst = (a == d - 1) ? out64 + (size_t)q * Mt : buf[cur ^ 1];
            k_ga_mode_product<<<blocks_for(pre * g->gd.N[a] * post), 256, 0, s>>>(pre, P[a], post, g->gd.N[a], W[a],
                                                                                 buf[cur], dst);
            c->launches++;
            cur ^= 1;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_convert(out64, 0, out32, 1, (long long)npk * Mt, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "ga_build_field");
        return fail(HG_ERR_CUDA);
    }
    c->launches++;
    return fail(HG_OK);
}

}  // namespace hgrt
