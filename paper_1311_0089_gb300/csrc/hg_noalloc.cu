// hg_apply_noalloc: the operator G_N A_N u without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need the
// operator: plug-ins of host applications whose device memory belongs to the
// host's own allocator, and real-time loops in which an allocation (with the
// synchronisation cudaMalloc and cudaFree imply) is not allowed.  For them
// this entry point keeps its scratch (FFT twiddles, the half spectrum, the
// reduction slots) in one file-scope device array of a fixed size,
// NOALLOC_SCRATCH_BYTES, that every GPU loading the library holds until the
// process exits.  The caller passes the coefficients, the input and the
// output as device pointers.
//
// The array is shared by every call: calls whose work overlaps on the GPU
// (for instance on two streams) race on it.  Each call clears what must start
// at zero before it uses it.  The first call on a device does the set-up
// (the device address of the array, kernel attributes, codelet constants);
// make that first call before any stream capture.
#include "hg.h"
#include "hg_internal.h"
#include "hg_runtime.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

using namespace hgk;
using namespace hgrt;

namespace {
constexpr size_t NOALLOC_SCRATCH_BYTES = 16u << 20;   // 16 MiB per device
}

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
void* g_scratch_dev[MAX_DEVICES];   // device address of g_noalloc_scratch per device
int g_max_smem[MAX_DEVICES];

// W_n^m = exp(-2 pi i m / n), m < n, written into the scratch array.
__global__ void k_noalloc_twiddles(double2* tw, int n) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < n) {
        double s, c;
        sincospi(-2.0 * (double)m / (double)n, &s, &c);
        tw[m] = make_double2(c, s);
    }
}

// Once per device, with that device current.
int noalloc_setup(int dev, unsigned char** base, int* max_smem) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (dev < 0 || dev >= MAX_DEVICES) return HG_ERR_ARG;
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_last_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
            return HG_ERR_CUDA;
        }
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const int ms = std::max(48 * 1024, optin - 4 * 1024);
        e = configure_kernels(ms);
        if (e != cudaSuccess) {
            set_last_cuda_error(e, "configure_kernels");
            return HG_ERR_CUDA;
        }
        g_max_smem[dev] = ms;
        g_scratch_dev[dev] = p;
    }
    *base = static_cast<unsigned char*>(g_scratch_dev[dev]);
    *max_smem = g_max_smem[dev];
    return HG_OK;
}

int check_length(int n) {
    if (n < 1 || n > 1024 || (n % 2) == 0) return HG_ERR_UNSUPPORTED_SIZE;
    int m = n;
    for (int r : {3, 5, 7})
        while (m % r == 0) m /= r;
    return m == 1 ? HG_OK : HG_ERR_UNSUPPORTED_SIZE;
}

}  // namespace

#define HG_CU(call)                                  \
    do {                                             \
        cudaError_t _e = (call);                     \
        if (_e != cudaSuccess) {                     \
            set_last_cuda_error(_e, #call);          \
            return HG_ERR_CUDA;                      \
        }                                            \
    } while (0)

extern "C" int hg_apply_noalloc(int d, const int* N, const uint8_t* phase, int n_phases,
                                const double* table, const double* u, double* out,
                                void* cuda_stream) {
    if ((d != 2 && d != 3) || !N || !phase || !table || !u || !out || n_phases < 1 || n_phases > 256)
        return HG_ERR_ARG;
    for (int a = 0; a < d; ++a) {
        const int st = check_length(N[a]);
        if (st) return st;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // grid description (Y = 1 on every axis, A0 = I)
    GridDev gd;
    memset(&gd, 0, sizeof(gd));
    gd.d = d;
    gd.M = 1;
    for (int a = 0; a < 3; ++a) {
        gd.N[a] = a < d ? N[a] : 1;
        gd.Y[a] = 1.0;
        gd.invY[a] = 1.0;
        gd.invYf[a] = 1.0f;
    }
    for (int a = 0; a < d; ++a) gd.M *= N[a];
    gd.Nl = N[d - 1];
    gd.H = (gd.Nl + 1) / 2;
    gd.rows = gd.M / gd.Nl;
    gd.Ms = gd.rows * gd.H;
    gd.invM = 1.0 / (double)gd.M;
    gd.invMf = (float)gd.invM;

    // scratch layout: scalars | counters | twiddles | reduction slots | half spectrum
    AxisPlanH plan[3];
    int tw_len[3], tw_at[3], ntab = 0, ntw = 0;   // one table per distinct length
    for (int a = 0; a < d; ++a) {
        if (!factor(N[a], plan[a])) return HG_ERR_UNSUPPORTED_SIZE;
        int q = 0;
        while (q < ntab && tw_len[q] != N[a]) ++q;
        if (q == ntab) { tw_len[q] = N[a]; tw_at[q] = ntw; ntw += N[a]; ++ntab; }
        plan[a].tw_off = tw_at[q];
    }
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return o;
    };
    // launch geometry needs the device's shared-memory limit: set up first
    int dev = 0;
    HG_CU(cudaGetDevice(&dev));
    unsigned char* base = nullptr;
    int max_smem = 0;
    {
        const int st = noalloc_setup(dev, &base, &max_smem);
        if (st) return st;
    }
    RowCfg rc;
    StrCfg sc[3];
    const int last = d - 1;
    if (!choose_row_cfg(0, gd.Nl, d, 1, min_radix(plan[last]), 16, max_smem, gd.rows, rc))
        return HG_ERR_UNSUPPORTED_SIZE;
    for (int a = 0; a < last; ++a) {
        const long long inner = (a == 0) ? gd.Ms / gd.N[0] : gd.H;
        const long long outer = (a == 0) ? 1 : gd.N[0];
        if (!choose_str_cfg(0, gd.N[a], d, min_radix(plan[a]), 16, max_smem, inner, outer, 1, sc[a]))
            return HG_ERR_UNSUPPORTED_SIZE;
    }
    const size_t o_sc = take(sizeof(Scalars) * MAXL);
    const size_t o_cnt = take(16 * sizeof(unsigned));
    const size_t o_tw = take((size_t)ntw * sizeof(double2));
    const size_t o_part = take((size_t)rc.nbx * MAXL * sizeof(double));
    const size_t o_S = take((size_t)d * gd.Ms * sizeof(double2));
    if (off > NOALLOC_SCRATCH_BYTES) return HG_ERR_TOO_LARGE;

    Scalars* scal = reinterpret_cast<Scalars*>(base + o_sc);
    unsigned* counters = reinterpret_cast<unsigned*>(base + o_cnt);
    double2* tw = reinterpret_cast<double2*>(base + o_tw);
    double* partial = reinterpret_cast<double*>(base + o_part);
    void* S = base + o_S;

    // what must start at zero: the CTA tickets and the scalars
    HG_CU(cudaMemsetAsync(counters, 0, 16 * sizeof(unsigned), s));
    HG_CU(cudaMemsetAsync(scal, 0, sizeof(Scalars) * MAXL, s));
    for (int q = 0; q < ntab; ++q) {
        k_noalloc_twiddles<<<(tw_len[q] + 127) / 128, 128, 0, s>>>(tw + tw_at[q], tw_len[q]);
        HG_CU(cudaGetLastError());
    }

    CoeffsDev co;
    co.mode = 0;
    co.n_phases = n_phases;
    co.phase = phase;
    co.table = table;
    co.field = nullptr;

    RowFwdArgs fa;
    memset(&fa, 0, sizeof(fa));
    fa.mode = FWD_APPLY; fa.L = 1; fa.co = co; fa.u = u; fa.S = S; fa.sc = scal;
    fa.partial = partial; fa.counter = counters + 0; fa.check_status = 0;
    HG_CU(launch_row_fwd(0, gd, plan[last], tw, rc, fa, s));

    StrArgs sa;
    memset(&sa, 0, sizeof(sa));
    sa.L = 1; sa.S = S; sa.sc = scal; sa.check_status = 0;
    if (d == 3) {
        sa.mode = STR_FWD; sa.axis = 1; sa.outer = gd.N[0]; sa.n = gd.N[1]; sa.inner = gd.H;
        HG_CU(launch_strided(0, gd, plan[1], tw, sc[1], sa, s));
    }
    sa.mode = STR_GAMMA; sa.axis = 0; sa.outer = 1; sa.n = gd.N[0]; sa.inner = gd.Ms / gd.N[0];
    HG_CU(launch_strided(0, gd, plan[0], tw, sc[0], sa, s));
    if (d == 3) {
        sa.mode = STR_INV; sa.axis = 1; sa.outer = gd.N[0]; sa.n = gd.N[1]; sa.inner = gd.H;
        HG_CU(launch_strided(0, gd, plan[1], tw, sc[1], sa, s));
    }

    RowInvArgs ia;
    memset(&ia, 0, sizeof(ia));
    ia.mode = INV_OUT; ia.L = 1; ia.S = S; ia.out = out; ia.sc = scal;
    ia.partial = partial; ia.counter = counters + 1; ia.check_status = 0;
    HG_CU(launch_row_inv(0, gd, plan[last], tw, rc, ia, s));
    return HG_OK;
}
