// kgs_noalloc.cu -- an allocation-free variant of the invariants reduction
// (declared in include/kgs.h as kgs_invariants_noalloc).
//
// Who needs it: callers that must not allocate device memory at the point they
// want the energy -- code that owns all GPU memory through its own arena or
// budget and forbids other allocations, host threads with latency limits that
// cannot afford cudaMalloc's implicit synchronisation, or a caller that is not
// allowed to create a kgs handle (whose creation allocates).  They pass their
// own state and output buffers; the only scratch this path uses is the
// file-scope array below, which every GPU that loads libkgs holds until the
// process exits.
//
// The scratch holds one partial (E_h, S_E, mass) triple per CTA of the first
// kernel.  Each CTA covers kPointsPerCta consecutive points, so a grid of M
// points needs ceil(M / kPointsPerCta) triples and the array's kMaxCtas
// triples bound M at kMaxCtas * kPointsPerCta points; larger grids are
// rejected with KGS_ERR_RANGE.  Every call writes each triple it later reads,
// so nothing has to start at zero, but all calls share the one array: calls
// that can overlap on the GPU (different streams without ordering between
// them) race and may return wrong values.
#include <cuda.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/kgs.h"
#include "kgs_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPointsPerThread = 16;
constexpr int64_t kPointsPerCta = (int64_t)kThreads * kPointsPerThread;  // 4096
constexpr int kMaxCtas = 8192;                                            // 192 KB of scratch
static_assert((int64_t)kMaxCtas * kPointsPerCta == KGS_NOALLOC_MAX_POINTS,
              "kgs.h states the limit");

static __device__ __align__(256) double g_noalloc_partials[3 * kMaxCtas];

// Device address of g_noalloc_partials, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_partials_addr[kMaxDevices] = {};
// the context each address was looked up in: a device reset replaces the
// device's context (and the module's copy of the array), so the address is
// looked up again when the current context differs
void* g_partials_ctx[kMaxDevices] = {};

struct Acc {
    double s, c;
};

__device__ __forceinline__ void acc_add(Acc& a, double x)
{
    double t = a.s + x;
    if (fabs(a.s) >= fabs(x)) a.c += (a.s - t) + x;
    else a.c += (x - t) + a.s;
    a.s = t;
}

// First level: CTA b sums the energy density, its absolute-term scale and
// |psi|^2 over points [b * kPointsPerCta, (b+1) * kPointsPerCta) of the
// four float64 fields and writes one triple to partials[3b..3b+2].
template <int D>
__global__ void __launch_bounds__(kThreads) noalloc_partials_kernel(
    const double* __restrict__ P, const double* __restrict__ Q, const double* __restrict__ U,
    const double* __restrict__ V, int64_t N, int64_t M, kgs::InvParams p, double* partials)
{
    Acc e{0, 0}, sc{0, 0}, ms{0, 0};
    const int64_t base = (int64_t)blockIdx.x * kPointsPerCta;
    for (int k = 0; k < kPointsPerThread; ++k) {
        const int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
        if (i >= M) break;
        int64_t up[D];
        {
            int64_t rem = i, st = 1;
            for (int ax = D - 1; ax >= 0; --ax) {
                const int64_t coord = rem % N;
                rem /= N;
                up[ax] = (coord == N - 1) ? i - (N - 1) * st : i + st;
                st *= N;
            }
        }
        const double p0 = P[i], q0 = Q[i], u0 = U[i], v0 = V[i];
        double gp = 0.0, gu = 0.0;
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
            const double dp = P[up[ax]] - p0, dq = Q[up[ax]] - q0, du = U[up[ax]] - u0;
            gp += dp * dp + dq * dq;
            gu += du * du;
        }
        // kappa1/2 |grad psi|^2 + kappa2/2 |grad u|^2 + (v^2 + mu^2 u^2)/2 - gamma |psi|^2 u
        const double rho = fma(p0, p0, q0 * q0);
        const double vu = fma(v0, v0, (p.mu2 * u0) * u0);
        const double t5 = (p.gamma * rho) * u0;
        acc_add(e, fma(p.k1, gp, fma(p.k2, gu, fma(0.5, vu, -t5))));
        acc_add(sc, fma(p.abs_k1, gp, fma(p.abs_k2, gu, fma(0.5, vu, fabs(t5)))));
        acc_add(ms, rho);
    }
    double v[3] = {e.s + e.c, sc.s + sc.c, ms.s + ms.c};
    __shared__ double red[3][kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double x = v[k];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) red[k][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) {
            double x = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) x += red[k][w];
            partials[3 * (int64_t)blockIdx.x + k] = x;
        }
}

// Second level: one CTA combines the nctas triples with compensated sums.
__global__ void __launch_bounds__(kThreads) noalloc_finalize_kernel(const double* partials,
                                                                   int nctas, double hd,
                                                                   double* __restrict__ out3)
{
    __shared__ Acc red[3][kThreads];
    for (int k = 0; k < 3; ++k) {
        Acc a{0, 0};
        for (int j = threadIdx.x; j < nctas; j += kThreads) acc_add(a, partials[3 * j + k]);
        red[k][threadIdx.x] = a;
    }
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 3; ++k) {
                Acc a = red[k][threadIdx.x];
                const Acc b = red[k][threadIdx.x + w];
                a.c += b.c;
                acc_add(a, b.s);
                red[k][threadIdx.x] = a;
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) out3[k] = (red[k][0].s + red[k][0].c) * hd;
}

// The calling thread's current driver context (nullptr if none or unknown),
// through the driver entry point the runtime exposes: no link to libcuda.
void* current_context()
{
    using CtxGetCurrent = CUresult (*)(CUcontext*);
    static const CtxGetCurrent fn = []() -> CtxGetCurrent {  // looked up once, thread-safely
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<CtxGetCurrent>(f);
        return nullptr;
    }();
    CUcontext ctx = nullptr;
    if (!fn || fn(&ctx) != CUDA_SUCCESS) return nullptr;
    return ctx;
}

// Resolve the scratch array's device address for the current device: once per
// device and context (again after a device reset, which replaces the context).
int scratch_address(double** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return kgs::report_error(KGS_ERR_CUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices)
        return kgs::report_error(KGS_ERR_RANGE, "device index beyond the supported 64");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    void* ctx = current_context();
    if (!g_partials_addr[dev] || !ctx || ctx != g_partials_ctx[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
        if (e != cudaSuccess || !ptr)
            return kgs::report_error(KGS_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
        g_partials_addr[dev] = static_cast<double*>(ptr);
        g_partials_ctx[dev] = current_context();  // now current, if it was not before the lookup
    }
    *out = g_partials_addr[dev];
    return KGS_OK;
}

}  // namespace

extern "C" int kgs_invariants_noalloc(int dim, int64_t N, double L, double kappa1, double kappa2,
                                      double mu, double gamma, const double* P, const double* Q,
                                      const double* U, const double* V, double* out3, void* stream)
{
    if (dim < 1 || dim > 3 || N < 2 || !(L > 0) || !std::isfinite(L) || !std::isfinite(kappa1) ||
        !std::isfinite(kappa2) || !std::isfinite(mu) || !std::isfinite(gamma) || !P || !Q || !U ||
        !V || !out3)
        return kgs::report_error(KGS_ERR_ARG, "kgs_invariants_noalloc: invalid argument");
    int64_t M = 1;
    for (int a = 0; a < dim; ++a) {
        if (M > KGS_NOALLOC_MAX_POINTS / N) {
            char msg[160];
            snprintf(msg, sizeof msg,
                     "kgs_invariants_noalloc: %lld^%d points exceed the limit of %lld points",
                     (long long)N, dim, (long long)KGS_NOALLOC_MAX_POINTS);
            return kgs::report_error(KGS_ERR_RANGE, msg);
        }
        M *= N;
    }
    double* partials = nullptr;
    int st = scratch_address(&partials);
    if (st != KGS_OK) return st;
    const kgs::InvParams p = kgs::make_inv_params(dim, L / (double)N, kappa1, kappa2, mu, gamma);
    const int nctas = (int)((M + kPointsPerCta - 1) / kPointsPerCta);
    cudaStream_t s = (cudaStream_t)stream;
    if (dim == 1)
        noalloc_partials_kernel<1><<<nctas, kThreads, 0, s>>>(P, Q, U, V, N, M, p, partials);
    else if (dim == 2)
        noalloc_partials_kernel<2><<<nctas, kThreads, 0, s>>>(P, Q, U, V, N, M, p, partials);
    else
        noalloc_partials_kernel<3><<<nctas, kThreads, 0, s>>>(P, Q, U, V, N, M, p, partials);
    noalloc_finalize_kernel<<<1, kThreads, 0, s>>>(partials, nctas, p.hd, out3);
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return kgs::report_error(KGS_ERR_CUDA, cudaGetErrorString(e));
    return KGS_OK;
}
