// kgs_probe.cu -- probes declared in include/kgs_probe.h: the FMA issue rate
// (the FP64 pipe rate that bounds the float64 colour passes, for the roofline
// denominator) and the colour passes' float64 neighbour sums and Psi weight
// exposed for accuracy tests.
#include "../../include/kgs_probe.h"

#include <cuda_runtime.h>

#include <cstring>

#include "kgs_internal.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(int64_t iters, T b, T c, T* sink)
{
    T a0 = (T)threadIdx.x * (T)1e-3, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
    T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
    for (int64_t k = 0; k < iters; ++k) {
        a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
        a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
    }
    T s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (s == (T)-12345.678) sink[blockIdx.x] = s;  // keeps the chains live
}

template <typename T>
int run(int64_t iters, int bps, cudaStream_t s, double* ms, double* rate)
{
    const int blocks = 148 * bps;
    T* sink = nullptr;
    if (cudaMalloc(&sink, blocks * sizeof(T)) != cudaSuccess) return -4;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_chains<T><<<blocks, 256, 0, s>>>(iters / 8 + 1, (T)0.999999, (T)1e-6, sink);  // warm-up
    cudaEventRecord(e0, s);
    fma_chains<T><<<blocks, 256, 0, s>>>(iters, (T)0.999999, (T)1e-6, sink);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return -4;
    *ms = t;
    *rate = (double)blocks * 256.0 * 8.0 * (double)iters / (t * 1e-3);
    return 0;
}

template <int K>
__global__ void nsum_kernel(const double* x, int64_t n, double beta, double* sum, double* scaled,
                            int32_t* exact)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v[K];
#pragma unroll
        for (int j = 0; j < K; ++j) v[j] = x[i * K + j];
        bool ok1, ok2;
        double s1 = kgs::nsum_try<K>(v, ok1);
        double s2 = kgs::nsum_scaled_try<K>(v, beta, ok2);
        if (!ok1) s1 = kgs::nsum_seq<K>(v);
        if (!ok2) s2 = kgs::nsum_seq_scaled<K>(v, beta);
        sum[i] = s1;
        scaled[i] = s2;
        int32_t f = (ok1 ? 1 : 0) | (ok2 ? 2 : 0);
        // the colour passes' entry points must agree with the two halves
        if (__double_as_longlong(kgs::nsum<K>(v)) != __double_as_longlong(s1)) f = -1;
        if (__double_as_longlong(kgs::nsum_scaled<K>(v, beta)) != __double_as_longlong(s2)) f = -1;
        exact[i] = f;
    }
}

__global__ void psi_weight_kernel(const double* r, int64_t n, double* w)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        w[i] = kgs::psi_weight(r[i]);
}

}  // namespace

extern "C" int kgs_probe_psi_weight(int64_t n, const double* r_host, double* w_host, void* stream)
{
    if (n < 0) return -1;
    if (n == 0) return 0;
    if (!r_host || !w_host) return -1;
    cudaStream_t s = (cudaStream_t)stream;
    double* dev = nullptr;
    if (cudaMalloc(&dev, 2 * (size_t)n * sizeof(double)) != cudaSuccess) return -3;
    cudaError_t e = cudaMemcpyAsync(dev, r_host, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const int blocks = (int)((n + 255) / 256 < 148 * 8 ? (n + 255) / 256 : 148 * 8);
        psi_weight_kernel<<<blocks, 256, 0, s>>>(dev, n, dev + n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w_host, dev + n, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dev);
    return e == cudaSuccess ? 0 : -4;
}

extern "C" int kgs_probe_nsum(int k, int64_t n, const double* x_host, double beta, double* sum_host,
                              double* scaled_host, int32_t* exact_host, void* stream)
{
    if ((k != 2 && k != 4 && k != 6) || n < 0) return -1;
    if (n == 0) return 0;
    if (!x_host || !sum_host || !scaled_host) return -1;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nb = (size_t)n * k * sizeof(double) + 2 * (size_t)n * sizeof(double) +
                      (size_t)n * sizeof(int32_t);
    char* dev = nullptr;
    if (cudaMalloc(&dev, nb) != cudaSuccess) return -3;
    double* dx = (double*)dev;
    double* dsum = dx + (size_t)n * k;
    double* dscaled = dsum + n;
    int32_t* dex = (int32_t*)(dscaled + n);
    cudaError_t e = cudaMemcpyAsync(dx, x_host, (size_t)n * k * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const int blocks = (int)((n + 255) / 256 < 148 * 8 ? (n + 255) / 256 : 148 * 8);
        if (k == 2) nsum_kernel<2><<<blocks, 256, 0, s>>>(dx, n, beta, dsum, dscaled, dex);
        if (k == 4) nsum_kernel<4><<<blocks, 256, 0, s>>>(dx, n, beta, dsum, dscaled, dex);
        if (k == 6) nsum_kernel<6><<<blocks, 256, 0, s>>>(dx, n, beta, dsum, dscaled, dex);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sum_host, dsum, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(scaled_host, dscaled, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && exact_host)
        e = cudaMemcpyAsync(exact_host, dex, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dev);
    return e == cudaSuccess ? 0 : -4;
}

extern "C" int kgs_probe_fma_rate(int precision, int64_t iters, int blocks_per_sm, void* stream,
                                  double* elapsed_ms, double* fma_per_s)
{
    if (iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 64 || !elapsed_ms || !fma_per_s) return -1;
    if (precision == 64) return run<double>(iters, blocks_per_sm, (cudaStream_t)stream, elapsed_ms, fma_per_s);
    if (precision == 32) return run<float>(iters, blocks_per_sm, (cudaStream_t)stream, elapsed_ms, fma_per_s);
    return -1;
}

extern "C" int kgs_debug_bounds(uint32_t* flags)
{
    if (!flags) return -1;
    if (cudaDeviceSynchronize() != cudaSuccess) return -4;
    const unsigned f[3] = {kgs::bounds_flags_sweep(), kgs::bounds_flags_stream(), kgs::bounds_flags_batch()};
    *flags = 0;
    for (unsigned v : f) {
        if (v == ~0u) return -4;
        *flags |= v;
    }
#ifdef KGS_DEBUG_BOUNDS
    return 1;
#else
    return 0;
#endif
}

extern "C" int kgs_stream2_side_list(int64_t N, uint16_t* out, int64_t cap)
{
    constexpr int64_t kEntries = 2 * 2 * 96 + 4;
    if (N < 4 || N % 2 || !out || cap < kEntries) return -1;
    alignas(16) unsigned char buf[kgs::kStream2SideBytes];
    if (kgs::stream2_prepare(N, buf)) return -2;
    memcpy(out, buf, kEntries * sizeof(uint16_t));
    return (int)kEntries;
}
