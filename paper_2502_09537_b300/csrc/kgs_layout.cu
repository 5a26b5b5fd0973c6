// kgs_layout.cu -- conversion between the public layout (four float64 arrays
// P, Q, U, V of N^d points) and the device state (vec2 arrays (P,Q) and (U,V)
// in the state precision).  Float32 state rounds to nearest on the way in and
// widens exactly on the way out.
#include "kgs_internal.h"

namespace kgs {

template <typename T>
__global__ void pack_kernel(vec2_t<T>* __restrict__ dst, int comp, const double* __restrict__ src,
                            int64_t M)
{
    T* d = reinterpret_cast<T*>(dst);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x)
        d[2 * i + comp] = (T)src[i];
}

template <typename T>
__global__ void unpack_kernel(double* __restrict__ dst, const vec2_t<T>* __restrict__ src, int comp,
                              int64_t M)
{
    const T* s = reinterpret_cast<const T*>(src);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (double)s[2 * i + comp];
}

static unsigned grid_for(int64_t M)
{
    int64_t b = (M + 255) / 256;
    const int64_t cap = 148 * 32;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename T>
int launch_pack(int64_t M, vec2_t<T>* dst, int comp, const double* src, cudaStream_t stream)
{
    pack_kernel<T><<<grid_for(M), 256, 0, stream>>>(dst, comp, src, M);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template <typename T>
int launch_unpack(int64_t M, double* dst, const vec2_t<T>* src, int comp, cudaStream_t stream)
{
    unpack_kernel<T><<<grid_for(M), 256, 0, stream>>>(dst, src, comp, M);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template int launch_pack<double>(int64_t, double2*, int, const double*, cudaStream_t);
template int launch_pack<float>(int64_t, float2*, int, const double*, cudaStream_t);
template int launch_unpack<double>(int64_t, double*, const double2*, int, cudaStream_t);
template int launch_unpack<float>(int64_t, double*, const float2*, int, cudaStream_t);

}  // namespace kgs
