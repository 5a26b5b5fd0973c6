// kgs_layout.cu -- conversion between the public layout (four float64 arrays
// P, Q, U, V of N^d points) and the device state (vec2 arrays (P,Q) and (U,V)
// in the state precision; a handle's in the colour-split layout of
// kgs_internal.h, a batch's in natural order), and between the natural and
// colour-split vec2 layouts.  Float32 state rounds to nearest on the way in
// and widens exactly on the way out.
#include "kgs_internal.h"

namespace kgs {

// dim > 0: the vec2 side is in the colour-split layout of an N^dim grid.
template <typename T>
__global__ void pack_kernel(vec2_t<T>* __restrict__ dst, int comp, const double* __restrict__ src,
                            int64_t M, int dim, int64_t N, bool planar)
{
    T* d = reinterpret_cast<T*>(dst);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = dim ? split_pos(i, dim, N, M >> 1) : i;
        d[planar ? comp * M + j : 2 * j + comp] = (T)src[i];
    }
}

template <typename T>
__global__ void unpack_kernel(double* __restrict__ dst, const vec2_t<T>* __restrict__ src, int comp,
                              int64_t M, int dim, int64_t N, bool planar)
{
    const T* s = reinterpret_cast<const T*>(src);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = dim ? split_pos(i, dim, N, M >> 1) : i;
        dst[i] = (double)s[planar ? comp * M + j : 2 * j + comp];
    }
}

template <typename T>
__global__ void split_convert_kernel(bool to_split, const vec2_t<T>* __restrict__ pq_in,
                                     const vec2_t<T>* __restrict__ uv_in, vec2_t<T>* __restrict__ pq_out,
                                     vec2_t<T>* __restrict__ uv_out, int64_t M, int dim, int64_t N)
{
    // the split side's (U,V) buffer is planar: U at j, V at M + j
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = split_pos(i, dim, N, M >> 1);
        if (to_split) {
            pq_out[j] = pq_in[i];
            T* o = reinterpret_cast<T*>(uv_out);
            o[j] = uv_in[i].x;
            o[M + j] = uv_in[i].y;
        } else {
            pq_out[i] = pq_in[j];
            const T* u = reinterpret_cast<const T*>(uv_in);
            vec2_t<T> b;
            b.x = u[j];
            b.y = u[M + j];
            uv_out[i] = b;
        }
    }
}

static unsigned grid_for(int64_t M)
{
    int64_t b = (M + 255) / 256;
    const int64_t cap = 148 * 32;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename T>
int launch_pack(int64_t M, vec2_t<T>* dst, int comp, const double* src, cudaStream_t stream, int dim,
                int64_t N, bool planar)
{
    pack_kernel<T><<<grid_for(M), 256, 0, stream>>>(dst, comp, src, M, dim, N, planar);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template <typename T>
int launch_unpack(int64_t M, double* dst, const vec2_t<T>* src, int comp, cudaStream_t stream, int dim,
                  int64_t N, bool planar)
{
    unpack_kernel<T><<<grid_for(M), 256, 0, stream>>>(dst, src, comp, M, dim, N, planar);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template <typename T>
int launch_split_convert(const Grid& g, bool to_split, const vec2_t<T>* pq_in, const vec2_t<T>* uv_in,
                         vec2_t<T>* pq_out, vec2_t<T>* uv_out, cudaStream_t stream)
{
    split_convert_kernel<T><<<grid_for(g.M), 256, 0, stream>>>(to_split, pq_in, uv_in, pq_out, uv_out,
                                                              g.M, g.dim, g.N);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template int launch_pack<double>(int64_t, double2*, int, const double*, cudaStream_t, int, int64_t, bool);
template int launch_pack<float>(int64_t, float2*, int, const double*, cudaStream_t, int, int64_t, bool);
template int launch_unpack<double>(int64_t, double*, const double2*, int, cudaStream_t, int, int64_t, bool);
template int launch_unpack<float>(int64_t, double*, const float2*, int, cudaStream_t, int, int64_t, bool);
template int launch_split_convert<double>(const Grid&, bool, const double2*, const double2*, double2*,
                                          double2*, cudaStream_t);
template int launch_split_convert<float>(const Grid&, bool, const float2*, const float2*, float2*, float2*,
                                         cudaStream_t);

}  // namespace kgs
