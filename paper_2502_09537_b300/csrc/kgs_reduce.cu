// kgs_reduce.cu -- discrete invariants of a KGS state in float64.
//
//   E_h  = h^d sum [ 1/2 (kappa1 |grad_h psi|^2 + kappa2 |grad_h u|^2 + v^2 + mu^2 u^2)
//                    - gamma |psi|^2 u ]            (Sec. 2 E_h, Eq. ene-origin)
//   S_E  = h^d sum of the absolute values of those five terms
//   mass = h^d sum |psi|^2                           (the discrete norm of Sec. 2)
// grad_h is the forward difference (summation by parts turns -X^T D X into
// sum |grad_h X|^2).  Float32 state is widened to float64 before differencing.
//
// Two kernels, deterministic for a given grid size: a grid-stride pass where
// each thread accumulates with Neumaier compensation and each block reduces
// with warp shuffles into per-block partials; then one block combines the
// partials with compensated (two-sum) arithmetic and scales by h^d.
#include "kgs_internal.h"

namespace kgs {

struct Comp {
    double s, c;
};

__device__ __forceinline__ void neumaier_add(Comp& a, double x)
{
    double t = a.s + x;
    if (fabs(a.s) >= fabs(x)) a.c += (a.s - t) + x;
    else a.c += (x - t) + a.s;
    a.s = t;
}

__device__ __forceinline__ Comp comp_merge(Comp a, Comp b)
{
    Comp r{a.s, a.c + b.c};
    neumaier_add(r, b.s);
    return r;
}

// SPLIT: the state is in the colour-split layout (a point and its neighbours
// are of opposite colours: the neighbours sit in the other half).
template <typename T, int D, bool SPLIT>
__global__ void __launch_bounds__(256) invariants_kernel(const vec2_t<T>* __restrict__ pq,
                                                         const vec2_t<T>* __restrict__ uv,
                                                         int64_t N, int64_t M, InvParams p,
                                                         double* __restrict__ partials)
{
    Comp e{0, 0}, sc{0, 0}, ms{0, 0};
    const T* u = reinterpret_cast<const T*>(uv);
    const int64_t half = M >> 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        // forward neighbours along each axis (periodic), and the point's colour
        int64_t up[D];
        int par = 0;
        {
            int64_t rem = i, st = 1;
            for (int ax = D - 1; ax >= 0; --ax) {
                const int64_t coord = rem % N;
                rem /= N;
                par += (int)(coord & 1);
                up[ax] = (coord == N - 1) ? i - (N - 1) * st : i + st;
                st *= N;
            }
        }
        const int64_t own = SPLIT ? ((par & 1) ? half : 0) + (i >> 1) : i;
        const int64_t oth = SPLIT ? ((par & 1) ? 0 : half) : 0;
        const vec2_t<T> a = pq[own];
        // (U,V): planar in the colour-split layout, vec2 otherwise
        const double P = (double)a.x, Q = (double)a.y;
        const double U = (double)(SPLIT ? u[own] : u[2 * own]);
        const double V = (double)(SPLIT ? u[M + own] : u[2 * own + 1]);
        double gp = 0.0, gu = 0.0;
#pragma unroll
        for (int ax = 0; ax < D; ++ax) {
            const int64_t k = SPLIT ? oth + (up[ax] >> 1) : up[ax];
            const vec2_t<T> c = pq[k];
            const double dp = (double)c.x - P, dq = (double)c.y - Q;
            const double du = (double)u[SPLIT ? k : 2 * k] - U;
            gp += dp * dp + dq * dq;
            gu += du * du;
        }
        const double t1 = 0.5 * p.kappa1 * gp * p.inv_h2;
        const double t2 = 0.5 * p.kappa2 * gu * p.inv_h2;
        const double t3 = 0.5 * V * V;
        const double t4 = 0.5 * p.mu * p.mu * U * U;
        const double rho = P * P + Q * Q;
        const double t5 = p.gamma * rho * U;
        neumaier_add(e, t1 + t2 + t3 + t4 - t5);
        neumaier_add(sc, fabs(t1) + fabs(t2) + t3 + t4 + fabs(t5));
        neumaier_add(ms, rho);
    }
    double v[3] = {e.s + e.c, sc.s + sc.c, ms.s + ms.c};
    __shared__ double red[3][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double x = v[k];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
        if (lane == 0) red[k][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < 3; ++k) {
            double x = 0.0;
            for (int w = 0; w < nw; ++w) x += red[k][w];
            partials[3 * (int64_t)blockIdx.x + k] = x;
        }
    }
}

__global__ void __launch_bounds__(256) invariants_finalize(const double* __restrict__ partials,
                                                           int nblocks, double hd,
                                                           double* __restrict__ out3)
{
    __shared__ Comp red[3][256];
    for (int k = 0; k < 3; ++k) {
        Comp a{0, 0};
        for (int j = threadIdx.x; j < nblocks; j += blockDim.x) neumaier_add(a, partials[3 * j + k]);
        red[k][threadIdx.x] = a;
    }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 3; ++k)
                red[k][threadIdx.x] = comp_merge(red[k][threadIdx.x], red[k][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) out3[k] = (red[k][0].s + red[k][0].c) * hd;
}

int invariants_blocks(int64_t M)
{
    int64_t b = (M + 255) / 256;
    const int64_t cap = 148 * 8;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename T>
int launch_invariants(const Grid& g, const vec2_t<T>* pq, const vec2_t<T>* uv, const InvParams& p,
                      double* partials, int nblocks, double* out3, cudaStream_t stream)
{
#define KGS_INV(DD)                                                                              \
    if (g.split) invariants_kernel<T, DD, true><<<nblocks, 256, 0, stream>>>(pq, uv, g.N, g.M, p, partials); \
    else invariants_kernel<T, DD, false><<<nblocks, 256, 0, stream>>>(pq, uv, g.N, g.M, p, partials);
    if (g.dim == 1) { KGS_INV(1) }
    else if (g.dim == 2) { KGS_INV(2) }
    else { KGS_INV(3) }
#undef KGS_INV
    invariants_finalize<<<1, 256, 0, stream>>>(partials, nblocks, p.hd, out3);
    return cudaPeekAtLastError() == cudaSuccess ? 2 : -1;
}

template int launch_invariants<double>(const Grid&, const double2*, const double2*, const InvParams&,
                                       double*, int, double*, cudaStream_t);
template int launch_invariants<float>(const Grid&, const float2*, const float2*, const InvParams&,
                                      double*, int, double*, cudaStream_t);

}  // namespace kgs
