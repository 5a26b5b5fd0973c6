// kgs_order.cu -- DP-AVF2 over an arbitrary update order (declared in
// include/kgs.h: kgs_order_schedule, kgs_set_order, kgs_order_levels).
//
// Sec. 3 of arXiv 2502.09537: every order of the grid points defines a DP-AVF
// scheme (which neighbours enter a point's update at the new level -- the
// S/W/E/N superscripts of Eq. LapP, fixed by Eqs. order1/order2 for the two
// lexicographic orders); the base half visits the points in the order, the
// adjoint half in the reverse order (Algorithm 1), in place.  Algorithm 2
// (block splitting) and Algorithm 3 (the checkerboard) are particular orders.
//
// On the GPU an order runs as a level schedule.  A point's level is one more
// than the largest level of its neighbours that come before it in the order
// (0 if none does).  Points of one level are never neighbours (of two
// neighbours the later one has the higher level), so a level's updates are
// independent; processing the levels in increasing order gives every point
// exactly the neighbour values the serial order gives it (earlier neighbours
// updated, later ones not yet), hence bitwise the serial result for the same
// pointwise arithmetic.  The adjoint half runs the levels in decreasing
// order.  The checkerboard has 2 levels, the lexicographic order 1 + d(N-1)
// (its anti-diagonal wavefronts).
#include <algorithm>
#include <new>
#include <vector>

#include "kgs_internal.h"

namespace kgs {

namespace {

// Linear indices of the 2d periodic neighbours of point i (axis 0 first; per
// axis the lower neighbour, then the upper), the order of the colour passes.
template <int D>
__host__ __device__ __forceinline__ void neighbours_of(int64_t i, int64_t N, int64_t nb[2 * D])
{
    int64_t st = 1;
    for (int a = 1; a < D; ++a) st *= N;
    int n = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const int64_t coord = (i / st) % N;
        nb[n++] = coord == 0 ? i + (N - 1) * st : i - st;
        nb[n++] = coord == N - 1 ? i - (N - 1) * st : i + st;
        st /= N;
    }
}

template <typename T, int D, int MODE>
__global__ void __launch_bounds__(256) level_kernel(vec2_t<T>* pq, vec2_t<T>* uv, const int64_t* list,
                                                    int64_t count, int64_t N, Coef<T> c)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int64_t i = list[k];
    int64_t nb[2 * D];
    neighbours_of<D>(i, N, nb);
    // the handle's colour-split layout: the neighbours are in the other half
    const int64_t half = (D == 1 ? N : (D == 2 ? N * N : N * N * N)) >> 1;
    const int par = point_parity(i, D, N);
    const int64_t own = (par ? half : 0) + (i >> 1), oth = par ? 0 : half;
    T* u = reinterpret_cast<T*>(uv);  // planar: U at a position, V at 2 half + position
    T p[2 * D], q[2 * D], w[2 * D];
#pragma unroll
    for (int m = 0; m < 2 * D; ++m) {
        const int64_t j = oth + (nb[m] >> 1);
        const vec2_t<T> b = pq[j];
        p[m] = b.x;
        q[m] = b.y;
        w[m] = u[j];
    }
    vec2_t<T> a = pq[own];
    T U = u[own], V = u[2 * half + own];
    update_point<T, D, MODE>(c, nsum_scaled(p, c.beta), nsum_scaled(q, c.beta), nsum_scaled(w, c.Bp), a.x,
                             a.y, U, V);
    pq[own] = a;
    u[own] = U;
    u[2 * half + own] = V;
}

template <int D>
int schedule_d(int64_t N, int64_t M, const int64_t* order, int32_t* level, int64_t* nlevels)
{
    std::vector<int64_t> pos;
    try {
        pos.assign((size_t)M, -1);
    } catch (const std::bad_alloc&) {
        return -3;
    }
    for (int64_t t = 0; t < M; ++t) {
        const int64_t p = order[t];
        if (p < 0 || p >= M || pos[(size_t)p] >= 0) return -1;
        pos[(size_t)p] = t;
    }
    int64_t nl = 0;
    for (int64_t t = 0; t < M; ++t) {
        const int64_t p = order[t];
        int64_t nb[2 * D];
        neighbours_of<D>(p, N, nb);
        int32_t lv = 0;
        for (int m = 0; m < 2 * D; ++m)
            if (pos[(size_t)nb[m]] < t) lv = std::max(lv, level[nb[m]] + 1);
        level[p] = lv;
        nl = std::max<int64_t>(nl, (int64_t)lv + 1);
    }
    *nlevels = nl;
    return 0;
}

}  // namespace

int order_schedule(int dim, int64_t N, const int64_t* order, int32_t* level, int64_t* nlevels)
{
    int64_t M = 1;
    for (int a = 0; a < dim; ++a) M *= N;
    if (dim == 1) return schedule_d<1>(N, M, order, level, nlevels);
    if (dim == 2) return schedule_d<2>(N, M, order, level, nlevels);
    return schedule_d<3>(N, M, order, level, nlevels);
}

int order_lists(int dim, int64_t N, const int64_t* order, std::vector<int64_t>& list,
                std::vector<int64_t>& offsets)
{
    int64_t M = 1;
    for (int a = 0; a < dim; ++a) M *= N;
    std::vector<int32_t> level;
    try {
        level.assign((size_t)M, 0);
        list.assign((size_t)M, 0);
    } catch (const std::bad_alloc&) {
        return -3;
    }
    int64_t nl = 0;
    int st = order_schedule(dim, N, order, level.data(), &nl);
    if (st) return st;
    // counting sort by level, stable in order position
    offsets.assign((size_t)nl + 1, 0);
    for (int64_t p = 0; p < M; ++p) ++offsets[(size_t)level[(size_t)p] + 1];
    for (int64_t l = 0; l < nl; ++l) offsets[(size_t)l + 1] += offsets[(size_t)l];
    std::vector<int64_t> fill(offsets.begin(), offsets.end() - 1);
    for (int64_t t = 0; t < M; ++t) {
        const int64_t p = order[t];
        list[(size_t)fill[(size_t)level[(size_t)p]]++] = p;
    }
    return 0;
}

template <typename T>
int launch_level(int dim, int mode, vec2_t<T>* pq, vec2_t<T>* uv, const int64_t* list, int64_t count,
                 int64_t N, const Coef<T>& c, cudaStream_t s)
{
    if (count <= 0) return 0;
    const unsigned blocks = (unsigned)((count + 255) / 256);
    const bool base = mode == RED_BASE;
#define KGS_LEVEL(DD)                                                                          \
    if (base) level_kernel<T, DD, RED_BASE><<<blocks, 256, 0, s>>>(pq, uv, list, count, N, c); \
    else level_kernel<T, DD, RED_ADJ><<<blocks, 256, 0, s>>>(pq, uv, list, count, N, c);
    if (dim == 1) { KGS_LEVEL(1) }
    else if (dim == 2) { KGS_LEVEL(2) }
    else { KGS_LEVEL(3) }
#undef KGS_LEVEL
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

template int launch_level<double>(int, int, vec2_t<double>*, vec2_t<double>*, const int64_t*, int64_t,
                                  int64_t, const Coef<double>&, cudaStream_t);
template int launch_level<float>(int, int, vec2_t<float>*, vec2_t<float>*, const int64_t*, int64_t,
                                 int64_t, const Coef<float>&, cudaStream_t);

}  // namespace kgs
