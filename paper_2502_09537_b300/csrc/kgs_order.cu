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
// (its anti-diagonal wavefronts).  Levels run as one launch each (a step
// captured in a CUDA graph), on the handle's colour-split layout or on a
// natural-order copy of the state, or all of a step's levels in one
// cooperative persistent launch with a grid barrier after each level
// (bounded: a barrier that does not complete within 2 s sets an error flag
// that the host reads).
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

// The device lists hold points as packed coordinates (the last axis in the
// lowest bits; 63, 31 or 21 bits per axis in 1, 2 or 3 dimensions, wider
// than any grid that fits in memory), so the kernels find a point's
// neighbours and colour without divisions.
template <int D> struct CoordBits {
    static constexpr int bits = D == 1 ? 63 : (D == 2 ? 31 : 21);
    static constexpr int64_t mask = (int64_t)(~uint64_t(0) >> (64 - bits));
};

template <int D> __host__ __device__ __forceinline__ int64_t pack_coords(int64_t i, int64_t N)
{
    int64_t packed = 0, rem = i;
    for (int a = 0; a < D; ++a) {
        packed |= (rem % N) << (CoordBits<D>::bits * a);
        rem /= N;
    }
    return packed;
}

// Update the point with packed coordinates pc in place.  CG: load and store
// through L2 only (ld/st .cg), for the persistent kernel, whose CTAs read in
// one level what other SMs wrote in an earlier one (L1 is not coherent
// across SMs).  Neighbours in the order of the colour passes (axis 0 first;
// per axis the lower, then the upper).
template <typename T, int D, int MODE, bool CG, bool SPLIT = true>
__device__ __forceinline__ void level_point(vec2_t<T>* pq, vec2_t<T>* uv, int64_t pc, int64_t N,
                                            const Coef<T>& c)
{
    int64_t x[3] = {0, 0, 0};  // x[0] = last axis
#pragma unroll
    for (int a = 0; a < D; ++a) x[a] = (pc >> (CoordBits<D>::bits * a)) & CoordBits<D>::mask;
    int64_t i = 0, st[3];
    {
        int64_t m = 1;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            st[a] = m;
            i += x[a] * m;
            m *= N;
        }
    }
    int64_t nb[2 * D];
#pragma unroll
    for (int a = D - 1, n = 0; a >= 0; --a) {  // axis 0 is the highest packed axis
        nb[n++] = x[a] == 0 ? i + (N - 1) * st[a] : i - st[a];
        nb[n++] = x[a] == N - 1 ? i - (N - 1) * st[a] : i + st[a];
    }
    if constexpr (!SPLIT) {
        // natural order, (P,Q) and (U,V) as vec2 arrays
        T p[2 * D], q[2 * D], w[2 * D];
#pragma unroll
        for (int m = 0; m < 2 * D; ++m) {
            const vec2_t<T> b = pq[nb[m]];
            p[m] = b.x;
            q[m] = b.y;
            w[m] = uv[nb[m]].x;
        }
        vec2_t<T> a = pq[i], e = uv[i];
        update_point<T, D, MODE>(c, nsum_scaled(p, c.beta), nsum_scaled(q, c.beta), nsum_scaled(w, c.Bp), a.x,
                                 a.y, e.x, e.y);
        pq[i] = a;
        uv[i] = e;
        return;
    }
    // the handle's colour-split layout: the neighbours are in the other half
    const int64_t half = (D == 1 ? N : (D == 2 ? N * N : N * N * N)) >> 1;
    const int par = (int)((x[0] + x[1] + x[2]) & 1);
    const int64_t own = (par ? half : 0) + (i >> 1), oth = par ? 0 : half;
    T* u = reinterpret_cast<T*>(uv);  // planar: U at a position, V at 2 half + position
    T p[2 * D], q[2 * D], w[2 * D];
#pragma unroll
    for (int m = 0; m < 2 * D; ++m) {
        const int64_t j = oth + (nb[m] >> 1);
        const vec2_t<T> b = CG ? __ldcg(&pq[j]) : pq[j];
        p[m] = b.x;
        q[m] = b.y;
        w[m] = CG ? __ldcg(&u[j]) : u[j];
    }
    vec2_t<T> a = CG ? __ldcg(&pq[own]) : pq[own];
    T U = CG ? __ldcg(&u[own]) : u[own];
    T V = CG ? __ldcg(&u[2 * half + own]) : u[2 * half + own];
    update_point<T, D, MODE>(c, nsum_scaled(p, c.beta), nsum_scaled(q, c.beta), nsum_scaled(w, c.Bp), a.x,
                             a.y, U, V);
    if (CG) {
        __stcg(&pq[own], a);
        __stcg(&u[own], U);
        __stcg(&u[2 * half + own], V);
    } else {
        pq[own] = a;
        u[own] = U;
        u[2 * half + own] = V;
    }
}

// One level.  Small levels are launched with programmatic dependent launch:
// the next level's grid may be scheduled as soon as every CTA of this one
// has started, and waits (griddepcontrol.wait) until this grid has completed
// and its stores are visible before it reads anything -- so the launch
// latency of level l + 1 overlaps the work of level l.  (Without the launch
// attribute both instructions are no-ops.)
template <typename T, int D, int MODE, bool SPLIT>
__global__ void __launch_bounds__(256) level_kernel(vec2_t<T>* pq, vec2_t<T>* uv, const int64_t* list,
                                                    int64_t count, int64_t N, Coef<T> c)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    level_point<T, D, MODE, false, SPLIT>(pq, uv, list[k], N, c);
}

template <typename T, int D, int MODE, bool SPLIT>
static cudaError_t launch_level_pdl(unsigned blocks, int threads, cudaStream_t s, vec2_t<T>* pq, vec2_t<T>* uv,
                                    const int64_t* list, int64_t count, int64_t N, const Coef<T>& c, bool pdl)
{
    if (!pdl) {
        level_kernel<T, D, MODE, SPLIT><<<blocks, threads, 0, s>>>(pq, uv, list, count, N, c);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, level_kernel<T, D, MODE, SPLIT>, pq, uv, list, count, N, c);
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier of the persistent level kernel (all its CTAs are co-resident:
// cooperative launch).  The last CTA to arrive resets the count and advances
// the generation; the others wait for the generation to change, for at most
// kBarrierNs of wall time, then set bar->err and give up.  Returns false once
// any CTA has given up (every CTA then leaves the kernel).
constexpr uint64_t kBarrierNs = 2000000000ull;

__device__ __forceinline__ bool grid_sync(OrderBarrier* bar, unsigned expected, unsigned& gen)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();  // this CTA's updates before its arrival
        if (atomicAdd(&bar->count, 1u) == expected - 1u) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            while (atomicAdd(&bar->gen, 0u) == gen) {
                if (atomicAdd(&bar->err, 0) != 0) break;
                if (globaltimer_ns() - t0 > kBarrierNs) {
                    atomicExch(&bar->err, 1);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();  // the other CTAs' updates before this CTA's next reads
    }
    ++gen;
    __syncthreads();
    return *(volatile int*)&bar->err == 0;
}

// One DP-AVF2 step in a single launch: the levels upward with base updates,
// then downward with adjoint updates, a grid barrier after each level.
// expected = gridDim.x normally; a test sets it higher to exercise the timeout.
constexpr int kPersistentThreads = 64;  // small CTAs: a level's points over many SMs

template <typename T, int D>
__global__ void __launch_bounds__(kPersistentThreads) level_persistent_kernel(vec2_t<T>* pq, vec2_t<T>* uv,
                                                               const int64_t* list, const int64_t* offsets,
                                                               int64_t nlevels, int64_t N, Coef<T> c,
                                                               OrderBarrier* bar, unsigned expected)
{
    unsigned gen = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int pass = 0; pass < 2; ++pass) {
        for (int64_t k = 0; k < nlevels; ++k) {
            const int64_t l = pass == 0 ? k : nlevels - 1 - k;
            const int64_t o = offsets[l], n = offsets[l + 1] - o;
            for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
                if (pass == 0) level_point<T, D, RED_BASE, true>(pq, uv, list[o + t], N, c);
                else level_point<T, D, RED_ADJ, true>(pq, uv, list[o + t], N, c);
            }
            if (!grid_sync(bar, expected, gen)) return;
        }
    }
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
        const int64_t pc = dim == 1 ? pack_coords<1>(p, N) : (dim == 2 ? pack_coords<2>(p, N) : pack_coords<3>(p, N));
        list[(size_t)fill[(size_t)level[(size_t)p]]++] = pc;
    }
    return 0;
}

template <typename T>
int launch_level(int dim, int mode, vec2_t<T>* pq, vec2_t<T>* uv, const int64_t* list, int64_t count,
                 int64_t N, const Coef<T>& c, bool split, cudaStream_t s)
{
    if (count <= 0) return 0;
    // small levels: small CTAs, spread over more SMs, and launched early
    // (programmatic dependent launch), since launch latency binds them;
    // large levels gain nothing from either (3D lexicographic: -9% with PDL)
    const bool small = count < 148 * 256;
    const int threads = small ? 64 : 256;
    const unsigned blocks = (unsigned)((count + threads - 1) / threads);
    const bool base = mode == RED_BASE;
    cudaError_t e = cudaSuccess;
#define KGS_LEVEL_S(DD, SP)                                                                            \
    if (base) e = launch_level_pdl<T, DD, RED_BASE, SP>(blocks, threads, s, pq, uv, list, count, N, c, small); \
    else e = launch_level_pdl<T, DD, RED_ADJ, SP>(blocks, threads, s, pq, uv, list, count, N, c, small);
#define KGS_LEVEL(DD)                 \
    if (split) { KGS_LEVEL_S(DD, true) } \
    else { KGS_LEVEL_S(DD, false) }
    if (dim == 1) { KGS_LEVEL(1) }
    else if (dim == 2) { KGS_LEVEL(2) }
    else { KGS_LEVEL(3) }
#undef KGS_LEVEL
#undef KGS_LEVEL_S
    return e == cudaSuccess ? 1 : -1;
}

template <typename T, int D>
static int launch_persistent_d(vec2_t<T>* pq, vec2_t<T>* uv, const int64_t* list, const int64_t* offsets,
                               int64_t nlevels, int64_t max_level, int64_t N, const Coef<T>& c,
                               OrderBarrier* bar, int extra, cudaStream_t s)
{
    int dev = 0, sms = 148, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, level_persistent_kernel<T, D>, kPersistentThreads, 0);
    if (per < 1) return -1;
    int64_t g = (max_level + kPersistentThreads - 1) / kPersistentThreads;
    const int64_t cap = (int64_t)sms * per;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    unsigned expected = (unsigned)g + (unsigned)(extra > 0 ? extra : 0);
    if (cudaMemsetAsync(bar, 0, sizeof(OrderBarrier), s) != cudaSuccess) return -1;
    Coef<T> cc = c;
    void* args[] = {&pq, &uv, &list, &offsets, &nlevels, &N, &cc, &bar, &expected};
    if (cudaLaunchCooperativeKernel((const void*)level_persistent_kernel<T, D>, dim3((unsigned)g),
                                    dim3(kPersistentThreads), args, 0, s) != cudaSuccess)
        return -1;
    return 1;
}

template <typename T>
int launch_level_persistent(int dim, vec2_t<T>* pq, vec2_t<T>* uv, const int64_t* list,
                            const int64_t* offsets, int64_t nlevels, int64_t max_level, int64_t N,
                            const Coef<T>& c, OrderBarrier* bar, int extra, cudaStream_t s)
{
    if (dim == 1) return launch_persistent_d<T, 1>(pq, uv, list, offsets, nlevels, max_level, N, c, bar, extra, s);
    if (dim == 2) return launch_persistent_d<T, 2>(pq, uv, list, offsets, nlevels, max_level, N, c, bar, extra, s);
    return launch_persistent_d<T, 3>(pq, uv, list, offsets, nlevels, max_level, N, c, bar, extra, s);
}

template int launch_level_persistent<double>(int, vec2_t<double>*, vec2_t<double>*, const int64_t*,
                                             const int64_t*, int64_t, int64_t, int64_t, const Coef<double>&,
                                             OrderBarrier*, int, cudaStream_t);
template int launch_level_persistent<float>(int, vec2_t<float>*, vec2_t<float>*, const int64_t*,
                                            const int64_t*, int64_t, int64_t, int64_t, const Coef<float>&,
                                            OrderBarrier*, int, cudaStream_t);

template int launch_level<double>(int, int, vec2_t<double>*, vec2_t<double>*, const int64_t*, int64_t,
                                  int64_t, const Coef<double>&, bool, cudaStream_t);
template int launch_level<float>(int, int, vec2_t<float>*, vec2_t<float>*, const int64_t*, int64_t,
                                 int64_t, const Coef<float>&, bool, cudaStream_t);

}  // namespace kgs
