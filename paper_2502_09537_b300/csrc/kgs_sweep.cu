// kgs_sweep.cu -- checkerboard colour-pass kernels of the DP-AVF2 scheme.
//
// The paper's GPU ordering (Sec. 4.2, Algorithm 3) updates every point of one
// colour concurrently, since no point has a neighbour of its own colour (N
// even).  Here one step is two fused colour passes (see PassMode in
// kgs_point.cuh) instead of Algorithm 3's four, and each pass computes its
// neighbour sums once for both of the half-step updates it applies.
//
// Two variants, bitwise identical (same pointwise code, same neighbour order):
//   pass_kernel       one launch per colour pass over an N^d grid in global
//                     memory; one thread per point of the pass's colour.
//   (kgs_tile.cu)     several passes per launch on shared-memory tiles.
//   smem_run_kernel   a whole n-step run inside one CTA with the state resident
//                     in shared memory (small grids: the 1D workloads).
#include <algorithm>

#include "kgs_internal.h"

namespace kgs {

// Linear index of the t-th point of the colour whose 0-based index sum has
// parity `parity`, and its 2*D periodic neighbours in the order
// (axis 0 down, axis 0 up, axis 1 down, ...).  Rows run along the last axis;
// each row holds N/2 points of each colour.
template <int D>
__device__ __forceinline__ int64_t colour_point(int64_t t, int64_t N, int parity, int64_t nb[2 * D])
{
    const int64_t hN = N >> 1;
    const int64_t row = t / hN;
    const int64_t kk = t - row * hN;
    int64_t i0 = 0, i1 = 0;
    int rp = 0;
    if (D == 2) {
        i0 = row;
        rp = (int)(i0 & 1);
    } else if (D == 3) {
        i0 = row / N;
        i1 = row - i0 * N;
        rp = (int)((i0 + i1) & 1);
    }
    const int64_t k = 2 * kk + ((parity - rp) & 1);
    const int64_t i = row * N + k;
    const int64_t km = (k == 0) ? i + (N - 1) : i - 1;
    const int64_t kp = (k == N - 1) ? i - (N - 1) : i + 1;
    if (D == 1) {
        nb[0] = km;
        nb[1] = kp;
    } else if (D == 2) {
        nb[0] = (i0 == 0) ? i + (N - 1) * N : i - N;
        nb[1] = (i0 == N - 1) ? i - (N - 1) * N : i + N;
        nb[2] = km;
        nb[3] = kp;
    } else {
        const int64_t N2 = N * N;
        nb[0] = (i0 == 0) ? i + (N - 1) * N2 : i - N2;
        nb[1] = (i0 == N - 1) ? i - (N - 1) * N2 : i + N2;
        nb[2] = (i1 == 0) ? i + (N - 1) * N : i - N;
        nb[3] = (i1 == N - 1) ? i - (N - 1) * N : i + N;
        nb[4] = km;
        nb[5] = kp;
    }
    return i;
}

// beta S_P, beta S_Q and B' S_U over the neighbours nb of colour_point.
// GLOBAL: the state is the handle's, in HBM in the colour-split layout (the
// neighbours sit in the other colour's half, from pq + oth; U planar); otherwise
// it is in shared memory in natural vec2 order (oth = 0, positions are linear
// indices).
template <typename T, int D, bool GLOBAL>
__device__ __forceinline__ void neighbour_sums(const vec2_t<T>* pq, const vec2_t<T>* uv,
                                               const int64_t nb[2 * D], int64_t oth, const Coef<T>& c,
                                               T& bSP, T& bSQ, T& BSU)
{
    const T* u = reinterpret_cast<const T*>(uv);
    T p[2 * D], q[2 * D], w[2 * D];
#pragma unroll
    for (int n = 0; n < 2 * D; ++n) {
        const int64_t k = GLOBAL ? oth + (nb[n] >> 1) : nb[n];
        const vec2_t<T> b = GLOBAL ? __ldg(&pq[k]) : pq[k];
        p[n] = b.x;
        q[n] = b.y;
        w[n] = GLOBAL ? __ldg(&u[k]) : u[2 * k];
    }
    bSP = nsum_scaled(p, c.beta);
    bSQ = nsum_scaled(q, c.beta);
    BSU = nsum_scaled(w, c.Bp);
}

template <typename T, int D, int MODE, bool GLOBAL>
__device__ __forceinline__ void colour_update(vec2_t<T>* pq, vec2_t<T>* uv, int64_t t, int64_t N,
                                              int64_t half, int parity, const Coef<T>& c)
{
    int64_t nb[2 * D];
    const int64_t i = colour_point<D>(t, N, parity, nb);
    const int64_t own = GLOBAL ? (parity ? half : 0) + (i >> 1) : i;
    const int64_t oth = GLOBAL ? (parity ? 0 : half) : 0;
    T bSP, bSQ, BSU;
    neighbour_sums<T, D, GLOBAL>(pq, uv, nb, oth, c, bSP, bSQ, BSU);
    vec2_t<T> a = pq[own];
    T* u = reinterpret_cast<T*>(uv);
    // (U,V): planar in HBM (U at own, V at 2 half + own), vec2 in shared memory
    const int64_t iu = GLOBAL ? own : 2 * own, iv = GLOBAL ? 2 * half + own : 2 * own + 1;
    T U = u[iu], V = u[iv];
    update_point<T, D, MODE>(c, bSP, bSQ, BSU, a.x, a.y, U, V);
    pq[own] = a;
    u[iu] = U;
    u[iv] = V;
}

// One launch per colour pass.  The launch grid carries the row coordinates
// (blockIdx.y = axis D-2, blockIdx.z = axis 0 for D = 3), so a thread finds its
// point without divisions; blockIdx.x * blockDim.x + threadIdx.x runs over the
// N/2 points of the pass's colour in the row.  32-bit indices when N^d < 2^31.
template <typename T, int D, int MODE, typename I>
__global__ void __launch_bounds__(512) pass_kernel(vec2_t<T>* pq, vec2_t<T>* uv, int N, Coef<T> c,
                                                   int parity, int plane0)
{
    const int kk = blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * kk >= N) return;
    const I n = N;
    int i0 = 0, i1 = 0, rp = 0;
    I row = 0;
    if (D == 2) {
        i0 = plane0 + (int)blockIdx.y;
        rp = i0 & 1;
        row = i0;
    } else if (D == 3) {
        i0 = plane0 + (int)blockIdx.z;
        i1 = blockIdx.y;
        rp = (i0 + i1) & 1;
        row = (I)i0 * n + i1;
    }
    const int k = 2 * kk + ((parity - rp) & 1);
    const I i = row * n + k;
    I nb[2 * D];
    const I km = (k == 0) ? i + (n - 1) : i - 1;
    const I kp = (k == N - 1) ? i - (n - 1) : i + 1;
    if (D == 1) {
        nb[0] = km;
        nb[1] = kp;
    } else if (D == 2) {
        nb[0] = (i0 == 0) ? i + (n - 1) * n : i - n;
        nb[1] = (i0 == N - 1) ? i - (n - 1) * n : i + n;
        nb[2] = km;
        nb[3] = kp;
    } else {
        const I n2 = n * n;
        nb[0] = (i0 == 0) ? i + (n - 1) * n2 : i - n2;
        nb[1] = (i0 == N - 1) ? i - (n - 1) * n2 : i + n2;
        nb[2] = (i1 == 0) ? i + (n - 1) * n : i - n;
        nb[3] = (i1 == N - 1) ? i - (n - 1) * n : i + n;
        nb[4] = km;
        nb[5] = kp;
    }
    // colour-split layout: this colour's half from pq + own, the other's from pq + oth
    const I half = (D == 1 ? n : (D == 2 ? n * n : n * n * n)) >> 1;
    const I own = (parity ? half : 0) + (i >> 1);
    const I oth = parity ? 0 : half;
    T* u = reinterpret_cast<T*>(uv);  // planar: U at a position, V at 2 half + position
    T p[2 * D], q[2 * D], w[2 * D];
#pragma unroll
    for (int m = 0; m < 2 * D; ++m) {
        const I k = oth + (nb[m] >> 1);
        const vec2_t<T> b = __ldg(&pq[k]);
        p[m] = b.x;
        q[m] = b.y;
        w[m] = __ldg(&u[k]);
    }
    vec2_t<T> a = pq[own];
    T U = u[own], V = u[2 * half + own];
    update_point<T, D, MODE>(c, nsum_scaled(p, c.beta), nsum_scaled(q, c.beta), nsum_scaled(w, c.Bp), a.x, a.y, U, V);
    pq[own] = a;
    u[own] = U;
    u[2 * half + own] = V;
}

// Persistent variant: a grid sized so that every thread gets nearly the same
// number of points (the colour's points walked with a grid stride), which
// trims the partial last wave of a one-thread-per-point launch.  Its index
// divisions run beside the FP64 pipe, so it pays off where that pipe binds.
template <typename T, int D, int MODE>
__global__ void __launch_bounds__(256) pass_persistent_kernel(vec2_t<T>* pq, vec2_t<T>* uv,
                                                              int64_t N, int64_t half, Coef<T> c,
                                                              int parity)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < half; t += stride)
        colour_update<T, D, MODE, true>(pq, uv, t, N, half, parity, c);
}

template <typename T, int D, int MODE>
__device__ __forceinline__ void smem_pass(vec2_t<T>* pq, vec2_t<T>* uv, int64_t N, int64_t half,
                                          int parity, const Coef<T>& c)
{
    for (int64_t t = threadIdx.x; t < half; t += blockDim.x)
        colour_update<T, D, MODE, false>(pq, uv, t, N, half, parity, c);
    __syncthreads();
}

template <typename T, int D>
__global__ void __launch_bounds__(1024) smem_run_kernel(vec2_t<T>* pq, vec2_t<T>* uv, int64_t N,
                                                        int64_t M, Coef<T> c, int64_t nsteps)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    vec2_t<T>* spq = reinterpret_cast<vec2_t<T>*>(smem_raw);
    vec2_t<T>* suv = spq + M;
    const int64_t half = M >> 1;
    // natural order in shared memory, the colour-split layout in HBM
    const T* gu = reinterpret_cast<const T*>(uv);  // planar U, V in HBM
    for (int64_t i = threadIdx.x; i < M; i += blockDim.x) {
        const int64_t j = split_pos(i, D, N, half);
        spq[i] = pq[j];
        vec2_t<T> b;
        b.x = gu[j];
        b.y = gu[M + j];
        suv[i] = b;
    }
    __syncthreads();
    const int red = red_parity(D), black = red ^ 1;
    smem_pass<T, D, RED_BASE>(spq, suv, N, half, red, c);
    for (int64_t n = 1; n < nsteps; ++n) {
        smem_pass<T, D, BLACK_FUSED>(spq, suv, N, half, black, c);
        smem_pass<T, D, RED_FUSED>(spq, suv, N, half, red, c);
    }
    smem_pass<T, D, BLACK_FUSED>(spq, suv, N, half, black, c);
    smem_pass<T, D, RED_ADJ>(spq, suv, N, half, red, c);
    T* pu = reinterpret_cast<T*>(uv);
    for (int64_t i = threadIdx.x; i < M; i += blockDim.x) {
        const int64_t j = split_pos(i, D, N, half);
        pq[j] = spq[i];
        pu[j] = suv[i].x;
        pu[M + j] = suv[i].y;
    }
}

int64_t smem_resident_max_points(int elem_bytes)
{
    // 227 KB of dynamic shared memory per CTA on sm_103a; 2 vec2 per point.
    const int64_t bytes = 227 * 1024;
    return bytes / (4 * (int64_t)elem_bytes);
}

template <typename T, int D, int MODE>
static void launch_pass_t(const Grid& g, vec2_t<T>* pq, vec2_t<T>* uv, const Coef<T>& c,
                          cudaStream_t s)
{
    const int hN = (int)(g.N >> 1);
    int threads = g.threads > 0 ? g.threads : 256;
    if (threads > hN) threads = (hN + 31) / 32 * 32;  // short rows: no idle warps
    const int64_t planes = (D >= 2 && g.planes > 0) ? g.planes : g.N;
    const int plane0 = D >= 2 ? (int)g.plane0 : 0;
    dim3 grid((unsigned)((hN + threads - 1) / threads), D == 2 ? (unsigned)planes : (D == 3 ? (unsigned)g.N : 1u),
              D == 3 ? (unsigned)planes : 1u);
    const int parity = (MODE == BLACK_FUSED) ? (red_parity(D) ^ 1) : red_parity(D);
    if (g.M < ((int64_t)1 << 31))
        pass_kernel<T, D, MODE, int32_t><<<grid, threads, 0, s>>>(pq, uv, (int)g.N, c, parity, plane0);
    else
        pass_kernel<T, D, MODE, int64_t><<<grid, threads, 0, s>>>(pq, uv, (int)g.N, c, parity, plane0);
}

// CTAs for the persistent pass: 148 SMs x b CTAs of 256 threads, b in 3..6
// chosen to minimise the idle fraction of the last grid-stride round.
static int64_t persistent_ctas(int64_t half)
{
    int64_t best = 148 * 4;
    double best_loss = 2.0;
    for (int b = 3; b <= 6; ++b) {
        const double threads = 148.0 * b * 256.0;
        const double x = (double)half / threads;
        const double rounds = (double)(int64_t)(x + 0.999999999);
        const double loss = rounds > 0 ? (rounds - x) / rounds : 1.0;
        if (loss < best_loss - 1e-3) {
            best_loss = loss;
            best = 148 * b;
        }
    }
    return best;
}

template <typename T, int D, int MODE>
static void launch_persistent_t(const Grid& g, vec2_t<T>* pq, vec2_t<T>* uv, const Coef<T>& c,
                                cudaStream_t s)
{
    const int64_t half = g.M >> 1;
    const int64_t ctas = std::min<int64_t>(persistent_ctas(half), (half + 255) / 256);
    const int parity = (MODE == BLACK_FUSED) ? (red_parity(D) ^ 1) : red_parity(D);
    pass_persistent_kernel<T, D, MODE><<<(unsigned)ctas, 256, 0, s>>>(pq, uv, g.N, half, c, parity);
}

template <typename T, int D>
static void launch_pass_d(const Grid& g, int mode, vec2_t<T>* pq, vec2_t<T>* uv,
                          const Coef<T>& c, cudaStream_t s)
{
    if (g.persistent) {
        switch (mode) {
        case RED_BASE: launch_persistent_t<T, D, RED_BASE>(g, pq, uv, c, s); break;
        case BLACK_FUSED: launch_persistent_t<T, D, BLACK_FUSED>(g, pq, uv, c, s); break;
        case RED_FUSED: launch_persistent_t<T, D, RED_FUSED>(g, pq, uv, c, s); break;
        default: launch_persistent_t<T, D, RED_ADJ>(g, pq, uv, c, s); break;
        }
        return;
    }
    switch (mode) {
    case RED_BASE: launch_pass_t<T, D, RED_BASE>(g, pq, uv, c, s); break;
    case BLACK_FUSED: launch_pass_t<T, D, BLACK_FUSED>(g, pq, uv, c, s); break;
    case RED_FUSED: launch_pass_t<T, D, RED_FUSED>(g, pq, uv, c, s); break;
    default: launch_pass_t<T, D, RED_ADJ>(g, pq, uv, c, s); break;
    }
}

template <typename T>
int launch_pass(const Grid& g, int mode, vec2_t<T>* pq, vec2_t<T>* uv, const Coef<T>& c,
                cudaStream_t stream)
{
    if (g.dim == 1) launch_pass_d<T, 1>(g, mode, pq, uv, c, stream);
    else if (g.dim == 2) launch_pass_d<T, 2>(g, mode, pq, uv, c, stream);
    else launch_pass_d<T, 3>(g, mode, pq, uv, c, stream);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template <typename T, int D>
static int launch_smem_d(const Grid& g, vec2_t<T>* pq, vec2_t<T>* uv, const Coef<T>& c,
                         int64_t nsteps, cudaStream_t s)
{
    const size_t bytes = (size_t)g.M * 2 * sizeof(vec2_t<T>);
    if (cudaFuncSetAttribute(smem_run_kernel<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes) != cudaSuccess)
        return -1;
    int threads = (int)((g.M / 2 + 31) / 32 * 32);
    if (threads > 1024) threads = 1024;
    if (threads < 32) threads = 32;
    smem_run_kernel<T, D><<<1, threads, bytes, s>>>(pq, uv, g.N, g.M, c, nsteps);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template <typename T>
int launch_smem_run(const Grid& g, vec2_t<T>* pq, vec2_t<T>* uv, const Coef<T>& c, int64_t nsteps,
                    cudaStream_t stream)
{
    if (g.M > smem_resident_max_points((int)sizeof(T))) return -1;
    if (g.dim == 1) return launch_smem_d<T, 1>(g, pq, uv, c, nsteps, stream);
    if (g.dim == 2) return launch_smem_d<T, 2>(g, pq, uv, c, nsteps, stream);
    return launch_smem_d<T, 3>(g, pq, uv, c, nsteps, stream);
}

template int launch_pass<double>(const Grid&, int, double2*, double2*, const Coef<double>&, cudaStream_t);
template int launch_pass<float>(const Grid&, int, float2*, float2*, const Coef<float>&, cudaStream_t);
template int launch_smem_run<double>(const Grid&, double2*, double2*, const Coef<double>&, int64_t, cudaStream_t);
template int launch_smem_run<float>(const Grid&, float2*, float2*, const Coef<float>&, int64_t, cudaStream_t);

}  // namespace kgs
