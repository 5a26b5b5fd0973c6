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

KGS_BOUNDS_TU
KGS_BOUNDS_READER(bounds_flags_sweep)

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

// Update the point k of row (i0, i1) (axis-0 and axis-1 coordinates; i1 = 0
// in 2D, both 0 in 1D) of the colour with 0-based index-sum parity `parity`,
// on the colour-split layout.  N_I = N in the index type I.  NC: read the
// other colour through the non-coherent (read-only) path, valid when no
// other CTA writes it during the launch; otherwise plain (coherent) loads.
template <typename T, int D, int MODE, typename I, bool NC>
__device__ __forceinline__ void pass_point(vec2_t<T>* pq, vec2_t<T>* uv, int N, const Coef<T>& c,
                                           int i0, int i1, int k)
{
    const I n = N;
    I row = 0;
    if (D == 2) row = i0;
    else if (D == 3) row = (I)i0 * n + i1;
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
    const int parity = (i0 + i1 + k) & 1;
    const I half = (D == 1 ? n : (D == 2 ? n * n : n * n * n)) >> 1;
    const I own = (parity ? half : 0) + (i >> 1);
    const I oth = parity ? 0 : half;
    T* u = reinterpret_cast<T*>(uv);  // planar: U at a position, V at 2 half + position
    {
        bool ok = own >= 0 && own < 2 * half;
#pragma unroll
        for (int m = 0; m < 2 * D; ++m) ok = ok && oth + (nb[m] >> 1) >= 0 && oth + (nb[m] >> 1) < 2 * half;
        if (!kgs_in_bounds(ok, 1u)) return;
    }
    T p[2 * D], q[2 * D], w[2 * D];
#pragma unroll
    for (int m = 0; m < 2 * D; ++m) {
        const I j = oth + (nb[m] >> 1);
        const vec2_t<T> b = NC ? __ldg(&pq[j]) : pq[j];
        p[m] = b.x;
        q[m] = b.y;
        w[m] = NC ? __ldg(&u[j]) : u[j];
    }
    vec2_t<T> a = pq[own];
    T U = u[own], V = u[2 * half + own];
    update_point<T, D, MODE>(c, nsum_scaled(p, c.beta), nsum_scaled(q, c.beta), nsum_scaled(w, c.Bp), a.x, a.y, U, V);
    pq[own] = a;
    u[own] = U;
    u[2 * half + own] = V;
}

// One launch per colour pass.  The launch grid carries the row coordinates
// (blockIdx.y = axis D-2, blockIdx.z = axis 0 for D = 3), so a thread finds its
// point without divisions; blockIdx.x * blockDim.x + threadIdx.x runs over the
// N/2 points of the pass's colour in the row.  32-bit indices when N^d < 2^31.
//
// In the slab schedule (pass_pair) the launches after a pair's first two are
// programmatic dependent launches: a black slab pass B(k) reads the red slabs
// k-1 .. k+1, which no launch still running writes (the red pass just before
// it writes slab k-2), so it starts at once and overlaps that red pass's
// tail; a red slab pass waits (griddepcontrol.wait) for the black pass just
// before it, which itself started only after the red pass before it had
// passed its own wait -- so the black slabs on both sides are complete.
// Both instructions are no-ops in a plain launch.
// Outside the slab schedule (wait_all) every pass waits for the one before it.
template <typename T, int D, int MODE, typename I>
__global__ void __launch_bounds__(512) pass_kernel(vec2_t<T>* pq, vec2_t<T>* uv, int N, Coef<T> c,
                                                   int parity, int plane0, int wait_all)
{
    if (MODE != BLACK_FUSED || wait_all) asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int kk = blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * kk >= N) return;
    int i0 = 0, i1 = 0, rp = 0;
    if (D == 2) {
        i0 = plane0 + (int)blockIdx.y;
        rp = i0 & 1;
    } else if (D == 3) {
        i0 = plane0 + (int)blockIdx.z;
        i1 = blockIdx.y;
        rp = (i0 + i1) & 1;
    }
    const int k = 2 * kk + ((parity - rp) & 1);
    pass_point<T, D, MODE, I, true>(pq, uv, N, c, i0, i1, k);
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

// ------------------------------------------------------------------ wave --
// One (BLACK_FUSED, REDMODE) pair of colour passes in one launch, so that a
// step reads and writes the state about once instead of once per pass.  The
// grid is cut along axis 0 into ns slabs of S planes; an item is one colour
// of one slab, cut into `chunks` chunks of `rows` rows (lines along the last
// axis).  Persistent CTAs take chunks in ticket order (one atomic counter):
//   B(0) .. B(lag), then B(k), R(k - lag) for k = lag+1 .. ns-1,
//   then R(ns-lag) .. R(ns-1), R(0),
// B = black, R = red.  A red slab needs the black slabs on both sides
// updated, and a black slab needs the red slabs on both sides not yet
// updated; so R(j) waits until B(j-1), B(j), B(j+1) (periodic) are complete,
// and comes after B(j+1) in ticket order (R(0), whose lower neighbour is
// B(ns-1), goes last).  Black chunks never wait.  A CTA takes its tickets in
// increasing order and a chunk waits only for chunks with earlier tickets,
// held by running CTAs, so the schedule cannot deadlock; the launch is
// cooperative all the same (all CTAs resident), and a wait longer than
// kWaveWaitNs sets the error words, after which every CTA leaves.  Black
// chunks read red values that no CTA writes before they finish, so the only
// cross-CTA reads are the red chunks' reads of black values, ordered by a
// release (CTA barrier, then thread 0's counter increment) and an acquire
// (thread 0's counter read, then a CTA barrier); the loads are plain,
// coherent ones (not the read-only path).  The pointwise code is pass_point,
// so the result is bitwise that of the two passes.  (Measured on B300 with
// FP32 state, 3D 256^3: 26% fewer DRAM bytes than the two passes, but at 37%
// of DRAM peak against their 67% -- latency-bound on the per-chunk barriers
// and the pipeline's fill and drain -- so it stays opt-in.)
constexpr uint64_t kWaveWaitNs = 2000000000ull;

__device__ __forceinline__ uint64_t wave_clock_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned load_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void add_release(unsigned* p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Item q of the ticket order: colour (1 = red) and slab.
__device__ __forceinline__ void wave_item(int q, int ns, int lag, int& red, int& slab)
{
    const int a = lag + 1, mid = 2 * (ns - 1 - lag);
    if (q < a) {
        red = 0;
        slab = q;
    } else if (q < a + mid) {
        const int r = q - a, k = a + (r >> 1);
        red = r & 1;
        slab = red ? k - lag : k;
    } else {
        const int r = q - a - mid;
        red = 1;
        slab = r < lag ? ns - lag + r : 0;
    }
}

template <typename T, int D, int MODE, typename I>
__device__ __forceinline__ void wave_chunk(vec2_t<T>* pq, vec2_t<T>* uv, int N, const Coef<T>& c,
                                           const WaveParams& wp, int slab, int chunk)
{
    const int parity = MODE == BLACK_FUSED ? (red_parity(D) ^ 1) : red_parity(D);
    const int rows_per_plane = D == 3 ? N : 1;
    const int row0 = slab * wp.S * rows_per_plane + chunk * wp.rows;
    const int hN = N >> 1;
    // the chunk's rows x N/2 points of the colour, spread over all threads
    for (int e = threadIdx.x; e < wp.rows * hN; e += blockDim.x) {
        const int r = e / hN, kk = e - r * hN;
        const int row = row0 + r;
        const int i0 = D == 3 ? row / N : row;
        const int i1 = D == 3 ? row - i0 * N : 0;
        const int rp = (i0 + i1) & 1;
        pass_point<T, D, MODE, I, false>(pq, uv, N, c, i0, i1, 2 * kk + ((parity - rp) & 1));
    }
}

template <typename T, int D, int REDMODE, typename I>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 8 : 3)
    wave_kernel(vec2_t<T>* pq, vec2_t<T>* uv, int N, Coef<T> c, WaveParams wp, unsigned* sync, int* err)
{
    __shared__ int s_ticket, s_go;
    const int total = 2 * wp.ns * wp.chunks;
    unsigned* derr = sync + 1;  // device copy of the error word
    unsigned* done = sync + 2;  // black slab k at k, red slab k at ns + k
    // thread 0 fetches the next ticket while the CTA works on the current one
    // (the CTA still takes its tickets in increasing order)
    int next = threadIdx.x == 0 ? (int)atomicAdd(&sync[0], 1u) : 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = next;
            int go = t < total;
            if (go) {
                int red, slab;
                wave_item(t / wp.chunks, wp.ns, wp.lag, red, slab);
                if (red) {
                    const unsigned need = (unsigned)(wp.chunks + wp.stall);
                    const int nb[3] = {slab == 0 ? wp.ns - 1 : slab - 1, slab, slab == wp.ns - 1 ? 0 : slab + 1};
                    const uint64_t t0 = wave_clock_ns();
                    for (int k = 0; k < 3 && go; ++k) {
                        while (load_acquire(&done[nb[k]]) < need) {
                            if (*(volatile unsigned*)derr || wave_clock_ns() - t0 > kWaveWaitNs) {
                                *(volatile unsigned*)derr = 1u;
                                *(volatile int*)err = 1;
                                go = 0;
                                break;
                            }
                            __nanosleep(64);
                        }
                    }
                }
            }
            if (go) next = (int)atomicAdd(&sync[0], 1u);
            s_ticket = t;
            s_go = go;
        }
        __syncthreads();  // also carries thread 0's acquire to the CTA
        const int t = s_ticket;
        if (!s_go) break;
        int red, slab;
        wave_item(t / wp.chunks, wp.ns, wp.lag, red, slab);
        const int chunk = t % wp.chunks;
        if (red) wave_chunk<T, D, REDMODE, I>(pq, uv, N, c, wp, slab, chunk);
        else wave_chunk<T, D, BLACK_FUSED, I>(pq, uv, N, c, wp, slab, chunk);
        __syncthreads();  // the CTA's stores precede thread 0's release
        if (threadIdx.x == 0) add_release(&done[(red ? wp.ns : 0) + slab], 1u);
    }
}

// Co-resident CTAs of the wave kernel for a grid (the cooperative launch's size).
template <typename T, int D>
static int wave_ctas_t(int64_t M)
{
    auto kern = M < ((int64_t)1 << 31) ? wave_kernel<T, D, RED_FUSED, int32_t> : wave_kernel<T, D, RED_FUSED, int64_t>;
    int dev = 0, sms = 148, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, 0) != cudaSuccess || per < 1) return -1;
    return sms * per;
}

int wave_ctas(int dim, int elem_bytes, int64_t M)
{
    if (dim == 2) return elem_bytes == 8 ? wave_ctas_t<double, 2>(M) : wave_ctas_t<float, 2>(M);
    if (dim == 3) return elem_bytes == 8 ? wave_ctas_t<double, 3>(M) : wave_ctas_t<float, 3>(M);
    return -1;
}

int wave_plan(int dim, int64_t N, int elem_bytes, int64_t want_S, int want_lag, int64_t want_chunk, int ctas,
              WaveParams& wp)
{
    if (dim < 2 || N < 64 || N > 65536 || ctas < 1) return -1;
    const int rows_per_plane = dim == 3 ? (int)N : 1;
    const int64_t plane_bytes = (dim == 3 ? N * N : N) * 4 * (int64_t)elem_bytes;
    // slab: about 4 MB of state unless given, and at most N/8 planes (so that
    // a small grid still gets a pipeline of slabs); S divides N
    int64_t S = want_S > 0 ? want_S
                           : std::max<int64_t>(1, std::min<int64_t>(((int64_t)4 << 20) / plane_bytes, N / 8));
    if (S > N) S = N;
    while (N % S) --S;
    const int64_t ns = N / S;
    // chunk: about 2048 points of a colour unless given (whole rows)
    const int64_t half_row = N / 2;
    int64_t rows = std::max<int64_t>(1, (want_chunk > 0 ? want_chunk : 2048) / half_row);
    const int64_t slab_rows = S * rows_per_plane;
    if (rows > slab_rows) rows = slab_rows;
    while (slab_rows % rows) --rows;
    const int64_t chunks = slab_rows / rows;
    if (2 * ns * chunks >= ((int64_t)1 << 31)) return -1;
    // lag: the red slabs trail far enough that the black slabs they wait for
    // have left the window of chunks in flight (one per CTA), unless given
    int64_t lag = want_lag > 0 ? want_lag : 2 + (ctas + 2 * chunks - 1) / (2 * chunks);
    if (want_lag <= 0 && lag > ns - 2) lag = ns - 2;
    if (lag < 1 || ns < lag + 2) return -1;
    wp.S = (int)S;
    wp.ns = (int)ns;
    wp.rows = (int)rows;
    wp.chunks = (int)chunks;
    wp.lag = lag;
    wp.stall = 0;
    return 0;
}

template <typename T, int D, int REDMODE>
static int launch_wave_t(const Grid& g, vec2_t<T>* pq, vec2_t<T>* uv, const Coef<T>& c, const WaveParams& wp,
                         unsigned* sync, int* err, cudaStream_t s)
{
    auto kern = g.M < ((int64_t)1 << 31) ? wave_kernel<T, D, REDMODE, int32_t> : wave_kernel<T, D, REDMODE, int64_t>;
    int dev = 0, sms = 148, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, 0) != cudaSuccess || per < 1) return -1;
    const int64_t total = 2 * (int64_t)wp.ns * wp.chunks;
    const unsigned grid = (unsigned)std::min<int64_t>((int64_t)sms * per, total);
    // every CTA may fetch one ticket past the end
    if (total + grid >= ((int64_t)1 << 31)) return -1;
    if (cudaMemsetAsync(sync, 0, (size_t)(2 + 2 * wp.ns) * sizeof(unsigned), s) != cudaSuccess) return -1;
    int n = (int)g.N;
    Coef<T> cc = c;
    WaveParams w = wp;
    void* args[] = {&pq, &uv, &n, &cc, &w, &sync, &err};
    if (cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(256), args, 0, s) != cudaSuccess) return -1;
    return 1;
}

template <typename T>
int launch_wave(const Grid& g, int red_mode, vec2_t<T>* pq, vec2_t<T>* uv, const Coef<T>& c,
                const WaveParams& wp, unsigned* sync, int* err, cudaStream_t s)
{
    const bool adj = red_mode == RED_ADJ;
    if (g.dim == 2)
        return adj ? launch_wave_t<T, 2, RED_ADJ>(g, pq, uv, c, wp, sync, err, s)
                   : launch_wave_t<T, 2, RED_FUSED>(g, pq, uv, c, wp, sync, err, s);
    if (g.dim == 3)
        return adj ? launch_wave_t<T, 3, RED_ADJ>(g, pq, uv, c, wp, sync, err, s)
                   : launch_wave_t<T, 3, RED_FUSED>(g, pq, uv, c, wp, sync, err, s);
    return -1;
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
    auto kern = g.M < ((int64_t)1 << 31) ? pass_kernel<T, D, MODE, int32_t> : pass_kernel<T, D, MODE, int64_t>;
    const int wait_all = g.pdl_wait ? 1 : 0;
    if (!g.pdl) {
        kern<<<grid, threads, 0, s>>>(pq, uv, (int)g.N, c, parity, plane0, wait_all);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3((unsigned)threads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, pq, uv, (int)g.N, c, parity, plane0, wait_all);
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
template int launch_wave<double>(const Grid&, int, double2*, double2*, const Coef<double>&, const WaveParams&,
                                 unsigned*, int*, cudaStream_t);
template int launch_wave<float>(const Grid&, int, float2*, float2*, const Coef<float>&, const WaveParams&,
                                unsigned*, int*, cudaStream_t);
template int launch_smem_run<double>(const Grid&, double2*, double2*, const Coef<double>&, int64_t, cudaStream_t);
template int launch_smem_run<float>(const Grid&, float2*, float2*, const Coef<float>&, int64_t, cudaStream_t);

}  // namespace kgs
