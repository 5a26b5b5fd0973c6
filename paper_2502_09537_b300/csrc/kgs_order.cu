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

// ---------------------------------------------------- lexicographic strips --
// The lexicographic order (Eq. order1) and its reverse in 2D, without one
// launch per level: a doacross sweep.  One warp owns a strip of 32 rows of
// the grid (natural order) and sweeps its columns with a skew of one column
// per lane: at step t lane a updates row r_a, column j = t - a (forward;
// mirrored for the reverse order: rows from the bottom, columns from the
// right).  In the forward order a point's earlier neighbours are the one
// above and the one to the left (new values), its later ones the one below
// and the one to the right (old values); at step t the point above was
// updated by lane a - 1 at step t - 1 (passed by a shuffle), the one to the
// left by the same lane at step t - 1 (kept in registers), and the ones
// below and to the right are not yet updated (read from memory).  The strip
// above is another warp's: lane 0 reads its last row from memory once that
// strip has published (release, every 8 steps) that it is at least 32 steps
// ahead of the column (acquire).  Wrap-around neighbours are read from memory:
// the left neighbour of column 0 is column N - 1 (still old), the right one
// of column N - 1 is column 0 (new, written by the same lane), the row above
// row 0 is row N - 1 (old: the last strip trails every other) and the row
// below row N - 1 is row 0 (new).  So every point sees exactly the values of
// the serial order, and with the same pointwise code and neighbour order as
// level_point the result is bitwise the level schedule's.  Warps take strips
// in ticket order (a strip waits only for the strip before it); the launch
// is cooperative; a wait longer than kLexWaitNs sets the error words and the
// warp leaves.
constexpr int kLexStrip = 32;
constexpr int kLexPublish = 8;  // steps between progress publications
constexpr uint64_t kLexWaitNs = 2000000000ull;

__device__ __forceinline__ unsigned lex_load_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// What one lane reads from memory for one step (all of it stable from the
// step before, so it is loaded one step ahead): its point, the later
// neighbours (next row, next column), and where they come from memory the
// earlier ones (lane 0's previous row; the first column's wrap-around column).
template <typename T> struct LexLoads {
    vec2_t<T> a, e;      // the point's (P,Q) and (U,V)
    vec2_t<T> nr, nc;    // (P,Q) of the next row's and the next column's neighbour
    T nrU, ncU;          // their U
    vec2_t<T> pr, pc;    // (P,Q) of the previous row's (lane 0) and previous column's (first column) neighbour
    T prU, pcU;
};

template <typename T, bool FWD>
__device__ __forceinline__ void lex_load(LexLoads<T>& L, const vec2_t<T>* pq, const vec2_t<T>* uv, int64_t N,
                                         int64_t r, int64_t rprev, int64_t rnext, int k, int lane)
{
    const T* u = reinterpret_cast<const T*>(uv);
    const int64_t j = FWD ? k : N - 1 - k;
    const int64_t jm = j == 0 ? N - 1 : j - 1, jp = j == N - 1 ? 0 : j + 1;
    const int64_t jprev = FWD ? jm : jp, jnext = FWD ? jp : jm;
    L.a = pq[r * N + j];
    L.e = uv[r * N + j];
    L.nr = pq[rnext * N + j];
    L.nrU = u[2 * (rnext * N + j)];
    L.nc = pq[r * N + jnext];
    L.ncU = u[2 * (r * N + jnext)];
    if (lane == 0) {
        L.pr = pq[rprev * N + j];
        L.prU = u[2 * (rprev * N + j)];
    }
    if (k == 0) {
        L.pc = pq[r * N + jprev];
        L.pcU = u[2 * (r * N + jprev)];
    }
}

template <typename T, int MODE, bool FWD>
__global__ void __launch_bounds__(32) lex_strip_kernel(vec2_t<T>* pq, vec2_t<T>* uv, int64_t N, Coef<T> c,
                                                       unsigned* sync, int* err, int stall)
{
    const int ns = (int)(N / kLexStrip);
    const int lane = threadIdx.x;
    const int steps = (int)N + kLexStrip - 1;
    unsigned* derr = sync + 1;
    unsigned* progress = sync + 2;  // steps strip s has completed, published
    for (;;) {
        int t0 = 0;
        if (lane == 0) t0 = (int)atomicAdd(&sync[0], 1u);
        t0 = __shfl_sync(0xffffffffu, t0, 0);
        if (t0 >= ns) break;
        const int s = FWD ? t0 : ns - 1 - t0;        // this strip
        const int sp = FWD ? s - 1 : s + 1;          // the strip updated before it (none at the ends)
        const bool has_prev = sp >= 0 && sp < ns;
        const int64_t r = FWD ? (int64_t)s * kLexStrip + lane : (int64_t)s * kLexStrip + kLexStrip - 1 - lane;
        const int64_t rm = r == 0 ? N - 1 : r - 1, rp = r == N - 1 ? 0 : r + 1;  // rows above and below
        const int64_t rprev = FWD ? rm : rp, rnext = FWD ? rp : rm;
        T cP = 0, cQ = 0, cU = 0;  // this lane's last update (the previous column's new values)
        LexLoads<T> cur, nxt;
        int ok = 1;
        for (int t = 0; t < steps; ++t) {
            if (has_prev && (t % kLexPublish) == 0) {
                // lane 0 reads the previous strip's last row at the columns of
                // steps t .. t + kLexPublish (the last one prefetched); that
                // strip's last lane reaches column x at its step x + 31
                if (lane == 0) {
                    const unsigned need = (unsigned)min(t + kLexPublish + kLexStrip, steps) + (unsigned)stall;
                    const uint64_t w0 = globaltimer_ns();
                    unsigned it = 0;
                    while (lex_load_acquire(&progress[sp]) < need) {
                        if (globaltimer_ns() - w0 > kLexWaitNs || ((++it & 63u) == 0u && *(volatile unsigned*)derr)) {
                            ok = 0;
                            break;
                        }
                        __nanosleep(32);
                    }
                }
                __syncwarp();  // carries lane 0's acquire to the warp
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) break;
            }
            const int k = t - lane;  // this lane's column index in sweep order
            const bool active = k >= 0 && k < (int)N;
            if (t == 0 || k == 0) {
                if (active) lex_load<T, FWD>(cur, pq, uv, N, r, rprev, rnext, k, lane);
            } else if (active) {
                cur = nxt;
            }
            if (k + 1 >= 0 && k + 1 < (int)N && k + 1 > 0)
                lex_load<T, FWD>(nxt, pq, uv, N, r, rprev, rnext, k + 1, lane);
            // the point updated by lane - 1 at step t - 1 (row rprev, this column)
            const T sP = __shfl_up_sync(0xffffffffu, cP, 1);
            const T sQ = __shfl_up_sync(0xffffffffu, cQ, 1);
            const T sU = __shfl_up_sync(0xffffffffu, cU, 1);
            if (active) {
                const T pP = lane == 0 ? cur.pr.x : sP, pQ = lane == 0 ? cur.pr.y : sQ, pU = lane == 0 ? cur.prU : sU;
                const T lP = k == 0 ? cur.pc.x : cP, lQ = k == 0 ? cur.pc.y : cQ, lU = k == 0 ? cur.pcU : cU;
                // the neighbours in level_point's order: axis 0 lower, upper; axis 1 lower, upper
                T p[4], q[4], w[4];
                p[0] = FWD ? pP : cur.nr.x;
                q[0] = FWD ? pQ : cur.nr.y;
                w[0] = FWD ? pU : cur.nrU;
                p[1] = FWD ? cur.nr.x : pP;
                q[1] = FWD ? cur.nr.y : pQ;
                w[1] = FWD ? cur.nrU : pU;
                p[2] = FWD ? lP : cur.nc.x;
                q[2] = FWD ? lQ : cur.nc.y;
                w[2] = FWD ? lU : cur.ncU;
                p[3] = FWD ? cur.nc.x : lP;
                q[3] = FWD ? cur.nc.y : lQ;
                w[3] = FWD ? cur.ncU : lU;
                vec2_t<T> a = cur.a, e = cur.e;
                update_point<T, 2, MODE>(c, nsum_scaled(p, c.beta), nsum_scaled(q, c.beta), nsum_scaled(w, c.Bp),
                                         a.x, a.y, e.x, e.y);
                const int64_t j = FWD ? k : N - 1 - k;
                pq[r * N + j] = a;
                uv[r * N + j] = e;
                cP = a.x;
                cQ = a.y;
                cU = e.x;
            }
            if ((t % kLexPublish) == kLexPublish - 1 || t == steps - 1) {
                __syncwarp();  // the warp's stores precede lane 0's release
                if (lane == 0)
                    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&progress[s]), "r"((unsigned)(t + 1))
                                 : "memory");
            }
        }
        if (!ok) {
            if (lane == 0) {
                *(volatile unsigned*)derr = 1u;
                *(volatile int*)err = 1;
            }
            break;
        }
    }
}

template <typename T, int MODE, bool FWD>
static int launch_lex_t(vec2_t<T>* pq, vec2_t<T>* uv, int64_t N, const Coef<T>& c, unsigned* sync, int* err,
                        int stall, cudaStream_t s)
{
    auto kern = lex_strip_kernel<T, MODE, FWD>;
    int dev = 0, sms = 148, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kLexStrip, 0) != cudaSuccess || per < 1) return -1;
    const int64_t ns = N / kLexStrip;
    const unsigned grid = (unsigned)std::min<int64_t>((int64_t)sms * per, ns);
    if (cudaMemsetAsync(sync, 0, (size_t)(2 + ns) * sizeof(unsigned), s) != cudaSuccess) return -1;
    Coef<T> cc = c;
    int64_t n = N;
    void* args[] = {&pq, &uv, &n, &cc, &sync, &err, &stall};
    if (cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(kLexStrip), args, 0, s) != cudaSuccess)
        return -1;
    return 1;
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
    cudaError_t e = cudaSuccess;
#define KGS_LEVEL_M(DD, SP, MM) e = launch_level_pdl<T, DD, MM, SP>(blocks, threads, s, pq, uv, list, count, N, c, small);
#define KGS_LEVEL_S(DD, SP)                                   \
    switch (mode) {                                           \
    case RED_BASE: KGS_LEVEL_M(DD, SP, RED_BASE) break;       \
    case RED_ADJ: KGS_LEVEL_M(DD, SP, RED_ADJ) break;         \
    case PSI_HALF: KGS_LEVEL_M(DD, SP, PSI_HALF) break;       \
    default: KGS_LEVEL_M(DD, SP, UV_HALF) break;              \
    }
#define KGS_LEVEL(DD)                 \
    if (split) { KGS_LEVEL_S(DD, true) } \
    else { KGS_LEVEL_S(DD, false) }
    if (dim == 1) { KGS_LEVEL(1) }
    else if (dim == 2) { KGS_LEVEL(2) }
    else { KGS_LEVEL(3) }
#undef KGS_LEVEL
#undef KGS_LEVEL_S
#undef KGS_LEVEL_M
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

bool lex_sweep_applies(int dim, int64_t N)
{
    return dim == 2 && N >= 2 * kLexStrip && N % kLexStrip == 0 && N <= 65534;
}

template <typename T>
int launch_lex_sweep(bool forward, int mode, vec2_t<T>* pq, vec2_t<T>* uv, int64_t N, const Coef<T>& c,
                     unsigned* sync, int* err, int stall, cudaStream_t s)
{
    const bool base = mode == RED_BASE;
    if (forward)
        return base ? launch_lex_t<T, RED_BASE, true>(pq, uv, N, c, sync, err, stall, s)
                    : launch_lex_t<T, RED_ADJ, true>(pq, uv, N, c, sync, err, stall, s);
    return base ? launch_lex_t<T, RED_BASE, false>(pq, uv, N, c, sync, err, stall, s)
                : launch_lex_t<T, RED_ADJ, false>(pq, uv, N, c, sync, err, stall, s);
}

template int launch_lex_sweep<double>(bool, int, vec2_t<double>*, vec2_t<double>*, int64_t, const Coef<double>&,
                                      unsigned*, int*, int, cudaStream_t);
template int launch_lex_sweep<float>(bool, int, vec2_t<float>*, vec2_t<float>*, int64_t, const Coef<float>&,
                                     unsigned*, int*, int, cudaStream_t);

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
