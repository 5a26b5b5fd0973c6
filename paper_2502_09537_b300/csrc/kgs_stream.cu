// kgs_stream.cu -- float32 3D DP-AVF2 step pairs streamed along axis 0:
// a step's black pass and red pass in one read and one write of the state.
//
// The checkerboard schedule of Algorithm 3, fused as in kgs_point.cuh, runs
// a step as (BLACK_FUSED, RED_FUSED) colour passes.  Two launches per step
// read the state twice and gather the other colour's values a third time
// (44 bytes per point-update in float32 against the 32 of one read and one
// write).  Here one launch applies both passes of a step while walking the
// grid plane by plane along axis 0: the black pass on plane i needs the red
// planes i-1, i, i+1 not yet updated, and the red pass on plane i-1 needs the
// black planes i-2, i-1, i updated -- both hold if the black pass runs one
// plane ahead of the red pass (Sec. 4.2: no point has a neighbour of its own
// colour, so each pass updates its plane's points in any order).
//
// Work: a tile is 29 x 64 points of the other two axes (29 rows along axis 1,
// 32 points of each colour along the last axis; the last tile of a grid has
// the rows that are left).  One CTA per SM takes work items of consecutive
// axis-0 planes of a tile (chunks: stream_auto_chunk, 256 planes at N = 512),
// round-robin in chunk-major order, so that CTAs on
// neighbouring tiles stream the same planes at about the same time and the
// halo rows they share come from L2 for the second.  For an item's planes
// [x0, x0 + L) it stages planes x0-2 .. x0+L+1 (mod N), updates black on
// x0-1 .. x0+L and red on x0 .. x0+L-1; the black values of the two outer
// planes are recomputed from the same inputs as their owner's, so bitwise the
// same.  Within a plane the black pass covers the tile and the ring of black
// points that the tile's red points read (two rows, and per row the one column
// beyond the tile on the side its red points' last-axis neighbours fall), which
// needs a two-point ring of red points: each staged plane is the tile plus a
// two-point halo, (29 + 4) x (32 + 4) points of each colour (rows beyond the
// grid, in a short last tile, are zero-filled by the load and never read).
// Warp t < 29 owns tile row t: each thread updates its black point of plane i,
// then the red point of plane i-1 at the same position, which reads black
// plane i only there -- the thread's own value; the other three warps update
// the ring, so every warp has at most two point updates per plane.
//
// Data: the state lives, for the launches of a kgs_step call, in a private
// packed layout: per colour (0-based coordinate-sum parity) and axis-0 plane,
// (N + 4) rows of (N/2 + 4) float4 (P, Q, U, V) -- the colour's points of a
// row in order, preceded and followed by two ghost copies of the row's
// periodic neighbours, and the plane's rows likewise preceded and followed by
// two ghost rows.  So a tile's staged box never wraps: one TMA tensor load
// (cp.async.bulk.tensor, 4D, no multicast) per plane fills a ring slot,
// completion signalled on the slot's mbarrier.  Launches read one buffer and
// write the other (ping-pong: other CTAs still read the old values of this
// CTA's halo), and whoever writes a point also writes its ghost copies.
// Conversions from and to the handle's colour-split layout run once per
// kgs_step call.
//
// Ring: six slots of 38 KB, four planes in use and two in flight; the load of
// staged plane j + 6 goes into the slot of plane j once the red pass of plane
// j + 1 is done with it, two plane iterations before it is needed, and
// planes further ahead are prefetched into L2 (KGS_OPT_STREAM_PREFETCH).  One
// CTA barrier per plane, after both passes, where the next plane's load is
// also awaited.  Every wait on an mbarrier is bounded (2 s of %globaltimer); a
// CTA whose wait runs out sets the error word, waits (bounded) for its loads
// in flight and leaves.
//
// Every point update is update_point (kgs_point.cuh) with the neighbour order
// of the one-launch-per-pass kernel, so the state is bitwise that of two pass
// launches per step.
#include <cuda.h>

#include <algorithm>
#include <cstring>

#include "kgs_internal.h"

namespace kgs {

KGS_BOUNDS_TU
KGS_BOUNDS_READER(bounds_flags_stream)

namespace {

constexpr int kTh = 32;                  // colour points per tile row (= warp lanes)
constexpr int kTy = 29;                  // tile rows (axis 1); the last tile of a grid may be shorter
constexpr int kRR = kTy + 4, kKK = kTh + 4;  // staged rows / columns per colour
constexpr int kSlotElems = 2 * kRR * kKK;    // float4 per staged plane
constexpr int kSlots = 6;
constexpr int kWarps = 32;               // warp t < kTy: tile row t; warps kTy .. kTy+2: the ring
constexpr int kThreads = 32 * kWarps;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr size_t kSmemBytes = (size_t)kSlots * kSlotElems * sizeof(float4) + (kSlots + 1) * sizeof(uint64_t);

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t clock_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait until the phase of bar with this parity has completed, at most kWaitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = clock_ns();
    while (!mbar_try_wait(bar, parity))
        if (clock_ns() - t0 > kWaitNs) return false;
    return true;
}

// One staged plane: the 4D box (4 kKK floats, kRR rows, 1 plane, 2 colours) at
// (c0 floats, c1 rows, plane c2, colour 0) of the packed buffer.
__device__ __forceinline__ void tma_load_plane(float4* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                               int c1, int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(0)
        : "memory");
}

// The same box into L2 only (no shared memory, no completion to wait for).
__device__ __forceinline__ void tma_prefetch_plane(const CUtensorMap* map, int c0, int c1, int c2)
{
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"(map), "r"(c0),
                 "r"(c1), "r"(c2), "r"(0)
                 : "memory");
}

// One point of colour `own_c` at staged (r, k) of plane slot `s` updated in
// shared memory (MODE BLACK_FUSED) or in registers (the red modes); dn / up
// are the slots of the axis-0 neighbour planes; zp = the point's last-axis
// parity, which places its two last-axis neighbours at columns k-1+zp, k+zp.
template <int MODE>
__device__ __forceinline__ float4 stream_point(const float4* s, const float4* dn, const float4* up, int own_c, int r,
                                               int k, int zp, const Coef<float>& c)
{
    const int oth = (own_c ^ 1) * kRR * kKK;
    const int at = r * kKK + k;
    if (!kgs_in_bounds(r >= 1 && r + 1 < kRR && k - 1 + zp >= 0 && k + zp < kKK && zp >= 0 && zp <= 1 &&
                           own_c >= 0 && own_c <= 1,
                       2u))
        return make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 n[6] = {dn[oth + at], up[oth + at], s[oth + at - kKK], s[oth + at + kKK],
                         s[oth + at - 1 + zp], s[oth + at + zp]};
    float p[6], q[6], w[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        p[m] = n[m].x;
        q[m] = n[m].y;
        w[m] = n[m].z;
    }
    float4 a = s[own_c * kRR * kKK + at];
    update_point<float, 3, MODE>(c, nsum_scaled(p, c.beta), nsum_scaled(q, c.beta), nsum_scaled(w, c.Bp), a.x, a.y,
                                 a.z, a.w);
    return a;
}

template <int REDMODE>
__global__ void __launch_bounds__(kThreads, 1)
    stream_kernel(const __grid_constant__ CUtensorMap src, float4* __restrict__ dst, int N, Coef<float> c, int* err,
                  int stall, int chunk, int pf)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4* slots = reinterpret_cast<float4*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)kSlots * kSlotElems * sizeof(float4));
    constexpr int cR = 0, cB = 1;  // 3D: red = even 0-based coordinate sum (red_parity(3) == 0)
    const int lane = threadIdx.x & 31, t = threadIdx.x >> 5;  // warp t: tile row t
    const int hN = N >> 1;
    const int tiles_z = hN / kTh, ntiles = ((N + kTy - 1) / kTy) * tiles_z;
    const int64_t cols = hN + 4, plane_elems = (int64_t)(N + 4) * cols;
    if (threadIdx.x == 0) {
        for (int s = 0; s <= kSlots; ++s) mbar_init(&bars[s], 1);  // bars[kSlots]: the stall test's
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;    // bit s: parity of slot s's next completion (same in every thread)
    uint32_t pending = 0;  // thread 0: slots with a load in flight
    int failed = 0;
    bool first = true;
    // This CTA's work, as segments (planes [x0, x0 + L) of one tile).  chunk = 0:
    // a contiguous share of the (tile, axis-0 plane) sequence, tile-major (one
    // or two segments per CTA).  chunk > 0: items of `chunk` planes taken
    // round-robin in chunk-major order, so that CTAs on neighbouring tiles
    // stream the same planes at about the same time and the halo rows they
    // share are read from L2 by the second.
    const int64_t W = (int64_t)ntiles * N;
    int64_t w0 = (int64_t)blockIdx.x * W / gridDim.x;
    const int64_t w1 = (int64_t)(blockIdx.x + 1) * W / gridDim.x;
    const int nchunks = chunk > 0 ? (N + chunk - 1) / chunk : 0;
    int64_t item = blockIdx.x;
    for (;;) {
        int tile, x0, L;
        if (chunk > 0) {
            if (item >= (int64_t)nchunks * ntiles || failed) break;
            tile = (int)(item % ntiles);
            x0 = (int)(item / ntiles) * chunk;
            L = N - x0 < chunk ? N - x0 : chunk;
            item += gridDim.x;
        } else {
            if (w0 >= w1 || failed) break;
            tile = (int)(w0 / N);
            x0 = (int)(w0 % N);
            L = (int)((w1 - w0) < (int64_t)(N - x0) ? (w1 - w0) : (int64_t)(N - x0));
            w0 += L;
        }
        const int y0 = (tile / tiles_z) * kTy, zh0 = (tile % tiles_z) * kTh;
        const int ty = N - y0 < kTy ? N - y0 : kTy;  // the tile's rows
        const int yp = y0 & 1;  // staged row r is axis-1 coordinate y0 - 2 + r, of parity yp ^ (r & 1)
        // staged plane j (0 .. L + 3) is axis-0 plane x0 - 2 + j mod N, in slot j % kSlots
        auto coords = [&](int j) {
            int p = x0 - 2 + j;
            return p < 0 ? p + N : (p >= N ? p - N : p);
        };
        auto issue = [&](int j) {
            const int s = j % kSlots;
            mbar_expect_tx(&bars[s], (unsigned)(kSlotElems * sizeof(float4)));
            tma_load_plane(slots + s * kSlotElems, &src, &bars[s], 4 * zh0, y0, coords(j));
            pending |= 1u << s;
        };
        auto prefetch = [&](int j) { tma_prefetch_plane(&src, 4 * zh0, y0, coords(j)); };
        auto wait = [&](int j) -> bool {
            const int s = j % kSlots;
            const bool ok = mbar_wait_bounded(&bars[s], (phase >> s) & 1u);
            if (ok) {
                phase ^= 1u << s;
                if (threadIdx.x == 0) pending &= ~(1u << s);
            }
            return ok;
        };
        // this thread's red point (tile row t, colour column lane) in the packed
        // output: its offset in a plane and those of its ghost copies (-1: none)
        const int y = y0 + (t < ty ? t : 0), zh = zh0 + lane;  // rows t >= ty have no point
        const int pr2 = y < 2 ? y + N + 2 : (y >= N - 2 ? y - N + 2 : -1);
        const int pc2 = zh < 2 ? zh + hN + 2 : (zh >= hN - 2 ? zh - hN + 2 : -1);
        const int64_t off0 = (int64_t)(y + 2) * cols + zh + 2;
        const int64_t offr = pr2 >= 0 ? (int64_t)pr2 * cols + zh + 2 : -1;
        const int64_t offc = pc2 >= 0 ? (int64_t)(y + 2) * cols + pc2 : -1;
        const int64_t offrc = (pr2 >= 0 && pc2 >= 0) ? (int64_t)pr2 * cols + pc2 : -1;
        auto store = [&](int col, int x, float4 v) {
            float4* pl = dst + ((int64_t)col * N + x) * plane_elems;
            if (!kgs_in_bounds(x >= 0 && x < N && off0 < plane_elems && offr < plane_elems && offc < plane_elems &&
                                   offrc < plane_elems,
                               4u))
                return;
            pl[off0] = v;
            if (offr >= 0) pl[offr] = v;
            if (offc >= 0) pl[offc] = v;
            if (offrc >= 0) pl[offrc] = v;
        };
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int j = 0; j < kSlots - 1 && j <= L + 3; ++j) issue(j);
            for (int j = kSlots - 1; j < kSlots - 1 + pf && j <= L + 3; ++j) prefetch(j);
        }
        int bad = 0;
        for (int j = 0; j < 3; ++j) bad |= !wait(j);
        failed = __syncthreads_or(bad);
        const int r = 2 + t, k = 2 + lane;
        for (int it = 0; it <= L + 1 && !failed; ++it) {
            const int cb = x0 - 1 + it;  // black plane; red plane cb - 1
            // black pass on plane cb (staged j = it + 1), red neighbours in j = it, it + 2:
            // this thread's interior point (r, k)
            const float4* sb = slots + ((it + 1) % kSlots) * kSlotElems;
            const float4* sbd = slots + (it % kSlots) * kSlotElems;
            const float4* sbu = slots + ((it + 2) % kSlots) * kSlotElems;
            float4* wb = const_cast<float4*>(sb) + cB * kRR * kKK;
            if (t < ty) wb[r * kKK + k] = stream_point<BLACK_FUSED>(sb, sbd, sbu, cB, r, k, (cB ^ cb ^ yp ^ r) & 1, c);
            // red pass on plane cb - 1 (staged j = it), black neighbours in j = it - 1, it + 1:
            // its point (r, k) needs black (cb) only at (r, k), just written by this thread
            if (it >= 2 && t < ty) {
                const int x = cb - 1;
                const float4* sr = slots + (it % kSlots) * kSlotElems;
                const float4* srd = slots + ((it + kSlots - 1) % kSlots) * kSlotElems;
                const float4 a = stream_point<REDMODE>(sr, srd, sb, cR, r, k, (cR ^ x ^ yp ^ r) & 1, c);
                store(cR, x, a);
                store(cB, x, sr[cB * kRR * kKK + r * kKK + k]);
            }
            // the ring of black points of plane cb that the red pass of plane cb
            // reads (next iteration): rows 1 and ty + 2, and per row the one
            // column beyond the tile on the side its red points' last-axis
            // neighbours fall -- by the three warps that own no tile row
            if (t >= kTy && (t < kTy + 2 || lane < ty)) {
                int rr, kk;
                if (t < kTy + 2) {
                    rr = t == kTy ? 1 : ty + 2;
                    kk = 2 + lane;
                } else {
                    rr = 2 + lane;
                    kk = ((cb ^ yp ^ rr) & 1) ? kTh + 2 : 1;
                }
                wb[rr * kKK + kk] = stream_point<BLACK_FUSED>(sb, sbd, sbu, cB, rr, kk, (cB ^ cb ^ yp ^ rr) & 1, c);
            }
            // the next black pass needs staged plane it + 3 (its upper neighbours)
            bad = 0;
            if (stall && first && it == 1) bad = !mbar_wait_bounded(&bars[kSlots], 0);  // never completes
            if (!bad && it + 3 <= L + 3) bad = !wait(it + 3);
            failed = __syncthreads_or(bad);
            // staged plane it - 1 is no longer read: load plane it - 1 + kSlots into its
            // slot, and prefetch the plane pf beyond it into L2
            if (!failed && threadIdx.x == 0) {
                if (it + kSlots - 1 <= L + 3) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue(it + kSlots - 1);
                }
                if (pf > 0 && it + kSlots - 1 + pf <= L + 3) prefetch(it + kSlots - 1 + pf);
            }
        }
        first = false;
    }
    if (failed && threadIdx.x == 0) {
        *(volatile int*)err = 2;
        // loads still in flight write this CTA's shared memory: wait (bounded) for them
        for (int s = 0; s < kSlots; ++s)
            if (pending & (1u << s)) mbar_wait_bounded(&bars[s], (phase >> s) & 1u);
    }
}

// Whole-state conversions between the colour-split layout (P,Q vec2 array;
// U then V planar) and the packed layout with ghost copies.
__global__ void to_packed_kernel(const float2* __restrict__ pq, const float* __restrict__ uv, float4* __restrict__ out,
                                 int N)
{
    const int hN = N >> 1;
    const int64_t cols = hN + 4, rows = N + 4;
    const int64_t total = 2 * (int64_t)N * rows * cols;
    const int64_t M = (int64_t)N * N * N, half = M >> 1;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int pc = (int)(e % cols);
        int64_t t = e / cols;
        const int pr = (int)(t % rows);
        t /= rows;
        const int x = (int)(t % N), col = (int)(t / N);
        int y = pr - 2, zh = pc - 2;
        y = y < 0 ? y + N : (y >= N ? y - N : y);
        zh = zh < 0 ? zh + hN : (zh >= hN ? zh - hN : zh);
        const int64_t pos = (col ? half : 0) + ((int64_t)x * N + y) * hN + zh;
        const float2 a = pq[pos];
        out[e] = make_float4(a.x, a.y, uv[pos], uv[M + pos]);
    }
}

__global__ void from_packed_kernel(const float4* __restrict__ in, float2* __restrict__ pq, float* __restrict__ uv,
                                   int N)
{
    const int hN = N >> 1;
    const int64_t cols = hN + 4, rows = N + 4;
    const int64_t M = (int64_t)N * N * N, half = M >> 1;
    for (int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pos < M; pos += (int64_t)gridDim.x * blockDim.x) {
        const int col = pos >= half;
        const int64_t q = pos - (col ? half : 0);
        const int zh = (int)(q % hN);
        const int64_t t = q / hN;
        const int y = (int)(t % N), x = (int)(t / N);
        const float4 v = in[(((int64_t)col * N + x) * rows + y + 2) * cols + zh + 2];
        pq[pos] = make_float2(v.x, v.y);
        uv[pos] = v.z;
        uv[M + pos] = v.w;
    }
}

unsigned conv_grid(int64_t n)
{
    return (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)148 * 16);
}

}  // namespace

bool stream_applies(int dim, int64_t N, int precision)
{
    return dim == 3 && precision == 32 && N >= 64 && N <= 1024 && N % 64 == 0;
}

int stream_auto_chunk(int64_t N, int sms)
{
    // the fewest chunks per tile column (at least two: a column alone measured
    // slower) whose items fill at least 95% of the rounds of `sms` CTAs, else
    // the best filling; measured at 512^3 (144 tiles): 256-plane chunks 0.750
    // of HBM, 171: 0.746, 128: 0.744, 512: 0.739, 64: 0.730
    const int64_t ntiles = ((N + kTy - 1) / kTy) * (N / 2 / kTh);
    int best = (int)N;
    double best_fill = 0.0;
    for (int64_t nc = 2; nc <= N / 16; ++nc) {
        const int64_t chunk = (N + nc - 1) / nc;
        const int64_t items = ntiles * ((N + chunk - 1) / chunk);
        const int64_t rounds = (items + sms - 1) / sms;
        const double fill = (double)items / (double)(rounds * sms);
        if (fill > best_fill + 1e-9) {
            best_fill = fill;
            best = (int)chunk;
        }
        if (fill >= 0.95) return (int)chunk;
    }
    return best;
}

size_t stream_buffer_bytes(int64_t N)
{
    return (size_t)2 * N * (N + 4) * (N / 2 + 4) * sizeof(float4);
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int stream_make_map(void* buf, int64_t N, void* map_out)
{
    static EncodeTiled encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return -1;
        encode = reinterpret_cast<EncodeTiled>(fn);
    }
    const int64_t hN = N / 2;
    // dims, innermost first: the floats of a padded row, rows, planes, colours
    const cuuint64_t dims[4] = {(cuuint64_t)(4 * (hN + 4)), (cuuint64_t)(N + 4), (cuuint64_t)N, 2};
    const cuuint64_t row = (cuuint64_t)(hN + 4) * sizeof(float4);
    const cuuint64_t strides[3] = {row, row * (cuuint64_t)(N + 4), row * (cuuint64_t)(N + 4) * (cuuint64_t)N};
    const cuuint32_t box[4] = {4 * kKK, kRR, 1, 2};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    // a staged row is 4 kKK floats = 576 bytes = 9 x 64: L2 promotion to 64-byte
    // lines fetches exactly the row (256-byte promotion read 768 bytes per row,
    // measured: 1.54x the algorithmic DRAM reads per launch at 512^3)
    CUresult r = encode(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, buf, dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_64B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

int launch_stream(const void* map, void* dst, int64_t N, const Coef<float>& c, int red_mode, int* err, int stall,
                  int chunk, int prefetch, cudaStream_t s)
{
    static bool attr_set[2] = {false, false};
    auto kern = red_mode == RED_ADJ ? stream_kernel<RED_ADJ> : stream_kernel<RED_FUSED>;
    const int which = red_mode == RED_ADJ ? 1 : 0;
    if (!attr_set[which]) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) != cudaSuccess)
            return -1;
        attr_set[which] = true;
    }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ntiles = ((N + kTy - 1) / kTy) * (N / 2 / kTh);
    const int64_t items = chunk > 0 ? ntiles * ((N + chunk - 1) / chunk) : ntiles * N;
    const unsigned grid = (unsigned)std::min<int64_t>(items, sms);
    CUtensorMap m;
    memcpy(&m, map, sizeof m);
    kern<<<grid, kThreads, kSmemBytes, s>>>(m, reinterpret_cast<float4*>(dst), (int)N, c, err, stall, chunk,
                                            prefetch);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_to_packed(const void* pq, const void* uv, void* out, int64_t N, cudaStream_t s)
{
    const int64_t total = 2 * N * (N + 4) * (N / 2 + 4);
    to_packed_kernel<<<conv_grid(total), 256, 0, s>>>(reinterpret_cast<const float2*>(pq),
                                                       reinterpret_cast<const float*>(uv),
                                                       reinterpret_cast<float4*>(out), (int)N);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_from_packed(const void* in, void* pq, void* uv, int64_t N, cudaStream_t s)
{
    from_packed_kernel<<<conv_grid(N * N * N), 256, 0, s>>>(reinterpret_cast<const float4*>(in),
                                                             reinterpret_cast<float2*>(pq),
                                                             reinterpret_cast<float*>(uv), (int)N);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace kgs
