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
// (N + 8) rows of (N/2 + 4) float4 (P, Q, U, V) -- the colour's points of a
// row in order, preceded and followed by two ghost copies of the row's
// periodic neighbours, and the plane's rows likewise preceded and followed by
// four ghost rows (the two-step kernel below stages a four-row halo).  So a
// tile's staged box never wraps: one TMA tensor load
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
#include <type_traits>
#include <vector>

#include "kgs_internal.h"

namespace kgs {

KGS_BOUNDS_TU
KGS_BOUNDS_READER(bounds_flags_stream)

namespace {

constexpr int kG = 4;                    // ghost rows on each side of a packed plane
constexpr int kTh = 32;                  // colour points per tile row (= warp lanes)
constexpr int kTy = 29;                  // tile rows (axis 1); the last tile of a grid may be shorter
constexpr int kRR = kTy + 4, kKK = kTh + 4;  // staged rows / columns per colour
constexpr int kSlotElems = 2 * kRR * kKK;    // float4 per staged plane
constexpr int kSlots = 6;
constexpr int kWarps = 32;               // warp t < kTy: tile row t; warps kTy .. kTy+2: the ring
constexpr int kThreads = 32 * kWarps;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr size_t kSmemBytes = (size_t)kSlots * kSlotElems * sizeof(float4) + (kSlots + 1) * sizeof(uint64_t);
static_assert(kSlotElems * sizeof(float4) % 128 == 0, "one-step kernel: TMA slots 128-byte aligned");

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

// One point of colour `own_c` at staged (r, k) of plane slot `s` (RR staged
// rows) updated in registers; ndn / nup are its axis-0 neighbours (the other
// colour at the same staged position in the planes below and above); zp = the
// point's last-axis parity, which places its two last-axis neighbours at
// columns k-1+zp, k+zp.
template <int MODE, int RR, int KK = kKK>
__device__ __forceinline__ float4 stream_point_v(const float4* s, float4 ndn, float4 nup, int own_c, int r, int k,
                                                 int zp, const Coef<float>& c)
{
    const int oth = (own_c ^ 1) * RR * KK;
    const int at = r * KK + k;
    if (!kgs_in_bounds(r >= 1 && r + 1 < RR && k - 1 + zp >= 0 && k + zp < KK && zp >= 0 && zp <= 1 &&
                           own_c >= 0 && own_c <= 1,
                       2u))
        return make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 n[6] = {ndn, nup, s[oth + at - KK], s[oth + at + KK], s[oth + at - 1 + zp], s[oth + at + zp]};
    float p[6], q[6], w[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        p[m] = n[m].x;
        q[m] = n[m].y;
        w[m] = n[m].z;
    }
    float4 a = s[own_c * RR * KK + at];
    update_point<float, 3, MODE>(c, nsum_scaled(p, c.beta), nsum_scaled(q, c.beta), nsum_scaled(w, c.Bp), a.x, a.y,
                                 a.z, a.w);
    return a;
}

// The same with the axis-0 neighbours read from the slots dn / up.
template <int MODE, int RR = kRR, int KK = kKK>
__device__ __forceinline__ float4 stream_point(const float4* s, const float4* dn, const float4* up, int own_c, int r,
                                               int k, int zp, const Coef<float>& c)
{
    const int oth = (own_c ^ 1) * RR * KK;
    const int at = r * KK + k;
    if (!kgs_in_bounds(r >= 0 && r < RR && k >= 0 && k < KK && own_c >= 0 && own_c <= 1, 2u))
        return make_float4(0.f, 0.f, 0.f, 0.f);
    return stream_point_v<MODE, RR, KK>(s, dn[oth + at], up[oth + at], own_c, r, k, zp, c);
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
    const int64_t cols = hN + 4, plane_elems = (int64_t)(N + 2 * kG) * cols;
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
            tma_load_plane(slots + s * kSlotElems, &src, &bars[s], 4 * zh0, y0 - 2 + kG, coords(j));
            pending |= 1u << s;
        };
        auto prefetch = [&](int j) { tma_prefetch_plane(&src, 4 * zh0, y0 - 2 + kG, coords(j)); };
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
        const int pr2 = y < kG ? y + N + kG : (y >= N - kG ? y - N + kG : -1);
        const int pc2 = zh < 2 ? zh + hN + 2 : (zh >= hN - 2 ? zh - hN + 2 : -1);
        const int64_t off0 = (int64_t)(y + kG) * cols + zh + 2;
        const int64_t offr = pr2 >= 0 ? (int64_t)pr2 * cols + zh + 2 : -1;
        const int64_t offc = pc2 >= 0 ? (int64_t)(y + kG) * cols + pc2 : -1;
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int j = 0; j < kSlots - 1 && j <= L + 3; ++j) issue(j);
            for (int j = kSlots - 1; j < kSlots - 1 + pf && j <= L + 3; ++j) prefetch(j);
        }
        int bad = 0;
        for (int j = 0; j < 3; ++j) bad |= !wait(j);
        failed = __syncthreads_or(bad);
        const int r = 2 + t, k = 2 + lane;
        // output offsets of this thread's point at the red pass's plane (x0 - 2 +
        // it), advanced one plane per iteration, and its ghost copies' offsets
        // relative to them
        int64_t oR_out = ((int64_t)cR * N + x0 - 2) * plane_elems + off0;
        int64_t oB_out = ((int64_t)cB * N + x0 - 2) * plane_elems + off0;
        const int dgr = offr >= 0 ? (int)(offr - off0) : 0, dgc = offc >= 0 ? (int)(offc - off0) : 0;
        const bool ghost = offr >= 0 || offc >= 0;
        auto put = [&](int64_t o, float4 v) {
            const int64_t end = 2 * (int64_t)N * plane_elems;
            if (!kgs_in_bounds(o >= 0 && o < end && o + dgr >= 0 && o + dgr < end && o + dgc >= 0 &&
                                   o + dgc < end && o + dgr + dgc >= 0 && o + dgr + dgc < end,
                               4u))
                return;
            dst[o] = v;
            if (ghost) {
                if (dgr) dst[o + dgr] = v;
                if (dgc) dst[o + dgc] = v;
                if (dgr && dgc) dst[o + dgr + dgc] = v;
            }
        };
        // one iteration; s0 = it % kSlots as a compile-time constant (the loop
        // below is unrolled six times), so every slot address is fixed
        auto body = [&](auto s0c, int it) {
            constexpr int s0 = decltype(s0c)::value;
            constexpr int jm1 = (s0 + kSlots - 1) % kSlots, jp1 = (s0 + 1) % kSlots, jp2 = (s0 + 2) % kSlots,
                          jp3 = (s0 + 3) % kSlots;
            const int cb = x0 - 1 + it;  // black plane; red plane cb - 1
            // black pass on plane cb (staged j = it + 1), red neighbours in j = it, it + 2:
            // this thread's interior point (r, k)
            const float4* sb = slots + jp1 * kSlotElems;
            const float4* sbd = slots + s0 * kSlotElems;
            const float4* sbu = slots + jp2 * kSlotElems;
            float4* wb = const_cast<float4*>(sb) + cB * kRR * kKK;
            if (t < ty) wb[r * kKK + k] = stream_point<BLACK_FUSED>(sb, sbd, sbu, cB, r, k, (cB ^ cb ^ yp ^ r) & 1, c);
            // red pass on plane cb - 1 (staged j = it), black neighbours in j = it - 1, it + 1:
            // its point (r, k) needs black (cb) only at (r, k), just written by this thread
            if (it >= 2 && t < ty) {
                const int x = cb - 1;
                const float4* sr = slots + s0 * kSlotElems;
                const float4* srd = slots + jm1 * kSlotElems;
                put(oR_out, stream_point<REDMODE>(sr, srd, sb, cR, r, k, (cR ^ x ^ yp ^ r) & 1, c));
                put(oB_out, sr[cB * kRR * kKK + r * kKK + k]);
            }
            oR_out += plane_elems;
            oB_out += plane_elems;
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
            if (!bad && it + 3 <= L + 3) {
                const bool ok = mbar_wait_bounded(&bars[jp3], (phase >> jp3) & 1u);
                if (ok) {
                    phase ^= 1u << jp3;
                    if (threadIdx.x == 0) pending &= ~(1u << jp3);
                }
                bad = !ok;
            }
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
        };
        for (int it = 0; it <= L + 1 && !failed;) {
            body(std::integral_constant<int, 0>{}, it);
            if (++it > L + 1 || failed) break;
            body(std::integral_constant<int, 1>{}, it);
            if (++it > L + 1 || failed) break;
            body(std::integral_constant<int, 2>{}, it);
            if (++it > L + 1 || failed) break;
            body(std::integral_constant<int, 3>{}, it);
            if (++it > L + 1 || failed) break;
            body(std::integral_constant<int, 4>{}, it);
            if (++it > L + 1 || failed) break;
            body(std::integral_constant<int, 5>{}, it);
            ++it;
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

// ---------------------------------------------------------------------------
// Two steps per launch (temporal depth 2).
//
// The same walk along axis 0 with a step pair's four colour passes chained
// plane by plane: at iteration `it` of a work item the first black pass (B1)
// updates plane a, the first red pass (R1) plane a - 1, the second black
// pass (B2) plane a - 2 and the second red pass (R2) plane a - 3.  Each pass
// needs the previous one's values on its plane and the planes on either side,
// which the lag of one plane provides.  Within a plane each pass is needed on
// a region one point wider than the next pass's (R2 on the tile, B2 on the
// tile and the ring its red points read, and so on), so a staged plane is the
// tile with a four-row halo above and below; along the last axis two colour
// columns on each side suffice, because every half step widens the region on
// one side of a row only, the side alternating with the row's parity.
//
// Every pass writes its values into the staged planes in place.  At one
// position the four passes of an iteration touch the planes in the order B1
// (writes black a, reads red a - 1 there), R1 (writes red a - 1, reads black
// a - 2 there), B2 (writes black a - 2, reads red a - 3 there), R2: one thread
// owns each position for the whole iteration and runs them in that order.
// Reads of other positions within an iteration go to planes no pass of the
// iteration writes (B1 reads red a, R1 black a - 1, B2 red a - 2, R2 black
// a - 3), so one CTA barrier per plane still suffices.
//
// Threads: warp w < kTy2 + 6 owns tile row w - 3 over the tile's 32 columns
// (rows -3 .. ty + 2 take B1, -2 .. ty + 1 also R1, -1 .. ty also B2, the
// tile rows also R2); the other three warps take the points beyond those
// columns, from a host-built list per tile height and plane parity
// (stream2_prepare), the points with the most passes first so that threads
// with the same passes share a warp.
//
// Slots: staged plane j (axis-0 plane x0 - 4 + j) in slot j % 6.  At
// iteration it the passes read slots it - 2 .. it + 2: R2 takes the B2
// values of plane a - 4 at its own position from the registers of the thread
// that computed them two iterations before, so the slot of staged plane it - 3
// is free at the start of the iteration and takes the load of plane it + 3,
// awaited at the iteration's end.  Final values go to the packed output as
// they are made: black at B2, red at R2.
constexpr int kTy2 = 23;                             // tile rows
constexpr int kRR2 = kTy2 + 8;                       // staged rows
constexpr int kKK2 = kKK + 1;                        // staged row pitch, 37 float4: see stream_make_map
constexpr int kSlotElems2 = 2 * kRR2 * kKK2;         // float4 per staged plane
constexpr int kSlotStride2 = (kSlotElems2 + 7) / 8 * 8;  // slots 128-byte aligned (a TMA destination must be)
constexpr int kSlots2 = 6;
constexpr int kMainWarps2 = kTy2 + 6;                // warp w: tile row w - 3
constexpr int kSide2 = 32 * (kWarps - kMainWarps2);  // threads for the points beyond the tile's columns
constexpr size_t kSmemBytes2 = (size_t)kSlots2 * kSlotStride2 * sizeof(float4) + (kSlots2 + 1) * sizeof(uint64_t);
static_assert(kSlotStride2 * sizeof(float4) % 128 == 0, "two-step kernel: TMA slots 128-byte aligned");
static_assert(kSmemBytes2 <= 232448, "two-step kernel: shared memory");
static_assert(kRR2 <= 32, "two-step kernel: staged rows are five bits in the side list");

// The points beyond the tile's 32 columns, per tile kind (0: kTy2 rows, 1:
// the grid's last, shorter tile row) and parity q = (B1's plane + the tile's
// first row) & 1: staged row | staged column << 5 | (passes - 1) << 11 |
// 0x8000, the points with more passes first; n: how many.
struct Side2 {
    uint16_t pos[2][2][kSide2];
    uint16_t n[2][2];
};

template <int REDMODE>
__global__ void __launch_bounds__(kThreads, 1)
    stream2_kernel(const __grid_constant__ CUtensorMap src, float4* __restrict__ dst, int N, Coef<float> c,
                   const __grid_constant__ Side2 side, int* err, int stall, int chunk, int pf)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4* slots = reinterpret_cast<float4*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)kSlots2 * kSlotStride2 * sizeof(float4));
    constexpr int cR = 0, cB = 1;  // 3D: red = even 0-based coordinate sum
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool is_main = w < kMainWarps2;
    const int sidx = (int)threadIdx.x - 32 * kMainWarps2;  // side threads: list index
    const int hN = N >> 1;
    const int tiles_z = hN / kTh, ntiles = ((N + kTy2 - 1) / kTy2) * tiles_z;
    const int64_t cols = hN + 4, plane_elems = (int64_t)(N + 2 * kG) * cols;
    if (threadIdx.x == 0) {
        for (int s = 0; s <= kSlots2; ++s) mbar_init(&bars[s], 1);  // bars[kSlots2]: the stall test's
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;    // bit s: parity of slot s's next completion (same in every thread)
    uint32_t pending = 0;  // thread 0: slots with a load in flight
    int failed = 0;
    bool first = true;
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
        const int y0 = (tile / tiles_z) * kTy2, zh0 = (tile % tiles_z) * kTh;
        const int ty = N - y0 < kTy2 ? N - y0 : kTy2;
        const int kind = ty == kTy2 ? 0 : 1;
        const int yp = y0 & 1;  // staged row r is axis-1 coordinate y0 - 4 + r, of parity yp ^ (r & 1)
        // staged plane j (0 .. L + 7) is axis-0 plane x0 - 4 + j mod N, in slot j % kSlots2
        auto coords = [&](int j) {
            int p = x0 - 4 + j;
            return p < 0 ? p + N : (p >= N ? p - N : p);
        };
        auto issue = [&](int j) {
            const int s = j % kSlots2;
            mbar_expect_tx(&bars[s], (unsigned)(kSlotElems2 * sizeof(float4)));
            tma_load_plane(slots + s * kSlotStride2, &src, &bars[s], 4 * zh0, y0 - 4 + kG, coords(j));
            pending |= 1u << s;
        };
        auto prefetch = [&](int j) { tma_prefetch_plane(&src, 4 * zh0, y0 - 4 + kG, coords(j)); };
        auto wait = [&](int j) -> bool {
            const int s = j % kSlots2;
            const bool ok = mbar_wait_bounded(&bars[s], (phase >> s) & 1u);
            if (ok) {
                phase ^= 1u << s;
                if (threadIdx.x == 0) pending &= ~(1u << s);
            }
            return ok;
        };
        // main threads: tile row w - 3 (staged row w + 1), colour column lane
        // (staged lane + 2), and how many of the four passes the row takes
        const int row = w - 3;
        const int dmain = !is_main || row > ty + 2
                              ? 0
                              : 1 + (row >= -2 && row <= ty + 1) + (row >= -1 && row <= ty) + (row >= 0 && row < ty);
        // side threads: their list entries for the two parities
        const uint32_t sp0 = !is_main && sidx < side.n[kind][0] ? side.pos[kind][0][sidx] : 0u;
        const uint32_t sp1 = !is_main && sidx < side.n[kind][1] ? side.pos[kind][1][sidx] : 0u;
        // a tile point's offset in a packed plane and those of its ghost copies (-1: none)
        const bool in_t = dmain == 4;
        const int y = y0 + (in_t ? row : 0), zh = zh0 + lane;
        const int pr2 = y < kG ? y + N + kG : (y >= N - kG ? y - N + kG : -1);
        const int pc2 = zh < 2 ? zh + hN + 2 : (zh >= hN - 2 ? zh - hN + 2 : -1);
        const int64_t off0 = (int64_t)(y + kG) * cols + zh + 2;
        const int64_t offr = pr2 >= 0 ? (int64_t)pr2 * cols + zh + 2 : -1;
        const int64_t offc = pc2 >= 0 ? (int64_t)(y + kG) * cols + pc2 : -1;
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int j = 0; j < kSlots2 && j <= L + 7; ++j) issue(j);
            for (int j = kSlots2; j < kSlots2 + pf && j <= L + 7; ++j) prefetch(j);
        }
        int bad = 0;
        for (int j = 0; j < 3; ++j) bad |= !wait(j);
        failed = __syncthreads_or(bad);
        float4 hA = make_float4(0.f, 0.f, 0.f, 0.f), hB = hA;  // this position's B2 values, one and two iterations back
        // output offsets of a tile point at B2's and R2's planes, advanced one
        // plane per iteration (B2 on plane x0 - 5 + it, R2 on x0 - 6 + it), and
        // its ghost copies' offsets relative to them
        int64_t oB = ((int64_t)cB * N + x0 - 5) * plane_elems + off0;
        int64_t oR = ((int64_t)cR * N + x0 - 6) * plane_elems + off0;
        const int dgr = offr >= 0 ? (int)(offr - off0) : 0, dgc = offc >= 0 ? (int)(offc - off0) : 0;
        const bool ghost = offr >= 0 || offc >= 0;
        auto put = [&](int64_t o, float4 v) {
            const int64_t end = 2 * (int64_t)N * plane_elems;
            if (!kgs_in_bounds(o >= 0 && o < end && o + dgr >= 0 && o + dgr < end && o + dgc >= 0 &&
                                   o + dgc < end && o + dgr + dgc >= 0 && o + dgr + dgc < end,
                               4u))
                return;
            dst[o] = v;
            if (ghost) {
                if (dgr) dst[o + dgr] = v;
                if (dgc) dst[o + dgc] = v;
                if (dgr && dgc) dst[o + dgr + dgc] = v;
            }
        };
        // one iteration; s0 = it % kSlots2 as a compile-time constant (the loop
        // below is unrolled six times), so every slot address is fixed
        auto body = [&](auto s0c, int it) {
            constexpr int s0 = decltype(s0c)::value;
            constexpr int jm2 = (s0 + 4) % kSlots2, jm1 = (s0 + 5) % kSlots2, jp1 = (s0 + 1) % kSlots2,
                          jp2 = (s0 + 2) % kSlots2, jp3 = (s0 + 3) % kSlots2;
            // the slot of staged plane it - 3 is read no more: load plane it + 3 into it
            if (it >= 3 && threadIdx.x == 0) {
                if (it + 3 <= L + 7) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue(it + 3);
                }
                if (pf > 0 && it + 3 + pf <= L + 7) prefetch(it + 3 + pf);
            }
            const int a = x0 - 3 + it;  // B1's plane (only its parity matters here)
            const int ap = a & 1;
            int sr, sc, d;
            if (is_main) {
                sr = w + 1;
                sc = lane + 2;
                d = dmain;
            } else {
                const uint32_t e = (ap ^ yp) & 1 ? sp1 : sp0;
                sr = (int)(e & 31u);
                sc = (int)((e >> 5) & 63u);
                d = (e & 0x8000u) ? (int)((e >> 11) & 3u) + 1 : 0;
            }
            float4* Sm2 = slots + jm2 * kSlotStride2;       // staged it - 2: R2's plane
            float4* Sm1 = slots + jm1 * kSlotStride2;       // staged it - 1: B2's
            float4* Sz = slots + s0 * kSlotStride2;         // staged it: R1's
            float4* Sp1 = slots + jp1 * kSlotStride2;       // staged it + 1: B1's
            const float4* Sp2 = slots + jp2 * kSlotStride2;
            const int at = sr * kKK2 + sc;
            if (d >= 1)  // B1, plane a: red neighbours of the input state
                Sp1[cB * kRR2 * kKK2 + at] =
                    stream_point<BLACK_FUSED, kRR2, kKK2>(Sp1, Sz, Sp2, cB, sr, sc, (cB ^ ap ^ yp ^ sr) & 1, c);
            if (d >= 2 && it >= 2)  // R1, plane a - 1: black of B1
                Sz[cR * kRR2 * kKK2 + at] =
                    stream_point<RED_FUSED, kRR2, kKK2>(Sz, Sm1, Sp1, cR, sr, sc, (cR ^ ap ^ 1 ^ yp ^ sr) & 1, c);
            float4 cur = hA;
            if (d >= 3 && it >= 4) {  // B2, plane a - 2: red of R1
                cur = stream_point<BLACK_FUSED, kRR2, kKK2>(Sm1, Sm2, Sz, cB, sr, sc, (cB ^ ap ^ yp ^ sr) & 1, c);
                Sm1[cB * kRR2 * kKK2 + at] = cur;
                if (d == 4 && it >= 5 && it < L + 5) put(oB, cur);  // planes x0 .. x0 + L - 1
            }
            if (d == 4) {
                if (it >= 6)  // R2, plane a - 3: black of B2 (below from two iterations back, above just made)
                    put(oR, stream_point_v<REDMODE, kRR2, kKK2>(Sm2, hB, cur, cR, sr, sc, (cR ^ ap ^ 1 ^ yp ^ sr) & 1, c));
                hB = hA;
                hA = cur;
            }
            oB += plane_elems;
            oR += plane_elems;
            // the next B1 needs staged plane it + 3 (its upper neighbours)
            bad = 0;
            if (stall && first && it == 1) bad = !mbar_wait_bounded(&bars[kSlots2], 0);  // never completes
            if (!bad && it + 3 <= L + 7) {
                const bool ok = mbar_wait_bounded(&bars[jp3], (phase >> jp3) & 1u);
                if (ok) {
                    phase ^= 1u << jp3;
                    if (threadIdx.x == 0) pending &= ~(1u << jp3);
                }
                bad = !ok;
            }
            failed = __syncthreads_or(bad);
        };
        for (int it = 0;;) {
            body(std::integral_constant<int, 0>{}, it);
            if (++it > L + 5 || failed) break;
            body(std::integral_constant<int, 1>{}, it);
            if (++it > L + 5 || failed) break;
            body(std::integral_constant<int, 2>{}, it);
            if (++it > L + 5 || failed) break;
            body(std::integral_constant<int, 3>{}, it);
            if (++it > L + 5 || failed) break;
            body(std::integral_constant<int, 4>{}, it);
            if (++it > L + 5 || failed) break;
            body(std::integral_constant<int, 5>{}, it);
            if (++it > L + 5 || failed) break;
        }
        first = false;
    }
    if (failed && threadIdx.x == 0) {
        *(volatile int*)err = 2;
        for (int s = 0; s < kSlots2; ++s)
            if (pending & (1u << s)) mbar_wait_bounded(&bars[s], (phase >> s) & 1u);
    }
}

// Whole-state conversions between the colour-split layout (P,Q vec2 array;
// U then V planar) and the packed layout with ghost copies.
__global__ void to_packed_kernel(const float2* __restrict__ pq, const float* __restrict__ uv, float4* __restrict__ out,
                                 int N)
{
    const int hN = N >> 1;
    const int64_t cols = hN + 4, rows = N + 2 * kG;
    const int64_t total = 2 * (int64_t)N * rows * cols;
    const int64_t M = (int64_t)N * N * N, half = M >> 1;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int pc = (int)(e % cols);
        int64_t t = e / cols;
        const int pr = (int)(t % rows);
        t /= rows;
        const int x = (int)(t % N), col = (int)(t / N);
        int y = pr - kG, zh = pc - 2;
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
    const int64_t cols = hN + 4, rows = N + 2 * kG;
    const int64_t M = (int64_t)N * N * N, half = M >> 1;
    for (int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pos < M; pos += (int64_t)gridDim.x * blockDim.x) {
        const int col = pos >= half;
        const int64_t q = pos - (col ? half : 0);
        const int zh = (int)(q % hN);
        const int64_t t = q / hN;
        const int y = (int)(t % N), x = (int)(t / N);
        const float4 v = in[(((int64_t)col * N + x) * rows + y + kG) * cols + zh + 2];
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

namespace {

// The fewest chunks per tile column (at least two: a column alone measured
// slower) whose items fill at least 95% of the rounds of `sms` CTAs, else
// the best filling.
int auto_chunk(int64_t N, int sms, int tile_rows)
{
    const int64_t ntiles = ((N + tile_rows - 1) / tile_rows) * (N / 2 / kTh);
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

// A region of one staged plane: tile-relative rows -8 .. ty + 7, colour
// columns -4 .. 39.
struct Region {
    static constexpr int kOffR = 8, kOffC = 4, kW = 44;
    int ty;
    std::vector<unsigned char> b;
    explicit Region(int ty_) : ty(ty_), b((size_t)(ty_ + 16) * kW, 0) {}
    bool in(int y, int k) const { return y >= -kOffR && y < ty + 8 && k >= -kOffC && k < kW - kOffC; }
    bool has(int y, int k) const { return in(y, k) && b[(size_t)(y + kOffR) * kW + k + kOffC]; }
    bool set(int y, int k)
    {
        if (!in(y, k)) return false;
        b[(size_t)(y + kOffR) * kW + k + kOffC] = 1;
        return true;
    }
    void add(const Region& o)
    {
        for (size_t i = 0; i < b.size(); ++i) b[i] |= o.b[i];
    }
};

// The points of the other colour that colour-`col` points of `r` read in
// their plane, whose parity with the tile's first row is P; false if one
// falls outside the region's frame.
bool add_inplane(const Region& r, int col, int P, Region& out)
{
    bool ok = true;
    for (int y = -Region::kOffR; y < r.ty + 8; ++y)
        for (int k = -Region::kOffC; k < Region::kW - Region::kOffC; ++k) {
            if (!r.has(y, k)) continue;
            const int zp = (col ^ P ^ y) & 1;
            ok = out.set(y - 1, k) && out.set(y + 1, k) && out.set(y, k - 1 + zp) && out.set(y, k + zp) && ok;
        }
    return ok;
}

// The side list of one tile height and parity q (see Side2): the points of
// B1's region beyond the main threads', each with the passes it takes.
// False if the regions break what the kernel assumes of them.
bool side_list(int ty, int q, uint16_t* pos, uint16_t& n)
{
    constexpr int cR = 0, cB = 1;
    Region T(ty);
    for (int y = 0; y < ty; ++y)
        for (int k = 0; k < kTh; ++k) T.set(y, k);
    bool ok = true;
    // D3(P): B2's region on a plane of parity P (R2 is on the tile of every plane)
    auto d3 = [&](int P) {
        Region r = T;
        ok = add_inplane(T, cR, P, r) && ok;
        return r;
    };
    auto d2 = [&](int P) {  // R1's
        Region a = d3(P), r = a;
        r.add(d3(P ^ 1));
        ok = add_inplane(a, cB, P, r) && ok;
        return r;
    };
    auto d1 = [&](int P) {  // B1's
        Region a = d2(P), r = a;
        r.add(d2(P ^ 1));
        ok = add_inplane(a, cR, P, r) && ok;
        return r;
    };
    // B1 on a plane of parity q, R1 on q ^ 1, B2 on q, R2 on the tile
    const Region D1 = d1(q), D2 = d2(q ^ 1), D3 = d3(q);
    // every point B1 updates reads inside the staged box: rows -4 .. ty + 3, columns -2 .. 33
    Region box(ty);
    ok = add_inplane(D1, cB, q, box) && ok;
    if (!ok) return false;
    struct E {
        int depth, y, k;
    };
    std::vector<E> side;
    for (int y = -Region::kOffR; y < ty + 8; ++y)
        for (int k = -Region::kOffC; k < Region::kW - Region::kOffC; ++k) {
            if (box.has(y, k) && (y < -4 || y > ty + 3 || k < -2 || k > kTh + 1)) return false;
            const bool in1 = D1.has(y, k), in2 = D2.has(y, k), in3 = D3.has(y, k), in4 = T.has(y, k);
            if ((in2 && !in1) || (in3 && !in2) || (in4 && !in3)) return false;  // nested
            const int depth = in1 + in2 + in3 + in4;
            const bool main_pos = y >= -3 && y <= ty + 2 && k >= 0 && k < kTh;
            if (main_pos) {
                const int want = 1 + (y >= -2 && y <= ty + 1) + (y >= -1 && y <= ty) + (y >= 0 && y < ty);
                if (depth != want) return false;  // the main threads' rule
            } else if (depth > 0) {
                if (depth > 3 || y < -3 || y > ty + 2) return false;
                side.push_back({depth, y, k});
            }
        }
    if (side.size() > (size_t)kSide2) return false;
    std::stable_sort(side.begin(), side.end(), [](const E& u, const E& v) { return u.depth > v.depth; });
    n = (uint16_t)side.size();
    for (size_t i = 0; i < side.size(); ++i)
        pos[i] = (uint16_t)((side[i].y + 4) | ((side[i].k + 2) << 5) | ((side[i].depth - 1) << 11) | 0x8000);
    return true;
}

}  // namespace

int stream_auto_chunk(int64_t N, int sms)
{
    // measured at 512^3 (144 tiles): 256-plane chunks 0.750 of HBM, 171:
    // 0.746, 128: 0.744, 512: 0.739, 64: 0.730
    return auto_chunk(N, sms, kTy);
}

int stream2_auto_chunk(int64_t N, int sms)
{
    return auto_chunk(N, sms, kTy2);
}

int stream2_prepare(int64_t N, void* side_out)
{
    static_assert(sizeof(Side2) <= kStream2SideBytes, "side list size");
    Side2 t;
    memset(&t, 0, sizeof t);
    const int last = (int)(N % kTy2);
    for (int q = 0; q < 2; ++q) {
        if (!side_list(kTy2, q, t.pos[0][q], t.n[0][q])) return -1;
        if (last && !side_list(last, q, t.pos[1][q], t.n[1][q])) return -1;
    }
    memcpy(side_out, &t, sizeof t);
    return 0;
}

size_t stream_buffer_bytes(int64_t N)
{
    return (size_t)2 * N * (N + 2 * kG) * (N / 2 + 4) * sizeof(float4);
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int stream_make_map(void* buf, int64_t N, int steps, void* map_out)
{
    // looked up once, thread-safely (a function-local static's initialisation)
    static const EncodeTiled encode = []() -> EncodeTiled {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return nullptr;
        return reinterpret_cast<EncodeTiled>(fn);
    }();
    if (!encode) return -1;
    const int64_t hN = N / 2;
    // dims, innermost first: the floats of a padded row, rows, planes, colours
    const cuuint64_t rows = (cuuint64_t)(N + 2 * kG);
    const cuuint64_t dims[4] = {(cuuint64_t)(4 * (hN + 4)), rows, (cuuint64_t)N, 2};
    const cuuint64_t row = (cuuint64_t)(hN + 4) * sizeof(float4);
    const cuuint64_t strides[3] = {row, row * rows, row * rows * (cuuint64_t)N};
    // the two-step kernel's box is one float4 wider than the 36 columns it
    // reads, so that its staged rows are 37 float4 apart in shared memory:
    // 16-byte accesses fall into 8 groups of four banks by (pitch x row +
    // column) mod 8, and a pitch of 36 put the points beyond a tile's columns
    // (a few columns on many rows) into two of the eight groups (modelled:
    // 84 wavefronts per warp and pass over them, 36 with a pitch of 37); in
    // the grid's last tile column the extra float4 lies beyond the row and
    // is zero-filled
    const cuuint32_t box[4] = {(cuuint32_t)(steps == 2 ? 4 * kKK2 : 4 * kKK), (cuuint32_t)(steps == 2 ? kRR2 : kRR),
                               1, 2};
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
    // the shared-memory allowance is a per-device function attribute: set it on
    // every launch (a host call of microseconds, next to a launch of a millisecond)
    auto kern = red_mode == RED_ADJ ? stream_kernel<RED_ADJ> : stream_kernel<RED_FUSED>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) != cudaSuccess)
        return -1;
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

int launch_stream2(const void* map, const void* side, void* dst, int64_t N, const Coef<float>& c, int red_mode,
                   int* err, int stall, int chunk, int prefetch, cudaStream_t s)
{
    // the shared-memory allowance is a per-device function attribute: set it on
    // every launch (a host call of microseconds, next to a launch of a millisecond)
    auto kern = red_mode == RED_ADJ ? stream2_kernel<RED_ADJ> : stream2_kernel<RED_FUSED>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes2) != cudaSuccess)
        return -1;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ntiles = ((N + kTy2 - 1) / kTy2) * (N / 2 / kTh);
    const int64_t items = chunk > 0 ? ntiles * ((N + chunk - 1) / chunk) : ntiles * N;
    const unsigned grid = (unsigned)std::min<int64_t>(items, sms);
    CUtensorMap m;
    memcpy(&m, map, sizeof m);
    Side2 t;
    memcpy(&t, side, sizeof t);
    kern<<<grid, kThreads, kSmemBytes2, s>>>(m, reinterpret_cast<float4*>(dst), (int)N, c, t, err, stall, chunk,
                                             prefetch);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_to_packed(const void* pq, const void* uv, void* out, int64_t N, cudaStream_t s)
{
    const int64_t total = 2 * N * (N + 2 * kG) * (N / 2 + 4);
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
