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
// Work: a CTA owns a tile of 32 x 64 points of the other two axes (32 rows
// along axis 1, 32 points of each colour along the last axis) and walks every
// axis-0 plane of it, periodically: planes -2 .. N+1 are staged, black is
// updated on planes -1 .. N and red on planes 0 .. N-1, the two ends
// recomputing the neighbouring planes' black values from the same inputs (so
// bitwise the values their owner computes).  Within a plane the black pass
// covers the tile and the ring of black points around it that the tile's red
// points read, which needs the red points of a two-point ring: each staged
// plane is the tile plus a two-point halo, (32 + 4) x (32 + 4) points of each
// colour.
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
// Ring: five slots; the load of plane j + 5 goes into the slot of plane j
// once the step at plane j + 2 is done with it, a full plane iteration before
// it is needed.  Two CTA barriers per plane: between the black and the red
// pass, and after the red pass (where the next plane's load is also awaited).
// Every wait on an mbarrier is bounded (2 s of %globaltimer); a CTA whose wait
// runs out sets the error word, waits (bounded) for its loads in flight and
// leaves.
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
constexpr int kTy = 32;                  // tile rows (axis 1)
constexpr int kRR = kTy + 4, kKK = kTh + 4;  // staged rows / columns per colour
constexpr int kSlotElems = 2 * kRR * kKK;    // float4 per staged plane
constexpr int kSlots = 5;
constexpr int kWarps = 18;               // black pass: (kTy + 4) row tasks over 18 warps = 2 each
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

// Store a point of colour c at (x, y, zh) of the packed layout, with its
// ghost copies (the periodic images two rows / two columns beyond the edges).
__device__ __forceinline__ void store_packed(float4* __restrict__ dst, int N, int c, int x, int y, int zh,
                                             float4 v)
{
    const int hN = N >> 1;
    const int64_t cols = hN + 4, rows = N + 4;
    float4* plane = dst + ((int64_t)c * N + x) * rows * cols;
    const int pr = y + 2, pc = zh + 2;
    const int pr2 = y < 2 ? y + N + 2 : (y >= N - 2 ? y - N + 2 : -1);
    const int pc2 = zh < 2 ? zh + hN + 2 : (zh >= hN - 2 ? zh - hN + 2 : -1);
    if (!kgs_in_bounds(c >= 0 && c < 2 && x >= 0 && x < N && pr < rows && pc < cols && pr2 < rows && pc2 < cols &&
                           y >= 0 && zh >= 0,
                       4u))
        return;
    plane[pr * cols + pc] = v;
    if (pr2 >= 0) plane[pr2 * cols + pc] = v;
    if (pc2 >= 0) {
        plane[pr * cols + pc2] = v;
        if (pr2 >= 0) plane[pr2 * cols + pc2] = v;
    }
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
                  int stall)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4* slots = reinterpret_cast<float4*>(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)kSlots * kSlotElems * sizeof(float4));
    constexpr int cR = 0, cB = 1;  // 3D: red = even 0-based coordinate sum (red_parity(3) == 0)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int hN = N >> 1;
    const int tiles_z = hN / kTh, ntiles = (N / kTy) * tiles_z;
    if (threadIdx.x == 0) {
        for (int s = 0; s <= kSlots; ++s) mbar_init(&bars[s], 1);  // bars[kSlots]: the stall test's
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;    // bit s: parity of slot s's next completion (same in every thread)
    uint32_t pending = 0;  // thread 0: slots with a load in flight
    int failed = 0;
    for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
        const int y0 = (tile / tiles_z) * kTy, zh0 = (tile % tiles_z) * kTh;
        // staged plane j (0 .. N+3) is axis-0 plane j - 2 mod N, in slot j % kSlots
        auto issue = [&](int j) {
            const int s = j % kSlots;
            int p = j - 2;
            p = p < 0 ? p + N : (p >= N ? p - N : p);
            mbar_expect_tx(&bars[s], (unsigned)(kSlotElems * sizeof(float4)));
            tma_load_plane(slots + s * kSlotElems, &src, &bars[s], 4 * zh0, y0, p);
            pending |= 1u << s;
        };
        auto wait = [&](int j) -> bool {
            const int s = j % kSlots;
            const bool ok = mbar_wait_bounded(&bars[s], (phase >> s) & 1u);
            if (ok) {
                phase ^= 1u << s;
                if (threadIdx.x == 0) pending &= ~(1u << s);
            }
            return ok;
        };
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int j = 0; j < kSlots - 1; ++j) issue(j);
        }
        int bad = 0;
        for (int j = 0; j < 3; ++j) bad |= !wait(j);
        failed = __syncthreads_or(bad);
        for (int cb = -1; cb <= N && !failed; ++cb) {
            // black pass on plane cb (staged j = cb + 2); red neighbours in j = cb + 1, cb + 3
            {
                const float4* s = slots + ((cb + 2) % kSlots) * kSlotElems;
                const float4* dn = slots + ((cb + 1) % kSlots) * kSlotElems;
                const float4* up = slots + ((cb + 3) % kSlots) * kSlotElems;
                float4* sw = slots + ((cb + 2) % kSlots) * kSlotElems + cB * kRR * kKK;
                for (int t = warp; t < kTy + 4; t += kWarps) {
                    int r, k;
                    if (t < kTy) {
                        r = 2 + t;
                        k = 2 + lane;
                    } else if (t < kTy + 2) {
                        r = t == kTy ? 1 : kTy + 2;
                        k = 2 + lane;
                    } else {
                        r = 2 + lane;
                        k = t == kTy + 2 ? 1 : kTh + 2;
                    }
                    // black (colour 1) at axis-0 plane cb, row y0 - 2 + r (y0 even)
                    const int zp = (cB ^ cb ^ r) & 1;
                    sw[r * kKK + k] = stream_point<BLACK_FUSED>(s, dn, up, cB, r, k, zp, c);
                }
            }
            __syncthreads();
            // red pass on plane cb - 1 (staged j = cb + 1); black neighbours in j = cb, cb + 2
            if (cb >= 1) {
                const int x = cb - 1;
                const float4* s = slots + ((cb + 1) % kSlots) * kSlotElems;
                const float4* dn = slots + (cb % kSlots) * kSlotElems;
                const float4* up = slots + ((cb + 2) % kSlots) * kSlotElems;
                for (int t = warp; t < kTy; t += kWarps) {
                    const int r = 2 + t, k = 2 + lane;
                    const int zp = (cR ^ x ^ r) & 1;
                    const float4 a = stream_point<REDMODE>(s, dn, up, cR, r, k, zp, c);
                    const int y = y0 + t, zh = zh0 + lane;
                    store_packed(dst, N, cR, x, y, zh, a);
                    store_packed(dst, N, cB, x, y, zh, s[cB * kRR * kKK + r * kKK + k]);
                }
            }
            // the next black pass needs staged plane cb + 4
            bad = 0;
            if (stall && cb == 0) bad = !mbar_wait_bounded(&bars[kSlots], 0);  // never completes
            if (!bad && cb + 4 <= N + 3) bad = !wait(cb + 4);
            failed = __syncthreads_or(bad);
            // staged plane cb (axis-0 plane cb - 2) is no longer read: load plane cb + 5 into its slot
            if (!failed && threadIdx.x == 0 && cb + 5 <= N + 3) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(cb + 5);
            }
        }
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
    CUresult r = encode(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, buf, dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

int launch_stream(const void* map, void* dst, int64_t N, const Coef<float>& c, int red_mode, int* err, int stall,
                  cudaStream_t s)
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
    const int ntiles = (int)((N / kTy) * (N / 2 / kTh));
    const unsigned grid = (unsigned)std::min(ntiles, sms);
    CUtensorMap m;
    memcpy(&m, map, sizeof m);
    kern<<<grid, kThreads, kSmemBytes, s>>>(m, reinterpret_cast<float4*>(dst), (int)N, c, err, stall);
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
