// kgs_tile.cu -- temporally blocked colour passes: several consecutive colour
// passes of a checkerboard DP-AVF2 run per launch, on shared-memory tiles.
//
// Layout of the work.  Axis 0 is streamed; the other axes are tiled.  A CTA
// owns the points [x0, x0+LX) along axis 0 and a T1 x T2 tile of the other
// axes (2D: a T2 strip of axis 1), loaded with a halo of H points on each
// side so that P <= H passes can run before the tile's own points need data
// from outside it.  Planes (one axis-0 index each, tile + halo) pass through a
// ring of 2H + 2 shared-memory slots, filled asynchronously (cp.async, 8 or 16
// bytes per copy; the periodic wrap is applied per copy).
//
// Shared-memory layout of a plane (A1 x A2 points, A2 even): the two
// checkerboard classes of the plane, (a1 + a2) even and odd, are stored as two
// row-major halves of A1 x A2/2 points, so that a colour pass -- which works on
// every second point of a row -- reads and writes consecutive addresses: its
// own points, their in-row and in-plane neighbours (the other class) and the
// same positions in the adjacent planes.  In the natural layout consecutive
// threads would be 16 or 32 bytes apart and conflict on the banks.
//
// The launch reads the state from one pair of arrays and writes the other
// (ping-pong): neighbouring CTAs read each other's halo from the input while
// finished planes are written, so the output must be a separate buffer.
//
// Pipeline (lag 2).  In the iteration after plane L has arrived, pass p
// (0-based within the launch) updates plane L-1-2p.  A colour pass reads only
// points of the other colour and writes only its own, so pass p on plane x
// needs x-1, x, x+1 with pass p-1 applied and pass p+1 not yet: plane x+1 got
// pass p-1 one iteration earlier, x two and x-1 three iterations earlier,
// while pass p+1 reaches them only in later iterations.  Within an iteration
// the passes write planes at odd offsets from L and read, besides their own
// plane, only planes at even offsets, so all passes of an iteration run
// concurrently with one barrier per iteration.  A plane is final after pass
// P-1 and is stored in the following iteration.  Pass p is skipped where its
// dependency cone leaves the loaded planes (the CTA's axis-0 ends) and on tile
// points within p+1 of the halo's edge.
//
// Every point update is the code of kgs_point.cuh with the neighbour order of
// the one-launch-per-pass kernel, so the state is bitwise the same as P
// launches of pass_kernel (tests check this for several tile shapes).
#include "kgs_internal.h"

namespace kgs {

namespace {

constexpr int kMaxPasses = 8;

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

template <int BYTES> __device__ __forceinline__ void cp_async(void* dst, const void* src)
{
    static_assert(BYTES == 8 || BYTES == 16, "cp.async size");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(dst)), "l"(src),
                 "n"(BYTES));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ int wrapi(int a, int N)
{
    a %= N;
    return a < 0 ? a + N : a;
}

// Mode of global pass g of an n-step run: R_base, then alternating
// B_fused (odd g) and R_fused, and R_adj last (g = 2n).
__device__ __forceinline__ int pass_mode(int64_t g, int64_t n)
{
    if (g == 0) return RED_BASE;
    if (g == 2 * n) return RED_ADJ;
    return (g & 1) ? BLACK_FUSED : RED_FUSED;
}

// One point update in shared memory.  own = the point's index; nb = its 2D
// neighbours in the order of the pass kernel (axis 0 down, axis 0 up, then
// axis 1 (3D), then the last axis).
template <typename T, int D, int MODE>
__device__ __forceinline__ void tile_point(vec2_t<T>* spq, vec2_t<T>* suv, int own,
                                           const int (&nb)[2 * D], const Coef<T>& c)
{
    T p[2 * D], q[2 * D], w[2 * D];
#pragma unroll
    for (int n = 0; n < 2 * D; ++n) {
        const vec2_t<T> b = spq[nb[n]];
        p[n] = b.x;
        q[n] = b.y;
        w[n] = suv[nb[n]].x;
    }
    vec2_t<T> a = spq[own];
    vec2_t<T> b = suv[own];
    update_point<T, D, MODE>(c, nsum_scaled(p, c.beta), nsum_scaled(q, c.beta), nsum_scaled(w, c.Bp), a.x, a.y, b.x, b.y);
    spq[own] = a;
    suv[own] = b;
}

// Per-thread copies of one plane: at most kMaxCopies elements per thread.
constexpr int kMaxCopies = 6;
// Per-thread positions of one class of a plane: at most kMaxPos.
constexpr int kMaxPos = 4;

template <typename T, int D>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 1024 : 512) tile_kernel(const vec2_t<T>* __restrict__ pq,
                                                    const vec2_t<T>* __restrict__ uv,
                                                    vec2_t<T>* __restrict__ pq_out,
                                                    vec2_t<T>* __restrict__ uv_out, TileParams tp,
                                                    Coef<T> c)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int H = tp.H, R = 2 * tp.H + 2, P = tp.P;
    const int A1 = (D == 2) ? 1 : tp.T1 + 2 * H;
    const int A2 = tp.T2 + 2 * H;
    const int plane = A1 * A2;
    const int W = A2 >> 1;          // points of one class per row
    const int HW = A1 * W;          // points of one class per plane
    const int ring = R * plane;
    vec2_t<T>* spq = reinterpret_cast<vec2_t<T>*>(smem_raw);
    vec2_t<T>* suv = spq + ring;
    const int N = (int)tp.N;

    // tile origin from the launch grid: x = tiles of the last axis, y = tiles of
    // axis 1 (3D), z = ranges of axis 0
    const int y2 = blockIdx.x * tp.T2;
    const int y1 = (D == 3) ? (int)blockIdx.y * tp.T1 : 0;
    const int x0 = blockIdx.z * tp.LX;
    const int lx = min(tp.LX, N - x0);
    const int e1 = (D == 3) ? min(tp.T1, N - y1) : 1;  // tile extent to store
    const int e2 = min(tp.T2, N - y2);
    const int64_t planelen = (D == 3) ? (int64_t)N * N : N;
    const int xfirst = x0 - H, xlast = x0 + lx + H - 1;  // loaded planes
    const int xend = x0 + lx + 2 * P - 2;                // last value of L

    // The in-plane part of every global address this thread copies is the same
    // for every plane: compute it once.
    int ld_goff[kMaxCopies], ld_soff[kMaxCopies], st_soff[kMaxCopies], st_goff[kMaxCopies];
    const int nld = (plane + blockDim.x - 1) / blockDim.x;
    const int cnt = e1 * e2;
    const int nst = (cnt + blockDim.x - 1) / blockDim.x;
#pragma unroll
    for (int k = 0; k < kMaxCopies; ++k) {
        const int q = threadIdx.x + k * blockDim.x;
        ld_goff[k] = -1;
        ld_soff[k] = 0;
        st_goff[k] = -1;
        st_soff[k] = 0;
        if (k < nld && q < plane) {
            int a1 = 0, a2 = q;
            if (D == 3) {
                a1 = q / A2;
                a2 = q - a1 * A2;
            }
            ld_goff[k] = ((D == 3) ? wrapi(y1 - H + a1, N) * N : 0) + wrapi(y2 - H + a2, N);
            ld_soff[k] = ((a1 + a2) & 1) * HW + a1 * W + (a2 >> 1);
        }
        if (k < nst && q < cnt) {
            int b1 = 0, b2 = q;
            if (D == 3) {
                b1 = q / e2;
                b2 = q - b1 * e2;
            }
            const int a1 = (D == 3) ? b1 + H : 0, a2 = b2 + H;
            st_soff[k] = ((a1 + a2) & 1) * HW + a1 * W + (a2 >> 1);
            st_goff[k] = (D == 3 ? (y1 + b1) * N : 0) + y2 + b2;
        }
    }

    // Positions this thread updates in every pass, the same for the whole
    // launch: in-plane indices j = a1 * W + k (k-th point of its class in row
    // a1) of either class, j = threadIdx.x + m * blockDim.x.
    int pos_j[kMaxPos], pos_a1[kMaxPos];
    const int npos = (HW + blockDim.x - 1) / blockDim.x;
#pragma unroll
    for (int m = 0; m < kMaxPos; ++m) {
        const int j = threadIdx.x + m * blockDim.x;
        pos_j[m] = (m < npos && j < HW) ? j : -1;
        pos_a1[m] = (D == 3 && pos_j[m] >= 0) ? j / W : 0;
    }

    // ring slot (element offset) of plane x, for x within R planes above xfirst
    // of a known slot: slot(x) = ((x - xfirst) mod R) * plane
    auto slot_of = [&](int x) {
        int r = x - xfirst;
        while (r >= R) r -= R;  // at most a few subtractions: x - xfirst < lx + 3H + 2
        return r * plane;
    };

    auto load_plane = [&](int x, int base) {
        const int64_t gx = (int64_t)wrapi(x, N) * planelen;
#pragma unroll
        for (int k = 0; k < kMaxCopies; ++k)
            if (ld_goff[k] >= 0) {
                const int si = base + ld_soff[k];
                cp_async<sizeof(vec2_t<T>)>(&spq[si], &pq[gx + ld_goff[k]]);
                cp_async<sizeof(vec2_t<T>)>(&suv[si], &uv[gx + ld_goff[k]]);
            }
        cp_async_commit();
    };

    auto store_plane = [&](int xs, int base) {
        if (xs < x0 || xs >= x0 + lx) return;
        const int64_t gx = (int64_t)xs * planelen;
#pragma unroll
        for (int k = 0; k < kMaxCopies; ++k)
            if (st_goff[k] >= 0) {
                pq_out[gx + st_goff[k]] = spq[base + st_soff[k]];
                uv_out[gx + st_goff[k]] = suv[base + st_soff[k]];
            }
    };

    auto dec = [&](int s, int k) {  // slot k planes below slot s
        int r = s - k * plane;
        return r < 0 ? r + ring : r;
    };

    load_plane(xfirst, 0);
    cp_async_wait_all();
    __syncthreads();
    const int red = red_parity(D);
    int sL = 0;  // slot of plane L
    for (int L = xfirst; L <= xend; ++L, sL = (sL + plane == ring) ? 0 : sL + plane) {
        const int sNext = (sL + plane == ring) ? 0 : sL + plane;
        if (L + 1 <= xlast) load_plane(L + 1, sNext);
        store_plane(L - 2 * P, dec(sL, 2 * P));  // final since the previous iteration

        // The passes of this iteration are independent (see the pipeline note
        // above).  In plane x the points of pass p's colour are exactly one of
        // the two classes, cls = (colour + x + y-origins) mod 2, so every thread
        // updates its own positions of that class, within pass p's region.
        for (int p = 0; p < P; ++p) {
            const int x = L - 1 - 2 * p;
            if (x - p - 1 < xfirst || x + p + 1 > xlast) continue;
            const int lo = p + 1, hi1 = A1 - lo, hi2 = A2 - lo;
            const int g = (int)(tp.g0 + p);
            const int colour = (g & 1) ? (red ^ 1) : red;
            const int s1 = (D == 3) ? y1 - H : 0;
            const int cls = (colour + x + s1 + y2 - H) & 1;
            const int cur = dec(sL, 1 + 2 * p), dn = dec(cur, 1), up = dec(sL, 2 * p);
            const int mode = pass_mode(tp.g0 + p, tp.nsteps);
            const int own_base = cls * HW, oth_base = (cls ^ 1) * HW;
#pragma unroll
            for (int m = 0; m < kMaxPos; ++m) {
                const int j = pos_j[m];
                if (j < 0) continue;
                const int a1 = pos_a1[m];
                const int k = j - a1 * W;
                const int b = (cls + a1) & 1;  // a2 = 2k + b has class cls
                const int a2 = 2 * k + b;
                if (a2 < lo || a2 >= hi2) continue;
                if (D == 3 && (a1 < lo || a1 >= hi1)) continue;
                const int own_h = own_base + j;
                const int oth = oth_base + a1 * W + k;
                int nb[2 * D];
                nb[0] = dn + own_h;
                nb[1] = up + own_h;
                if (D == 3) {
                    nb[2] = cur + oth - W;
                    nb[3] = cur + oth + W;
                }
                nb[2 * D - 2] = cur + oth + b - 1;
                nb[2 * D - 1] = cur + oth + b;
                const int own = cur + own_h;
                switch (mode) {
                case RED_BASE: tile_point<T, D, RED_BASE>(spq, suv, own, nb, c); break;
                case BLACK_FUSED: tile_point<T, D, BLACK_FUSED>(spq, suv, own, nb, c); break;
                case RED_FUSED: tile_point<T, D, RED_FUSED>(spq, suv, own, nb, c); break;
                default: tile_point<T, D, RED_ADJ>(spq, suv, own, nb, c); break;
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();
    }
    store_plane(xend + 1 - 2 * P, slot_of(xend + 1 - 2 * P));
}

}  // namespace

int64_t tile_smem_bytes(int dim, int elem_bytes, const TileParams& tp)
{
    const int64_t A1 = (dim == 2) ? 1 : tp.T1 + 2 * tp.H;
    const int64_t A2 = tp.T2 + 2 * tp.H;
    return (int64_t)(2 * tp.H + 2) * A1 * A2 * 4 * elem_bytes;
}

template <typename T>
int launch_tile(const Grid& g, TileParams tp, const vec2_t<T>* pq, const vec2_t<T>* uv,
                vec2_t<T>* pq_out, vec2_t<T>* uv_out, const Coef<T>& c, cudaStream_t stream)
{
    if (g.dim < 2 || tp.P < 1 || tp.P > tp.H || tp.H > kMaxPasses || tp.T2 < 2 || (tp.T2 & 1) ||
        (g.dim == 3 && tp.T1 < 2) || tp.LX < 1 || g.M >= ((int64_t)1 << 31))
        return -1;
    {
        // every thread copies at most kMaxCopies elements of a plane
        const int64_t A1 = (g.dim == 2) ? 1 : tp.T1 + 2 * tp.H, A2 = tp.T2 + 2 * tp.H;
        const int thr = tp.threads > 0 ? tp.threads : 256;
        if (A1 * A2 > (int64_t)kMaxCopies * thr || A1 * (A2 / 2) > (int64_t)kMaxPos * thr) return -1;
    }
    tp.N = g.N;
    const int64_t bytes = tile_smem_bytes(g.dim, (int)sizeof(T), tp);
    if (bytes > 227 * 1024) return -1;
    const int64_t nt2 = (g.N + tp.T2 - 1) / tp.T2;
    const int64_t nt1 = (g.dim == 3) ? (g.N + tp.T1 - 1) / tp.T1 : 1;
    const int64_t nx = (g.N + tp.LX - 1) / tp.LX;
    if (nt1 > 65535 || nx > 65535) return -1;
    dim3 grid((unsigned)nt2, (unsigned)nt1, (unsigned)nx);
    const int threads = tp.threads > 0 ? tp.threads : 256;
    if (g.dim == 2) {
        if (cudaFuncSetAttribute(tile_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes) != cudaSuccess)
            return -1;
        tile_kernel<T, 2><<<grid, threads, bytes, stream>>>(pq, uv, pq_out, uv_out, tp, c);
    } else {
        if (cudaFuncSetAttribute(tile_kernel<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes) != cudaSuccess)
            return -1;
        tile_kernel<T, 3><<<grid, threads, bytes, stream>>>(pq, uv, pq_out, uv_out, tp, c);
    }
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

template int launch_tile<double>(const Grid&, TileParams, const double2*, const double2*, double2*,
                                 double2*, const Coef<double>&, cudaStream_t);
template int launch_tile<float>(const Grid&, TileParams, const float2*, const float2*, float2*,
                                float2*, const Coef<float>&, cudaStream_t);

}  // namespace kgs
