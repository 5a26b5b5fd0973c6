// kgs_reduce.cu -- discrete invariants of a KGS state in float64.
//
//   E_h  = h^d sum [ 1/2 (kappa1 |grad_h psi|^2 + kappa2 |grad_h u|^2 + v^2 + mu^2 u^2)
//                    - gamma |psi|^2 u ]            (Sec. 2 E_h, Eq. ene-origin)
//   S_E  = h^d sum of the absolute values of those five terms
//   mass = h^d sum |psi|^2                           (the discrete norm of Sec. 2)
// grad_h is the forward difference (summation by parts turns -X^T D X into
// sum |grad_h X|^2).  Float32 state is widened to float64 before differencing.
//
// Two kernels, deterministic for a given grid size: a pass over the rows in
// which each thread sums its points (plainly over 8 points, those sums with
// Neumaier compensation) and each block reduces with warp shuffles into
// per-block partials; then one block combines the partials with compensated
// arithmetic and scales by h^d.
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

// Float32 state value widened to float64 exactly, with integer operations
// (the FP64 pipe binds this kernel): re-bias the exponent and shift the
// significand.  Zeros keep their sign; subnormal, infinite and NaN inputs
// take the hardware conversion in a call (kept out of line so that the
// common path does not execute it).
static __device__ __noinline__ double widen_slow(float x) { return (double)x; }
__device__ __forceinline__ double widen(float x)
{
    const uint32_t b = __float_as_uint(x);
    const uint32_t mag = b & 0x7FFFFFFFu;
    if (mag - 0x00800000u >= 0x7F000000u) {  // not a normal number
        if (mag == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
        return widen_slow(x);
    }
    const uint32_t hi = (b & 0x80000000u) | ((mag >> 3) + (896u << 20));
    return __hiloint2double((int)hi, (int)(b << 29));
}
__device__ __forceinline__ double widen(double x) { return x; }

// Energy terms of one point from its values and forward differences:
// gp = sum over axes of |Psi_{+e} - Psi|^2, gu = sum of (U_{+e} - U)^2.
// Adds the point's energy density to e, its absolute terms to sc and
// |Psi|^2 to ms.  k1 = kappa1 / (2 h^2), k2 = kappa2 / (2 h^2).
__device__ __forceinline__ void point_terms(const InvParams& p, double gp, double gu, double P, double Q,
                                            double U, double V, double& e, double& sc, double& ms)
{
    const double rho = fma(P, P, Q * Q);
    const double q = fma(V, V, (p.mu2 * U) * U);  // v^2 + mu^2 u^2
    const double t5 = (p.gamma * rho) * U;       // gamma |psi|^2 u
    e += fma(p.k1, gp, fma(p.k2, gu, fma(0.5, q, -t5)));
    sc += fma(p.abs_k1, gp, fma(p.abs_k2, gu, fma(0.5, q, fabs(t5))));
    ms += rho;
}

// One CTA walks rows of the grid (lines along the last axis); each thread
// takes the pairs (2m, 2m+1) of a row, whose two points have opposite
// colours.  In the colour-split layout (N even) point 2m of row r sits at
// A + r N/2 + m and point 2m+1 at B + r N/2 + m, where A is the half of the
// row's first point's colour and B the other half; the forward neighbour of
// either point along another axis lies in the forward row r' at the same m,
// in the opposite half.  Each thread sums 8 points plainly, then adds that
// sum to its compensated (Neumaier) accumulators.
template <typename T, int D>
__global__ void __launch_bounds__(256) invariants_kernel(const vec2_t<T>* __restrict__ pq,
                                                         const vec2_t<T>* __restrict__ uv,
                                                         int64_t N, int64_t M, InvParams p,
                                                         double* __restrict__ partials)
{
    Comp e{0, 0}, sc{0, 0}, ms{0, 0};
    double le = 0.0, ls = 0.0, lm = 0.0;
    int pending = 0;
    const T* u = reinterpret_cast<const T*>(uv);  // planar: U at a position, V at M + position
    const int64_t half = M >> 1, hp = N >> 1;
    const int64_t rows = M / N;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        // coordinates of the row (D - 1 of them), its colour parity and the
        // forward rows along the other axes
        int64_t fr[2] = {0, 0};
        int pr = 0;
        if (D == 2) {
            pr = (int)(r & 1);
            fr[0] = r == N - 1 ? 0 : r + 1;
        } else if (D == 3) {
            const int64_t i0 = (int64_t)((uint64_t)r / (uint64_t)N), i1 = r - i0 * N;
            pr = (int)((i0 + i1) & 1);
            fr[0] = (i0 == N - 1 ? 0 : i0 + 1) * N + i1;
            fr[1] = i0 * N + (i1 == N - 1 ? 0 : i1 + 1);
        }
        const int64_t A = pr ? half : 0, B = pr ? 0 : half;
        for (int64_t m = threadIdx.x; m < hp; m += blockDim.x) {
            const int64_t pe = A + r * hp + m, po = B + r * hp + m;
            const vec2_t<T> ae = pq[pe], ao = pq[po];
            const double Pe = widen(ae.x), Qe = widen(ae.y), Ue = widen(u[pe]), Ve = widen(u[M + pe]);
            const double Po = widen(ao.x), Qo = widen(ao.y), Uo = widen(u[po]), Vo = widen(u[M + po]);
            // last axis: the even point's neighbour is the odd one; the odd
            // point's is the next pair's even point
            const int64_t pn = A + r * hp + (m + 1 == hp ? 0 : m + 1);
            const vec2_t<T> an = pq[pn];
            double dp = Po - Pe, dq = Qo - Qe, du = Uo - Ue;
            double gpe = fma(dp, dp, dq * dq), gue = du * du;
            dp = widen(an.x) - Po;
            dq = widen(an.y) - Qo;
            du = widen(u[pn]) - Uo;
            double gpo = fma(dp, dp, dq * dq), guo = du * du;
#pragma unroll
            for (int ax = 0; ax < D - 1; ++ax) {
                const int64_t qe = B + fr[ax] * hp + m, qo = A + fr[ax] * hp + m;
                const vec2_t<T> be = pq[qe], bo = pq[qo];
                dp = widen(be.x) - Pe;
                dq = widen(be.y) - Qe;
                du = widen(u[qe]) - Ue;
                gpe = fma(dp, dp, fma(dq, dq, gpe));
                gue = fma(du, du, gue);
                dp = widen(bo.x) - Po;
                dq = widen(bo.y) - Qo;
                du = widen(u[qo]) - Uo;
                gpo = fma(dp, dp, fma(dq, dq, gpo));
                guo = fma(du, du, guo);
            }
            point_terms(p, gpe, gue, Pe, Qe, Ue, Ve, le, ls, lm);
            point_terms(p, gpo, guo, Po, Qo, Uo, Vo, le, ls, lm);
            if (++pending == 4) {
                neumaier_add(e, le);
                neumaier_add(sc, ls);
                neumaier_add(ms, lm);
                le = ls = lm = 0.0;
                pending = 0;
            }
        }
    }
    neumaier_add(e, le);
    neumaier_add(sc, ls);
    neumaier_add(ms, lm);
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

int invariants_blocks(int dim, int64_t N)
{
    int64_t rows = 1;
    for (int a = 1; a < dim; ++a) rows *= N;  // one CTA per row at most
    const int64_t cap = 148 * 8;
    return (int)(rows < 1 ? 1 : (rows > cap ? cap : rows));
}

template <typename T>
int launch_invariants(const Grid& g, const vec2_t<T>* pq, const vec2_t<T>* uv, const InvParams& p,
                      double* partials, int nblocks, double* out3, cudaStream_t stream)
{
    if (!g.split) return -1;  // every state on the device is in the colour-split layout
#define KGS_INV(DD) invariants_kernel<T, DD><<<nblocks, 256, 0, stream>>>(pq, uv, g.N, g.M, p, partials);
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
