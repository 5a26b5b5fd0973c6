// kgs_point.cuh -- pointwise DP-AVF2 updates of the KGS equations
// (arXiv 2502.09537, Eq. scheme1 and the adjoint Eq. dp-avf-kj-adj), shared by
// every kernel of libkgs.
//
// All arithmetic goes through explicitly rounded intrinsics (__fma_rn,
// __dmul_rn, ...), so the compiler cannot contract or reassociate it and every
// kernel variant (one launch per colour pass, shared-memory resident, tiled)
// produces bitwise the same state.
//
// Notation (half step s = tau/2, dimension d, grid spacing h):
//   beta  = s kappa1 / (2 h^2)      neighbour weight in the Psi equation
//   alpha = d beta                  its diagonal
//   g     = s gamma / 2
//   A     = d s kappa2 / h^2 + s mu^2 / 2,   B = s kappa2 / h^2,   E = s gamma
// Psi update (first equation of Eq. scheme1), r = alpha - g U*:
//   (i - r) Psi' = (i + r) Psi - beta S,   S = sum of the 2d neighbours' Psi,
// solved in increment form  (i - r) dPsi = 2 r Psi - beta S:
//   N = 2 r Psi - beta S,   dPsi = N / (i - r) = -N (r + i) / (1 + r^2)
//   dP = (N_im - r N_re) / (1 + r^2),   dQ = -(N_re + r N_im) / (1 + r^2).
// (U,V) update (last two equations of Eq. scheme1) in increment form:
//   (1 + A s/2) dV = B SU + E rho - 2 A U - A s V,   dU = s V + (s/2) dV,
// with SU the sum of the neighbours' U and rho = |Psi|^2 at the point.
// Increment form keeps each update's rounding proportional to the increment
// (constants that are not exact multiply only the increment); the direct form
// drifts E_h by about one ulp per step.
//
// The colour passes are bound by the FP64 pipe, so the code below is arranged
// to minimise FP64 instructions per point (about 47 in 2D) without giving up
// the exact structure described below.
//
// Which U* and rho each half uses (Eqs. scheme1, dp-avf-kj-adj):
//   base Phi_s    : Psi with U^n, then (U,V) with |Psi^{n+1}|^2
//   adjoint Phi*_s: (U,V) with |Psi^n|^2, then Psi with U^{n+1} (both sides)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kgs {

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };
template <typename T> using vec2_t = typename Vec2<T>::type;

// Half-step coefficients in the state precision (computed on the host in FP64,
// see kgs_api.cu).  Names as in the header comment; primes mark constants
// pre-multiplied by inv_det = 1 / (1 + A s/2).
template <typename T> struct Coef {
    T alpha, g;        // r = alpha - g U
    T beta;            // Psi neighbour weight
    T Bp, Ep, twoAp;   // B', E', 2A'
    T s, hs;           // s = tau/2, s/2
};

// ------------------------------------------------- rounded arithmetic --
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
// Reciprocal of a >= 1 in float64: the hardware estimate (rcp.approx.ftz.f64,
// about 20 correct bits from the high word) refined by one step of the
// cubically convergent Newton-Raphson iteration for 1/a,
//   e = 1 - a y,   y <- y + y (e + e^2)
// (J.-M. Muller et al., Handbook of Floating-Point Arithmetic, ch. on Newton-
// Raphson division), whose error after the step is about e^3 ~ 2^-60 before
// the final rounding: within one ulp of the IEEE quotient (kgs_probe.h
// measures it against CUDA's division).  Three FP64 FMAs instead of the
// longer correctly rounded sequence; here the reciprocal only scales an
// increment, so one ulp in it is far below one ulp of the state.
__device__ __forceinline__ double rcp_(double a)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
    const double e = __fma_rn(-a, y, 1.0);
    return __fma_rn(y, __fma_rn(e, e, e), y);
}
__device__ __forceinline__ float rcp_(float a) { return __frcp_rn(a); }

// ---------------------------------------------------- neighbour sums --
// S = the sum of a field over the 2d neighbours of a point (Eq. scheme1's
// discrete Laplacian without the centre term).
//
// FP32: the left-to-right sum.
//
// FP64: the correctly rounded sum (round to nearest even of the exact sum),
// formed without the FP64 pipe.  On this part the FP64 pipe executes two
// thread-instructions per cycle per SM and bounds the colour passes, while the
// 32-bit integer pipe (64 per cycle per SM) is nearly idle; the 2d-1 FP64
// additions per field are 20% (2D) to 29% (3D) of a pass's FP64 instructions.
// Each value is split into sign, exponent and 53-bit significand, shifted to
// the largest exponent in a signed 128-bit fixed-point accumulator (the
// largest significand's leading bit at bit 123, so up to 8 terms cannot
// overflow and any term within 71 binades of the largest is added exactly),
// and the exact sum is rounded once.  Where that does not apply -- an input is
// infinite, NaN or subnormal, a nonzero term lies more than 71 binades below
// the largest, or the sum is not a normal number -- the left-to-right FP64 sum
// is taken instead, in a function call so the compiler cannot execute it
// speculatively for every lane.  A zero sum is -0 only if every term is -0,
// as in IEEE addition.  The result does not depend on the neighbour order.
template <int K>
__device__ __noinline__ double nsum_seq(const double (&v)[K])
{
    double s = v[0];
#pragma unroll
    for (int i = 1; i < K; ++i) s = __dadd_rn(s, v[i]);
    return s;
}

template <int K>
__device__ __forceinline__ double nsum_exact(const double (&v)[K], bool& ok)
{
    static_assert(K >= 2 && K <= 8, "2 to 8 terms");
    uint64_t m[K];
    int e[K];
    uint32_t sg[K];
    int emax = 0;
    bool allnz = true;
    ok = true;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const uint64_t b = (uint64_t)__double_as_longlong(v[i]);
        const int ei = (int)(b >> 52) & 0x7FF;
        const uint64_t f = b & 0x000FFFFFFFFFFFFFull;
        ok = ok && (ei != 0x7FF) && (ei != 0 || f == 0);
        m[i] = ei ? (f | 0x0010000000000000ull) : 0ull;
        e[i] = ei;
        sg[i] = (uint32_t)(b >> 63);
        emax = ei > emax ? ei : emax;
        allnz = allnz && (b == 0x8000000000000000ull);
    }
    // signed 128-bit accumulator (ahi:alo), unit 2^(emax - 1146)
    uint64_t alo = 0, ahi = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const int d = emax - e[i];
        ok = ok && (m[i] == 0 || d <= 71);
        const int sh = 71 - d;
        uint64_t th, tl;
        if (sh >= 64) { th = m[i] << (sh - 64); tl = 0; }
        else if (sh > 0) { th = m[i] >> (64 - sh); tl = m[i] << sh; }
        else { th = 0; tl = sh == 0 ? m[i] : 0; }
        const uint64_t neg = 0ull - (uint64_t)sg[i];  // two's complement: (t ^ neg) + (neg & 1)
        const uint64_t xl = tl ^ neg, xh = th ^ neg;
        const uint64_t l1 = alo + xl;
        const uint64_t c1 = l1 < alo ? 1ull : 0ull;
        const uint64_t l2 = l1 + (neg & 1ull);
        const uint64_t c2 = l2 < l1 ? 1ull : 0ull;
        alo = l2;
        ahi = ahi + xh + c1 + c2;
    }
    if ((alo | ahi) == 0ull) return allnz ? -0.0 : 0.0;
    const uint64_t sgn = ahi >> 63;
    if (sgn) {
        alo = ~alo + 1ull;
        ahi = ~ahi + (alo == 0ull ? 1ull : 0ull);
    }
    // normalise the magnitude so that its leading one is bit 127
    const int c = ahi ? __clzll((long long)ahi) : 64 + __clzll((long long)alo);
    uint64_t h, l;
    if (c >= 64) { h = alo << (c - 64); l = 0; }
    else if (c > 0) { h = (ahi << c) | (alo >> (64 - c)); l = alo << c; }
    else { h = ahi; l = alo; }
    const int er = emax + 4 - c;  // biased exponent of the sum
    ok = ok && er >= 1 && er <= 0x7FE;
    uint64_t M = h >> 11;  // 53 bits with the leading one
    const uint64_t rb = (h >> 10) & 1ull;
    const uint64_t st = ((h & 0x3FFull) | l) != 0ull ? 1ull : 0ull;
    M += rb & (st | (M & 1ull));  // a carry out of M lands in the exponent field
    const uint64_t bits = (sgn << 63) | ((((uint64_t)(er - 1)) << 52) + M);
    return __longlong_as_double((long long)bits);
}

template <int K> __device__ __forceinline__ double nsum(const double (&v)[K])
{
    bool ok;
    double s = nsum_exact<K>(v, ok);
    if (!ok) s = nsum_seq<K>(v);
    return s;
}

template <int K> __device__ __forceinline__ float nsum(const float (&v)[K])
{
    float s = v[0];
#pragma unroll
    for (int i = 1; i < K; ++i) s = __fadd_rn(s, v[i]);
    return s;
}

// --------------------------------------------------------- pointwise --
// Structure that must hold exactly in floating point, not only algebraically:
// the Psi update is a Cayley transform, (i - r) Psi' = (i + r) Psi - beta S,
// which keeps |Psi| when S = 0.  Its increment 2 r Psi - beta S is formed
// with 2r = r + r (exact) and the same r as the denominator, so rounding only
// enters through per-point roundings of unbiased sign; scaling 2r by a
// rounded constant instead would break |i + r| = |i - r| by that constant's
// rounding at every update and drift E_h steadily.  Likewise the (U,V) update
// is written as the implicit midpoint rule it is, U' = U + (s/2)(V + V'), so
// that s enters through s/2 alone.

// The Psi update for one value of r, prepared once and applied once or twice
// (the red pass applies the adjoint and the next base update with the same U,
// hence the same r).
template <typename T> struct PsiPrep {
    T r, r2, w;  // r, 2r, 1/(1 + r^2)
};

template <typename T> __device__ __forceinline__ PsiPrep<T> psi_prep(const Coef<T>& c, T u)
{
    PsiPrep<T> pp;
    pp.r = fma_(-c.g, u, c.alpha);
    pp.r2 = add_(pp.r, pp.r);
    pp.w = rcp_(fma_(pp.r, pp.r, T(1)));
    return pp;
}

// dPsi = (2r Psi - beta S) / (i - r):
//   N = 2r Psi - bS,  dP = (N_im - r N_re) w,  dQ = -(N_re + r N_im) w,
// with (bSP, bSQ) = beta S computed once per point and pass.
template <typename T>
__device__ __forceinline__ void psi_apply(const PsiPrep<T>& pp, T bSP, T bSQ, T& P, T& Q)
{
    const T nre = fma_(pp.r2, P, -bSP);
    const T nim = fma_(pp.r2, Q, -bSQ);
    const T tP = fma_(-pp.r, nre, nim);
    const T tQ = fma_(pp.r, nim, nre);
    P = fma_(tP, pp.w, P);
    Q = fma_(-tQ, pp.w, Q);
}

// t' = (B SU + E |Psi|^2) / (1 + A s/2): the part of the (U,V) right side
// fixed by the neighbours and the point's |Psi|^2.
template <typename T> __device__ __forceinline__ T uv_src(const Coef<T>& c, T SU, T P, T Q)
{
    const T rho = fma_(P, P, mul_(Q, Q));
    return fma_(c.Bp, SU, mul_(c.Ep, rho));
}

// One (U,V) update, the implicit midpoint rule of the last two equations of
// Eq. scheme1:  a = U + (s/2) V,  dV = t' - 2A' a,  V' = V + dV,  U' = a + (s/2) V'.
template <typename T> __device__ __forceinline__ void uv_step(const Coef<T>& c, T t, T& U, T& V)
{
    const T a = fma_(c.hs, V, U);
    const T dV = fma_(-c.twoAp, a, t);
    V = add_(V, dV);
    U = fma_(c.hs, V, a);
}

// The four kinds of colour pass of a checkerboard DP-AVF2 run
// (Algorithm 3: per step red-base, black-base, black-adjoint, red-adjoint).
// Black-base and black-adjoint see the same red neighbours, so they fuse;
// red-adjoint of step n and red-base of step n+1 see the same black
// neighbours, so they fuse too.  A run of n steps is
//   RED_BASE, (BLACK_FUSED, RED_FUSED) x (n-1), BLACK_FUSED, RED_ADJ.
// RED_FUSED computes exactly RED_ADJ followed by RED_BASE, so a run split
// into several calls gives bitwise the same state.
enum PassMode { RED_BASE = 0, BLACK_FUSED = 1, RED_FUSED = 2, RED_ADJ = 3 };

// Update one point of the pass's colour in registers.  SP, SQ, SU are the
// neighbour sums (neighbours are of the other colour and fixed for the pass).
template <typename T, int MODE>
__device__ __forceinline__ void update_point(const Coef<T>& c, T SP, T SQ, T SU,
                                             T& P, T& Q, T& U, T& V)
{
    const T bSP = mul_(c.beta, SP), bSQ = mul_(c.beta, SQ);
    if (MODE == RED_BASE) {
        psi_apply(psi_prep(c, U), bSP, bSQ, P, Q);  // base Psi with U^n
        uv_step(c, uv_src(c, SU, P, Q), U, V);      // base (U,V) with |Psi^{n+1}|^2
    } else if (MODE == BLACK_FUSED) {
        psi_apply(psi_prep(c, U), bSP, bSQ, P, Q);  // base Psi with U^n
        // base and adjoint (U,V): both use |Psi^{n+1}|^2 of the base half (the
        // adjoint's |Psi^n|^2) and the same neighbours
        const T t = uv_src(c, SU, P, Q);
        uv_step(c, t, U, V);
        uv_step(c, t, U, V);
        psi_apply(psi_prep(c, U), bSP, bSQ, P, Q);  // adjoint Psi with U^{n+1}
    } else if (MODE == RED_FUSED) {
        uv_step(c, uv_src(c, SU, P, Q), U, V);      // adjoint (U,V) with |Psi^n|^2
        const PsiPrep<T> pp = psi_prep(c, U);
        psi_apply(pp, bSP, bSQ, P, Q);              // adjoint Psi with U^{n+1}
        psi_apply(pp, bSP, bSQ, P, Q);              // next base Psi: same U, same r
        uv_step(c, uv_src(c, SU, P, Q), U, V);      // next base (U,V)
    } else {  // RED_ADJ
        uv_step(c, uv_src(c, SU, P, Q), U, V);
        psi_apply(psi_prep(c, U), bSP, bSQ, P, Q);
    }
}

// Colour parity: a point is red when its 1-based index sum is odd, i.e. when
// the 0-based sum plus d is odd.  parity_of(colour) is the 0-based sum's parity.
__host__ __device__ __forceinline__ int red_parity(int dim) { return (dim + 1) & 1; }

}  // namespace kgs
