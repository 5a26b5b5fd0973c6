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
// Reciprocal in float32 (the float64 passes form 1/(1 + r^2) by psi_weight).
__device__ __forceinline__ float rcp_(float a) { return __frcp_rn(a); }

// ---------------------------------------------------- neighbour sums --
// S = the sum of a field over the 2d neighbours of a point (Eq. scheme1's
// discrete Laplacian without the centre term), and c S for a constant c
// (beta for the Psi fields, B' for U).
//
// FP32: the left-to-right sum, and c S as one more rounded product.
//
// FP64: the correctly rounded sum (round to nearest even of the exact sum) and
// the correctly rounded beta S (one rounding of beta times the exact sum),
// formed without the FP64 pipe.  On this part the FP64 pipe executes two
// thread-instructions per cycle per SM and bounds the colour passes, while the
// 32-bit integer pipes (64 ALU and 64 multiply-add lanes per cycle per SM)
// are nearly idle; the 2d-1 FP64 additions per field and the two products
// beta S are a quarter (2D) to a third (3D) of a pass's FP64 instructions.
// Each value is split into sign, exponent and significand (subnormals exactly,
// as exponent 1 without the hidden bit), shifted to the largest exponent in a
// signed 96-bit fixed-point accumulator held in three 32-bit words (the
// largest significand's leading bit at bit 83, so up to 6 terms cannot
// overflow and any term within 31 binades of the largest is added exactly)
// and added with the PTX carry chain (add.cc/addc; a negative term enters as
// its one's complement, the +1s added once at the end).  The exact sum is
// then rounded once, or multiplied exactly by beta's significand (64 x 53
// bits) and rounded once.  Where that does not apply -- an input is infinite
// or NaN, a nonzero term lies more than 31 binades below the largest, beta is
// zero or subnormal, or the result is not a normal number -- the
// left-to-right FP64 sum (times beta, rounded) is taken instead, in a
// function call so that the compiler cannot execute it speculatively for
// every lane.  A zero sum is -0 only if every term is -0, as in IEEE
// addition.  The results do not depend on the neighbour order.
// The fallback: left-to-right sum of the first k of six values, times beta.
// Values are passed by value so that the colour passes keep them in
// registers (an array argument would be stored to local memory at every call
// site, taken or not).
static __device__ __noinline__ double seq_sum6(int k, double beta, double v0, double v1, double v2,
                                        double v3, double v4, double v5)
{
    double s = __dadd_rn(v0, v1);
    if (k > 2) s = __dadd_rn(__dadd_rn(s, v2), v3);
    if (k > 4) s = __dadd_rn(__dadd_rn(s, v4), v5);
    return beta == 1.0 ? s : __dmul_rn(beta, s);
}

template <int K> __device__ __forceinline__ double nsum_seq(const double (&v)[K])
{
    static_assert(K == 2 || K == 4 || K == 6, "2, 4 or 6 neighbours");
    return seq_sum6(K, 1.0, v[0], v[1], v[K > 2 ? 2 : 0], v[K > 2 ? 3 : 0], v[K > 4 ? 4 : 0],
                    v[K > 4 ? 5 : 0]);
}

template <int K> __device__ __forceinline__ double nsum_seq_scaled(const double (&v)[K], double beta)
{
    static_assert(K == 2 || K == 4 || K == 6, "2, 4 or 6 neighbours");
    return seq_sum6(K, beta, v[0], v[1], v[K > 2 ? 2 : 0], v[K > 2 ? 3 : 0], v[K > 4 ? 4 : 0],
                    v[K > 4 ? 5 : 0]);
}

// The exact sum, normalised: |S| = (h + l 2^-64) 2^(er - 1086) with the
// leading one of h at bit 63 (er is the biased exponent of S when S is
// normal), sign sgn; zero = the sum is exactly zero (then negzero = every term
// is -0).  ok = false where the exact accumulator does not apply.
struct ExactSum {
    uint64_t h, l;
    int er;
    uint64_t sgn;
    bool zero, negzero, ok;
};

// (a2:a1:a0) += (x2:x1:x0): one carry chain.
__device__ __forceinline__ void add96(uint32_t& a0, uint32_t& a1, uint32_t& a2, uint32_t x0, uint32_t x1,
                                      uint32_t x2)
{
    asm("add.cc.u32 %0, %0, %3;\n\t"
        "addc.cc.u32 %1, %1, %4;\n\t"
        "addc.u32 %2, %2, %5;"
        : "+r"(a0), "+r"(a1), "+r"(a2)
        : "r"(x0), "r"(x1), "r"(x2));
}

template <int K>
__device__ __forceinline__ ExactSum exact_sum(const double (&v)[K])
{
    static_assert(K >= 2 && K <= 6, "2 to 6 terms");
    uint32_t hi[K], lo[K];
    int e[K];
    int emax = 1, emin = 0x7FF;  // largest exponent; smallest of a nonzero term
    uint32_t hand = 0xFFFFFFFFu, lor = 0u;  // AND of the high words; OR of the magnitude bits
#pragma unroll
    for (int i = 0; i < K; ++i) {
        hi[i] = (uint32_t)__double2hiint(v[i]);
        lo[i] = (uint32_t)__double2loint(v[i]);
        e[i] = (int)(hi[i] >> 20) & 0x7FF;
        const int ei = e[i] > 1 ? e[i] : 1;  // subnormal: exponent 1, no hidden bit
        emax = ei > emax ? ei : emax;
        const uint32_t mag = (hi[i] << 1) | lo[i];  // 0 only for +-0
        const int key = mag ? ei : 0x7FF;
        emin = key < emin ? key : emin;
        hand &= hi[i];
        lor |= mag;
    }
    ExactSum r;
    r.ok = emax != 0x7FF && emax - emin <= 31;  // holds for all-zero rows (emin = 0x7FF)
    // signed 96-bit accumulator (a2:a1:a0), unit 2^(emax - 1106): a term's
    // significand shifted left by 31 - (emax - e) <= 31 stays in three words
    // and six terms stay below 2^87.  A negative term enters as its one's
    // complement; the +1s of the two's complements are added once at the end.
    uint32_t a0 = 0, a1 = 0, a2 = 0, nneg = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const uint32_t mh = (hi[i] & 0xFFFFFu) | (e[i] ? 0x100000u : 0u);
        const int ei = e[i] > 1 ? e[i] : 1;
        // a zero term shifts anything by anything; a nonzero one below the
        // window has made the row not ok
        const uint32_t b = (uint32_t)(31 - emax + ei) & 31u;
        const uint32_t s = (uint32_t)((int32_t)hi[i] >> 31);
        add96(a0, a1, a2, (lo[i] << b) ^ s, __funnelshift_l(lo[i], mh, b) ^ s, __funnelshift_l(mh, 0u, b) ^ s);
        nneg -= s;
    }
    add96(a0, a1, a2, nneg, 0u, 0u);
    const uint32_t sm = (uint32_t)((int32_t)a2 >> 31);
    r.sgn = sm & 1u;
    uint32_t m0 = a0 ^ sm, m1 = a1 ^ sm, m2 = a2 ^ sm;  // magnitude: one's complement + 1
    add96(m0, m1, m2, sm & 1u, 0u, 0u);
    r.zero = (m0 | m1 | m2) == 0u;
    r.negzero = lor == 0u && (hand >> 31) != 0u;
    // normalise: the leading word, then the bits below its leading one
    const bool w2nz = m2 != 0u, w1nz = m1 != 0u;
    const uint32_t p2 = w2nz ? m2 : (w1nz ? m1 : m0);
    const uint32_t p1 = w2nz ? m1 : (w1nz ? m0 : 0u);
    const uint32_t p0 = w2nz ? m0 : 0u;
    const int cb = __clz((int)p2);
    const int c = (w2nz ? 0 : (w1nz ? 32 : 64)) + cb;
    const uint32_t n2 = __funnelshift_l(p1, p2, (uint32_t)cb);
    const uint32_t n1 = __funnelshift_l(p0, p1, (uint32_t)cb);
    const uint32_t n0 = p0 << (cb & 31);
    r.h = ((uint64_t)n2 << 32) | n1;
    r.l = (uint64_t)n0 << 32;
    r.er = emax + 12 - c;
    return r;
}

// Round-to-nearest-even of a significand M (53 bits, leading one at bit 52)
// with round bit rb and sticky st, packed with sign and biased exponent er
// (1 <= er <= 0x7FE; a carry out of M lands in the exponent field).
__device__ __forceinline__ double pack_rn(uint64_t sgn, int er, uint64_t M, uint64_t rb, uint64_t st)
{
    M += rb & (st | (M & 1ull));
    return __longlong_as_double((long long)((sgn << 63) | ((((uint64_t)(er - 1)) << 52) + M)));
}

// S rounded once; ok = false where the caller must take the fallback.
template <int K> __device__ __forceinline__ double nsum_try(const double (&v)[K], bool& ok)
{
    const ExactSum x = exact_sum<K>(v);
    ok = x.ok && (x.zero || (x.er >= 1 && x.er <= 0x7FE));
    if (x.zero) return x.negzero ? -0.0 : 0.0;
    return pack_rn(x.sgn, x.er, x.h >> 11, (x.h >> 10) & 1ull,
                   ((x.h & 0x3FFull) | x.l) != 0ull ? 1ull : 0ull);
}

// beta S rounded once; ok as above.
template <int K>
__device__ __forceinline__ double nsum_scaled_try(const double (&v)[K], double beta, bool& ok)
{
    const ExactSum x = exact_sum<K>(v);
    const uint64_t bb = (uint64_t)__double_as_longlong(beta);
    const int eb = (int)(bb >> 52) & 0x7FF;
    const uint64_t mb = (bb & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const uint64_t sgn = x.sgn ^ (bb >> 63);
    // (h + l 2^-64) mb in [2^115, 2^117): the integer part in (ph:pl), exact,
    // and whether a fraction remains (the low half of l mb)
    const uint64_t lh = __umul64hi(x.l, mb), frac = x.l * mb;
    const uint64_t pl0 = x.h * mb;
    const uint64_t pl = pl0 + lh;
    const uint64_t ph = __umul64hi(x.h, mb) + (pl < pl0 ? 1ull : 0ull);
    const bool top = (ph >> 52) != 0ull;
    const uint64_t M = top ? ph : (ph << 1) | (pl >> 63);
    const uint64_t rb = top ? pl >> 63 : (pl >> 62) & 1ull;
    const uint64_t rest = top ? pl << 1 : pl << 2;
    const int er = x.er + eb - (top ? 1022 : 1023);
    ok = x.ok && eb != 0 && eb != 0x7FF && (x.zero || (er >= 1 && er <= 0x7FE));
    if (x.zero) return (x.negzero ? 1ull : 0ull) ^ (bb >> 63) ? -0.0 : 0.0;
    return pack_rn(sgn, er, M, rb, (rest | frac) != 0ull ? 1ull : 0ull);
}

template <int K> __device__ __forceinline__ double nsum(const double (&v)[K])
{
    bool ok;
    const double r = nsum_try<K>(v, ok);
    return ok ? r : nsum_seq<K>(v);
}

template <int K> __device__ __forceinline__ double nsum_scaled(const double (&v)[K], double beta)
{
    bool ok;
    const double r = nsum_scaled_try<K>(v, beta, ok);
    return ok ? r : nsum_seq_scaled<K>(v, beta);
}

template <int K> __device__ __forceinline__ float nsum(const float (&v)[K])
{
    float s = v[0];
#pragma unroll
    for (int i = 1; i < K; ++i) s = __fadd_rn(s, v[i]);
    return s;
}

template <int K> __device__ __forceinline__ float nsum_scaled(const float (&v)[K], float beta)
{
    return __fmul_rn(beta, nsum<K>(v));
}

// x + x (exact) without the FP64 pipe: one more in the exponent field for a
// normal x whose double is normal, the significand shifted for zero and
// subnormals (a carry moves into the exponent field as it should), infinity
// on overflow, infinities and NaNs kept.
__device__ __forceinline__ double twice(double x)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t e = (uint32_t)(b >> 52) & 0x7FFu;
    const uint64_t sign = b & 0x8000000000000000ull;
    uint64_t r;
    if (e - 1u < 0x7FDu) r = b + (1ull << 52);
    else if (e == 0u) r = sign | ((b << 1) & 0x7FFFFFFFFFFFFFFFull);
    else if (e == 0x7FEu) r = sign | 0x7FF0000000000000ull;
    else r = b;
    return __longlong_as_double((long long)r);
}
__device__ __forceinline__ float twice(float x) { return __fadd_rn(x, x); }

// ------------------------------------------------------ 1 / (1 + r^2) --
// The weight w = 1 / (1 + r^2) of the Psi update.
//
// FP32: the correctly rounded reciprocal of the rounded 1 + r^2.
//
// FP64, off the FP64 pipe (four FMAs and the FP64 reciprocal estimate per
// Psi prepare otherwise): with r = m 2^(e-1075), the top 64 bits of m^2 come
// from one 64 x 64 integer product; 1 is added at its fixed-point position,
// giving a = A 2^(ea-63) with A in [2^63, 2^64) (relative truncation below
// 2^-62); Y ~ 2^127 / A starts from the FP32 reciprocal estimate of A's top
// 24 bits (about 22 correct bits) and takes two Newton-Raphson steps
// Y <- Y + Y (2^127 - A Y) / 2^127 in 64/128-bit integer arithmetic (the
// error squares: 2^-44, then the 2^-62 of the truncations); w = Y 2^(-64-ea)
// rounded to nearest.  The result is within one ulp of the exact
// 1 / (1 + r^2) (faithful; correctly rounded unless the exact value lies
// within about 2^-61 of a rounding boundary), subnormal results included
// (|r| > 2^511, where the FP64 1 + r^2 would overflow).  |r| < 2^-27 gives
// w = 1, the correctly rounded value.  The common path is branch-free; a
// subnormal result and non-finite r (infinite r gives 0, NaN gives NaN) are
// finished in a call.

// a = A 2^(ea-63) ~ 1 + r^2 for finite r, then Y ~ 2^127 / A: 1/a = Y 2^(-64-ea).
__device__ __forceinline__ void psi_weight_core(uint64_t b, int er, uint64_t& Y, int& ea)
{
    const uint64_t M = ((b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 11;
    uint64_t S = __umul64hi(M, M);  // top 64 bits of m^2
    const bool low = (S >> 63) == 0ull;
    S = low ? S << 1 : S;
    const int e2 = 2 * er - 2108 - (low ? 1 : 0);  // r^2 ~ S 2^e2, S in [2^63, 2^64)
    // r^2 >= 1: 1 sits at bit -e2 <= 63 (or below bit 0); r^2 < 1: a in [1, 2)
    const bool big = e2 >= -63;
    const uint64_t Ab = S + ((big && e2 <= 0) ? 1ull << ((-e2) & 63) : 0ull);
    const bool cy = Ab < S;  // carry out of bit 63
    const int ks = -e2 - 63;
    const uint64_t As = 0x8000000000000000ull + (ks < 64 ? S >> (ks & 63) : 0ull);
    const uint64_t A = big ? (cy ? (Ab >> 1) | 0x8000000000000000ull : Ab) : As;
    ea = big ? e2 + 63 + (cy ? 1 : 0) : 0;
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"((float)(uint32_t)(A >> 40)));
    const uint32_t fb = __float_as_uint(rf);
    Y = ((fb >> 23) & 0xFFu) >= 104u ? ~0ull : (uint64_t)((fb & 0x7FFFFFu) | 0x800000u) << 40;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const uint64_t plo = A * Y, phi = __umul64hi(A, Y);
        const int64_t dh = (int64_t)(0x8000000000000000ull - phi - (plo != 0ull ? 1ull : 0ull));
        const uint64_t adh = dh < 0 ? (uint64_t)(-dh) : (uint64_t)dh;
        const uint64_t corr = __umul64hi(Y, adh << 1);  // Y |D| / 2^127
        const uint64_t ya = Y + corr;
        Y = dh < 0 ? Y - corr : (ya < Y ? ~0ull : ya);
    }
}

static __device__ __noinline__ double psi_weight_slow(double r)
{
    const uint64_t b = (uint64_t)__double_as_longlong(r);
    const int er = (int)(b >> 52) & 0x7FF;
    if (er == 0x7FF) return 1.0 / __fma_rn(r, r, 1.0);
    uint64_t Y;
    int ea;
    psi_weight_core(b, er, Y, ea);
    // subnormal w = F 2^-1074 with F = Y 2^(E-12), E = 1022 - ea < 1
    const int sh = 12 - (1022 - ea);  // >= 12
    if (sh > 64) return 0.0;
    uint64_t F = sh == 64 ? 0ull : Y >> sh;
    const uint64_t rb = (Y >> (sh - 1)) & 1ull;
    const uint64_t st = (Y & ((1ull << (sh - 1)) - 1ull)) != 0ull ? 1ull : 0ull;
    F += rb & (st | (F & 1ull));  // a carry into bit 52 gives the least normal
    return __longlong_as_double((long long)F);
}

__device__ __forceinline__ double psi_weight_try(double r, bool& ok)
{
    const uint64_t b = (uint64_t)__double_as_longlong(r);
    const int er = (int)(b >> 52) & 0x7FF;
    uint64_t Y;
    int ea;
    psi_weight_core(b, er, Y, ea);
    const int E = 1022 - ea;  // biased exponent of w when normal
    ok = er < 996 || (er != 0x7FF && E >= 1);
    const double w = pack_rn(0ull, E, Y >> 11, (Y >> 10) & 1ull, (Y & 0x3FFull) != 0ull ? 1ull : 0ull);
    return er < 996 ? 1.0 : w;
}

__device__ __forceinline__ double psi_weight(double r)
{
    bool ok;
    const double w = psi_weight_try(r, ok);
    return ok ? w : psi_weight_slow(r);
}
__device__ __forceinline__ float psi_weight(float r) { return rcp_(fma_(r, r, 1.0f)); }

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

template <typename T, int D> __device__ __forceinline__ PsiPrep<T> psi_prep(const Coef<T>& c, T u)
{
    PsiPrep<T> pp;
    pp.r = fma_(-c.g, u, c.alpha);
    pp.r2 = twice(pp.r);
    pp.w = psi_weight(pp.r);
    return pp;
}

// dPsi = (2r Psi - beta S) / (i - r):
//   N = 2r Psi - bS,  dP = (N_im - r N_re) w,  dQ = -(N_re + r N_im) w,
// with (bSP, bSQ) = beta S formed once per point and pass with the sums.
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
// fixed by the neighbours and the point's |Psi|^2, from BSU = B' SU (formed
// once per point and pass with the neighbour sum: the red pass uses it twice).
template <typename T> __device__ __forceinline__ T uv_src(const Coef<T>& c, T BSU, T P, T Q)
{
    const T rho = fma_(P, P, mul_(Q, Q));
    return fma_(c.Ep, rho, BSU);
}

// One (U,V) update, the implicit midpoint rule of the last two equations of
// Eq. scheme1:  a = U + (s/2) V,  dV = t' - 2A' a,  V' = V + dV,  U' = a + (s/2) V'.
// V + dV correctly rounded on the integer pipes (a two-term exact sum): the
// same value as the FP64 addition, for passes whose integer pipes have room.
__device__ __forceinline__ double add_int(double a, double b)
{
    const double v[2] = {a, b};
    return nsum<2>(v);
}
__device__ __forceinline__ float add_int(float a, float b) { return add_(a, b); }

template <typename T, bool INT_ADD = false>
__device__ __forceinline__ void uv_step(const Coef<T>& c, T t, T& U, T& V)
{
    const T a = fma_(c.hs, V, U);
    const T dV = fma_(-c.twoAp, a, t);
    V = INT_ADD ? add_int(V, dV) : add_(V, dV);
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
enum PassMode { RED_BASE = 0, BLACK_FUSED = 1, RED_FUSED = 2, RED_ADJ = 3, PSI_HALF = 4, UV_HALF = 5 };
// PSI_HALF and UV_HALF: one variable's update alone, for update orders that
// differ per variable (kgs_set_orders): the Psi update with the point's
// current U, the (U,V) update with the point's current |Psi|^2.  RED_BASE is
// PSI_HALF then UV_HALF at a point, RED_ADJ is UV_HALF then PSI_HALF, with
// the same arithmetic.

// Update one point of the pass's colour in registers.  bSP, bSQ = beta S_P,
// beta S_Q and BSU = B' S_U from the neighbour sums above (neighbours are of
// the other colour and fixed for the pass).
// INT_ADD, INT_ADD1: the fused red pass forms both of its V additions, or
// only the first, on the integer pipes (bitwise the same values): both in
// 1D/2D, where that pass's integer pipes have room, the first in 3D, where
// its 6-term sums leave room for one (measured: two slow it down).
template <typename T, int D, int MODE, bool INT_ADD = (D <= 2), bool INT_ADD1 = true>
__device__ __forceinline__ void update_point(const Coef<T>& c, T bSP, T bSQ, T BSU,
                                             T& P, T& Q, T& U, T& V)
{
    if (MODE == RED_BASE) {
        psi_apply(psi_prep<T, D>(c, U), bSP, bSQ, P, Q);  // base Psi with U^n
        uv_step(c, uv_src(c, BSU, P, Q), U, V);      // base (U,V) with |Psi^{n+1}|^2
    } else if (MODE == BLACK_FUSED) {
        psi_apply(psi_prep<T, D>(c, U), bSP, bSQ, P, Q);  // base Psi with U^n
        // base and adjoint (U,V): both use |Psi^{n+1}|^2 of the base half (the
        // adjoint's |Psi^n|^2) and the same neighbours
        const T t = uv_src(c, BSU, P, Q);
        uv_step(c, t, U, V);
        uv_step(c, t, U, V);
        psi_apply(psi_prep<T, D>(c, U), bSP, bSQ, P, Q);  // adjoint Psi with U^{n+1}
    } else if (MODE == RED_FUSED) {
        // this pass's integer pipes have room (one Psi weight): its V
        // additions can run there, both in 1D/2D, one in 3D
        uv_step<T, INT_ADD || INT_ADD1>(c, uv_src(c, BSU, P, Q), U, V);  // adjoint (U,V) with |Psi^n|^2
        const PsiPrep<T> pp = psi_prep<T, D>(c, U);
        psi_apply(pp, bSP, bSQ, P, Q);              // adjoint Psi with U^{n+1}
        psi_apply(pp, bSP, bSQ, P, Q);              // next base Psi: same U, same r
        uv_step<T, INT_ADD>(c, uv_src(c, BSU, P, Q), U, V);  // next base (U,V)
    } else if (MODE == RED_ADJ) {
        uv_step(c, uv_src(c, BSU, P, Q), U, V);
        psi_apply(psi_prep<T, D>(c, U), bSP, bSQ, P, Q);
    } else if (MODE == PSI_HALF) {
        psi_apply(psi_prep<T, D>(c, U), bSP, bSQ, P, Q);
    } else {  // UV_HALF
        uv_step(c, uv_src(c, BSU, P, Q), U, V);
    }
}

// Colour parity: a point is red when its 1-based index sum is odd, i.e. when
// the 0-based sum plus d is odd.  parity_of(colour) is the 0-based sum's parity.
__host__ __device__ __forceinline__ int red_parity(int dim) { return (dim + 1) & 1; }

}  // namespace kgs
