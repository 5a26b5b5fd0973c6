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
// Increment form keeps each update's rounding proportional to the increment;
// the direct form drifts E_h by about one ulp per step.
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

// Half-step coefficients in the state precision (computed on the host in FP64).
template <typename T> struct Coef {
    T beta, alpha, g;
    T B, E, twoA, As;
    T s, hs, inv_det;
};

// ------------------------------------------------- rounded arithmetic --
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rcp_(double a) { return __drcp_rn(a); }
__device__ __forceinline__ float rcp_(float a) { return __frcp_rn(a); }

// --------------------------------------------------------- pointwise --
template <typename T> __device__ __forceinline__ T r_of(const Coef<T>& c, T u)
{
    return fma_(-c.g, u, c.alpha);
}

template <typename T> __device__ __forceinline__ T inv_of(T r)
{
    return rcp_(fma_(r, r, T(1)));
}

// Psi <- Psi + dPsi for a given r and inv = 1 / (1 + r^2).
template <typename T>
__device__ __forceinline__ void psi_step(const Coef<T>& c, T r, T inv, T SP, T SQ, T& P, T& Q)
{
    T r2 = add_(r, r);
    T nre = fma_(r2, P, -mul_(c.beta, SP));
    T nim = fma_(r2, Q, -mul_(c.beta, SQ));
    T dP = mul_(fma_(-r, nre, nim), inv);
    T dQ = -mul_(fma_(r, nim, nre), inv);
    P = add_(P, dP);
    Q = add_(Q, dQ);
}

// t = B SU + E rho: the part of the (U,V) right side fixed by the neighbours and |Psi|^2.
template <typename T> __device__ __forceinline__ T uv_src(const Coef<T>& c, T SU, T P, T Q)
{
    T rho = fma_(P, P, mul_(Q, Q));
    return fma_(c.B, SU, mul_(c.E, rho));
}

template <typename T> __device__ __forceinline__ void uv_step(const Coef<T>& c, T t, T& U, T& V)
{
    T rhs = fma_(-c.twoA, U, fma_(-c.As, V, t));
    T dV = mul_(rhs, c.inv_det);
    T dU = fma_(c.hs, dV, mul_(c.s, V));
    U = add_(U, dU);
    V = add_(V, dV);
}

// The four kinds of colour pass of a checkerboard DP-AVF2 run
// (Algorithm 3: per step red-base, black-base, black-adjoint, red-adjoint).
// Black-base and black-adjoint see the same red neighbours, so they fuse;
// red-adjoint of step n and red-base of step n+1 see the same black
// neighbours, so they fuse too.  A run of n steps is
//   RED_BASE, (BLACK_FUSED, RED_FUSED) x (n-1), BLACK_FUSED, RED_ADJ.
enum PassMode { RED_BASE = 0, BLACK_FUSED = 1, RED_FUSED = 2, RED_ADJ = 3 };

// Update one point of the pass's colour in registers.  SP, SQ, SU are the
// neighbour sums (neighbours are of the other colour and fixed for the pass).
template <typename T, int MODE>
__device__ __forceinline__ void update_point(const Coef<T>& c, T SP, T SQ, T SU,
                                             T& P, T& Q, T& U, T& V)
{
    if (MODE == RED_BASE) {
        T r = r_of(c, U);
        psi_step(c, r, inv_of(r), SP, SQ, P, Q);
        uv_step(c, uv_src(c, SU, P, Q), U, V);
    } else if (MODE == BLACK_FUSED) {
        T r = r_of(c, U);
        psi_step(c, r, inv_of(r), SP, SQ, P, Q);   // base Psi with U^n
        T t = uv_src(c, SU, P, Q);                 // |Psi^{n+1}|^2 = the adjoint's |Psi^n|^2
        uv_step(c, t, U, V);                       // base (U,V)
        uv_step(c, t, U, V);                       // adjoint (U,V)
        T r2 = r_of(c, U);
        psi_step(c, r2, inv_of(r2), SP, SQ, P, Q); // adjoint Psi with U^{n+1}
    } else if (MODE == RED_FUSED) {
        uv_step(c, uv_src(c, SU, P, Q), U, V);     // adjoint (U,V) with |Psi^n|^2
        T r = r_of(c, U);
        T inv = inv_of(r);
        psi_step(c, r, inv, SP, SQ, P, Q);         // adjoint Psi with U^{n+1}
        psi_step(c, r, inv, SP, SQ, P, Q);         // next step's base Psi: same U, same r
        uv_step(c, uv_src(c, SU, P, Q), U, V);     // base (U,V)
    } else {  // RED_ADJ
        uv_step(c, uv_src(c, SU, P, Q), U, V);
        T r = r_of(c, U);
        psi_step(c, r, inv_of(r), SP, SQ, P, Q);
    }
}

// Colour parity: a point is red when its 1-based index sum is odd, i.e. when
// the 0-based sum plus d is odd.  parity_of(colour) is the 0-based sum's parity.
__host__ __device__ __forceinline__ int red_parity(int dim) { return (dim + 1) & 1; }

}  // namespace kgs
