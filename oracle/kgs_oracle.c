/*
 * kgs_oracle.c -- plain FP64 CPU oracle of the DP-AVF2 scheme for the periodic
 * Klein-Gordon-Schroedinger (KGS) equations (arXiv 2502.09537).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load or call this file.  It shares no code,
 * header, table or helper with the CUDA library, and the library never calls it.
 *
 * What it computes, section by section of the paper:
 *   - State: the four real grid functions P = Re psi, Q = Im psi, U, V = U_t of
 *     Eq. (kgs-semi) on the periodic grid x_j = a + (j-1) h, h = L/N (Sec. 2).
 *     Arrays are C-ordered with shape N^d, index [ix][iy][iz] (the paper's
 *     linear index i = (j-1)N + k, Sec. 2).
 *   - One pointwise Psi update: the first equation of Eq. (scheme1), written
 *     for a step s and dimension d, solved as a complex scalar division (in
 *     increment form, see orc_psi_update):
 *         (i - alpha + g U*) Psi' = (i + alpha - g U*) Psi - beta * sum_nb Psi
 *     with alpha = d s kappa1/(2h^2), beta = s kappa1/(2h^2), g = s gamma/2.
 *     U* is the U value stored at the point when the update runs: U^n in the
 *     base scheme (Eq. scheme1) and U^{n+1} in the adjoint (Eq. dp-avf-kj-adj;
 *     the printed Eq. scheme1-adj shows U^n on its right side, which breaks the
 *     energy identity of Thm. 3.1 -- see the reading recorded with the tests).
 *   - One pointwise (U,V) update: the last two equations of Eq. (scheme1),
 *         U' - (s/2) V' = U + (s/2) V
 *         A U'  + V'    = V - A U + B sum_nb U + s gamma |Psi|^2
 *     with A = d s kappa2/h^2 + s mu^2/2, B = s kappa2/h^2; the constant 2x2
 *     system is reduced once in advance (Algorithm 1, first step) to one
 *     scalar division per point (see orc_uv_update).  |Psi|^2 is the value
 *     stored at the point when the update runs: Psi^{n+1} in the base scheme,
 *     Psi^n in the adjoint (Eq. scheme1-adj).
 *   - One DP-AVF2 step = Phi*_{tau/2} o Phi_{tau/2} (Eq. dp-comp): an in-place
 *     forward sweep over the update order doing (Psi, then U,V) at each point,
 *     then an in-place sweep over the reversed order doing (U,V, then Psi)
 *     (Algorithm 1).  In-place storage supplies the S/W/E/N level flags of
 *     Eq. (LapP) from the actual update order (Sec. 4.1).
 *   - Checkerboard order (Sec. 4.2, Algorithm 3): red points are those whose
 *     1-based index sum is odd; the base half sweeps red then black, the
 *     adjoint half black then red.
 *   - Discrete energy (Sec. 2, E_h; Eq. ene-origin), written with forward
 *     differences via summation by parts and weighted by h^d, and the discrete
 *     mass h^d sum |Psi|^2 (the norm of Sec. 2).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (oracle/build.py).
 * -ffp-contract=off keeps every product and sum rounded as written.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Deliberate mistakes a test may plant in the oracle to show that the pins
 * catch them (bit mask; 0 = the scheme as the paper defines it). */
#define ORC_MUT_ADJ_LITERAL   1  /* adjoint Psi: U^n on the right side (printed Eq. scheme1-adj) */
#define ORC_MUT_NO_REVERSE    2  /* adjoint half swept in the forward order */
#define ORC_MUT_RHO_OLD_BASE  4  /* base (U,V) uses |Psi^n|^2 instead of |Psi^{n+1}|^2 */
#define ORC_MUT_ALPHA_2D      8  /* Laplacian diagonal fixed at the 2D value 4 instead of 2d */
#define ORC_MUT_NO_ADJ_SWAP  16  /* adjoint half keeps the base variable order (Psi, then U,V) */
#define ORC_MUT_COLOUR_0BASED 32 /* colour rule on 0-based indices: red = 0-based index sum odd */

typedef struct {
    int dim;
    int64_t N, M;
    int64_t stride[3];
    double alpha, beta, g;     /* Psi equation */
    double A, B, E;            /* (U,V) equations */
    double half_s;             /* s/2 */
    double det;                /* determinant 1 + A s/2 of [[1, -s/2], [A, 1]] */
    int mut;
} orc_ctx;

static void orc_setup(orc_ctx* c, int dim, int64_t N, double L, double kappa1,
                      double kappa2, double mu, double gamma, double s, int mut)
{
    double h = L / (double)N;
    double h2 = h * h;
    int lapdiag = (mut & ORC_MUT_ALPHA_2D) ? 2 : dim;
    c->dim = dim;
    c->N = N;
    c->M = 1;
    for (int a = 0; a < dim; ++a) c->M *= N;
    /* axis 0 is slowest: stride[a] = N^(dim-1-a) */
    for (int a = 0; a < 3; ++a) c->stride[a] = 0;
    {
        int64_t st = 1;
        for (int a = dim - 1; a >= 0; --a) { c->stride[a] = st; st *= N; }
    }
    c->alpha = (double)lapdiag * s * kappa1 / (2.0 * h2);
    c->beta = s * kappa1 / (2.0 * h2);
    c->g = s * gamma / 2.0;
    c->A = (double)dim * s * kappa2 / h2 + s * mu * mu / 2.0;
    c->B = s * kappa2 / h2;
    c->E = s * gamma;
    c->half_s = s / 2.0;
    c->det = 1.0 + c->A * c->half_s;
    c->mut = mut;
}

/* Linear indices of the 2d periodic nearest neighbours of point i. */
static int orc_neighbours(const orc_ctx* c, int64_t i, int64_t nb[6])
{
    int n = 0;
    for (int a = 0; a < c->dim; ++a) {
        int64_t st = c->stride[a];
        int64_t coord = (i / st) % c->N;
        int64_t up = (coord + 1 == c->N) ? i - (c->N - 1) * st : i + st;
        int64_t dn = (coord == 0) ? i + (c->N - 1) * st : i - st;
        nb[n++] = dn;
        nb[n++] = up;
    }
    return n;
}

/* Psi update at point i (first equation of Eq. scheme1 / scheme1-adj):
 *     (i - r_l) Psi' = (i + r_r) Psi - beta S,   r = alpha - g U*,
 * S the sum of the neighbours' Psi.  Subtracting (i - r_l) Psi from both sides
 * gives the increment form solved here (the delta_t^+ form of Eq. dp-avf-kj):
 *     (i - r_l) dPsi = (r_l + r_r) Psi - beta S,   Psi' = Psi + dPsi.
 * Both sides use the same U* (r_l = r_r) unless a test plants the printed
 * Eq. scheme1-adj.  Solving for the increment keeps the rounding of each update
 * proportional to the (small) increment; solving the direct form for Psi' adds
 * a rounding bias of about one unit in the last place of E_h per step. */
static void orc_psi_update(const orc_ctx* c, int64_t i, double* P, double* Q,
                           double u_lhs, double u_rhs)
{
    int64_t nb[6];
    int n = orc_neighbours(c, i, nb);
    double complex sum = 0.0;
    for (int t = 0; t < n; ++t) sum += P[nb[t]] + I * Q[nb[t]];
    double complex psi = P[i] + I * Q[i];
    double r_l = c->alpha - c->g * u_lhs;
    double r_r = c->alpha - c->g * u_rhs;
    double complex dpsi = ((r_l + r_r) * psi - c->beta * sum) / (I - r_l);
    P[i] = P[i] + creal(dpsi);
    Q[i] = Q[i] + cimag(dpsi);
}

/* (U,V) update at point i (last two equations of Eq. scheme1 / scheme1-adj),
 * with rho = |Psi|^2 supplied by the caller.  In increment form
 * (dU = U' - U, dV = V' - V; the delta_t^+ form of Eq. dp-avf-kj):
 *     dU = s V + (s/2) dV
 *     dV = B sum_nb U - 2 A U - A dU + s gamma rho
 * Eliminating dU leaves the scalar equation
 *     (1 + A s/2) dV = B sum_nb U - 2 A U - A s V + s gamma rho,
 * whose coefficient 1 + A s/2 is the determinant of the constant 2x2 matrix
 * [[1, -s/2], [A, 1]] of Eq. scheme1, computed once in advance. */
static void orc_uv_update(const orc_ctx* c, int64_t i, double* U, double* V, double rho)
{
    int64_t nb[6];
    int n = orc_neighbours(c, i, nb);
    double sum = 0.0;
    for (int t = 0; t < n; ++t) sum += U[nb[t]];
    double s = 2.0 * c->half_s;
    double rhs = c->B * sum - 2.0 * c->A * U[i] - c->A * s * V[i] + c->E * rho;
    double dV = rhs / c->det;
    double dU = s * V[i] + c->half_s * dV;
    U[i] = U[i] + dU;
    V[i] = V[i] + dV;
}

static double orc_rho(const double* P, const double* Q, int64_t i)
{
    return P[i] * P[i] + Q[i] * Q[i];
}

/* Base scheme Phi_s at one point: Psi first (with U^n), then (U,V) with |Psi^{n+1}|^2. */
static void orc_base_point(const orc_ctx* c, int64_t i, double* P, double* Q, double* U, double* V)
{
    double rho_old = orc_rho(P, Q, i);
    orc_psi_update(c, i, P, Q, U[i], U[i]);
    double rho = (c->mut & ORC_MUT_RHO_OLD_BASE) ? rho_old : orc_rho(P, Q, i);
    orc_uv_update(c, i, U, V, rho);
}

/* Adjoint scheme Phi*_s at one point: (U,V) first with |Psi^n|^2, then Psi with U^{n+1}. */
static void orc_adjoint_point(const orc_ctx* c, int64_t i, double* P, double* Q, double* U, double* V)
{
    if (c->mut & ORC_MUT_NO_ADJ_SWAP) {
        orc_psi_update(c, i, P, Q, U[i], U[i]);
        orc_uv_update(c, i, U, V, orc_rho(P, Q, i));
        return;
    }
    double u_old = U[i];
    orc_uv_update(c, i, U, V, orc_rho(P, Q, i));
    double u_rhs = (c->mut & ORC_MUT_ADJ_LITERAL) ? u_old : U[i];
    orc_psi_update(c, i, P, Q, U[i], u_rhs);
}

/* nsteps DP-AVF2 steps over an arbitrary update order (a permutation of 0..M-1),
 * in place (Algorithm 1). */
void orc_steps_order(int dim, int64_t N, double L, double kappa1, double kappa2,
                     double mu, double gamma, double tau,
                     double* P, double* Q, double* U, double* V,
                     const int64_t* order, int64_t nsteps, int mut)
{
    orc_ctx c;
    orc_setup(&c, dim, N, L, kappa1, kappa2, mu, gamma, tau / 2.0, mut);
    for (int64_t n = 0; n < nsteps; ++n) {
        for (int64_t t = 0; t < c.M; ++t)
            orc_base_point(&c, order[t], P, Q, U, V);
        if (c.mut & ORC_MUT_NO_REVERSE) {
            for (int64_t t = 0; t < c.M; ++t)
                orc_adjoint_point(&c, order[t], P, Q, U, V);
        } else {
            for (int64_t t = c.M - 1; t >= 0; --t)
                orc_adjoint_point(&c, order[t], P, Q, U, V);
        }
    }
}

/* 1 if point i is red: its 1-based index sum is odd (Algorithm 3). */
/* nsteps DP-AVF2 steps with a separate update order for Psi (order_psi) and
 * for (U,V) (order_uv), in place.  The remark after Eq. dp-avf-kj-adj allows
 * different orders per variable; Algorithm 1 states the pointwise procedure
 * for one common order.  Reading: a point's Psi update reads U only at that
 * point and its (U,V) update reads Psi only at that point, so Algorithm 1's
 * per-point interleaving over one order equals two whole sweeps -- every Psi
 * update in the order (with U^n), then every (U,V) update in the order (with
 * |Psi^{n+1}|^2) -- and per-variable orders are those two sweeps in their own
 * orders.  The adjoint half reverses both: the (U,V) sweep over order_uv
 * reversed (with the |Psi|^2 the base half left), then the Psi sweep over
 * order_psi reversed (with U^{n+1}).  With order_psi == order_uv this is
 * orc_steps_order exactly (the same updates with the same inputs). */
static void orc_psi_sweep(const orc_ctx* c, const int64_t* order, int forward, double* P, double* Q,
                          const double* U)
{
    for (int64_t k = 0; k < c->M; ++k) {
        const int64_t i = order[forward ? k : c->M - 1 - k];
        orc_psi_update(c, i, P, Q, U[i], U[i]);
    }
}

static void orc_uv_sweep(const orc_ctx* c, const int64_t* order, int forward, const double* P,
                         const double* Q, double* U, double* V)
{
    for (int64_t k = 0; k < c->M; ++k) {
        const int64_t i = order[forward ? k : c->M - 1 - k];
        orc_uv_update(c, i, U, V, orc_rho(P, Q, i));
    }
}

void orc_steps_orders2(int dim, int64_t N, double L, double kappa1, double kappa2,
                       double mu, double gamma, double tau,
                       double* P, double* Q, double* U, double* V,
                       const int64_t* order_psi, const int64_t* order_uv, int64_t nsteps, int mut)
{
    orc_ctx c;
    orc_setup(&c, dim, N, L, kappa1, kappa2, mu, gamma, tau / 2.0, mut);
    for (int64_t n = 0; n < nsteps; ++n) {
        orc_psi_sweep(&c, order_psi, 1, P, Q, U);      /* base half: Psi with U^n */
        orc_uv_sweep(&c, order_uv, 1, P, Q, U, V);     /* then (U,V) with |Psi^{n+1}|^2 */
        if (c.mut & ORC_MUT_NO_ADJ_SWAP) {             /* planted: adjoint keeps Psi first */
            orc_psi_sweep(&c, order_psi, 0, P, Q, U);
            orc_uv_sweep(&c, order_uv, 0, P, Q, U, V);
        } else {
            orc_uv_sweep(&c, order_uv, 0, P, Q, U, V);  /* adjoint: (U,V) with |Psi^n|^2 */
            orc_psi_sweep(&c, order_psi, 0, P, Q, U);   /* then Psi with U^{n+1} */
        }
    }
}

/* Colour of point i (Sec. 4.2 figures; Algorithm 3's test on (j + k)): red
 * when the sum of its 1-based indices is odd.  The planted mistake
 * ORC_MUT_COLOUR_0BASED sums 0-based indices instead (the same colouring in
 * 2D, the opposite one in 1D and 3D). */
static int orc_is_red(const orc_ctx* c, int64_t i, int mut)
{
    int64_t s = 0;
    int base = (mut & ORC_MUT_COLOUR_0BASED) ? 0 : 1;
    for (int a = 0; a < c->dim; ++a) s += (i / c->stride[a]) % c->N + base;
    return (int)(s & 1);
}

/* Fill order[0..M) with the checkerboard order: the first colour's points in
 * lexicographic order, then the other colour's.  red_first = 1 gives the
 * paper's order (red first in the base half); mut may plant
 * ORC_MUT_COLOUR_0BASED. */
void orc_checkerboard_order_mut(int dim, int64_t N, int red_first, int mut, int64_t* order)
{
    orc_ctx c;
    orc_setup(&c, dim, N, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0);
    int64_t k = 0;
    for (int pass = 0; pass < 2; ++pass) {
        int want_red = (pass == 0) ? red_first : !red_first;
        for (int64_t i = 0; i < c.M; ++i)
            if (orc_is_red(&c, i, mut) == want_red) order[k++] = i;
    }
}

void orc_checkerboard_order(int dim, int64_t N, int red_first, int64_t* order)
{
    orc_checkerboard_order_mut(dim, N, red_first, 0, order);
}

/* nsteps DP-AVF2 steps in the checkerboard order (red first), serial. */
void orc_steps_checkerboard(int dim, int64_t N, double L, double kappa1, double kappa2,
                            double mu, double gamma, double tau,
                            double* P, double* Q, double* U, double* V, int64_t nsteps)
{
    int64_t M = 1;
    for (int a = 0; a < dim; ++a) M *= N;
    int64_t* order = (int64_t*)malloc((size_t)M * sizeof(int64_t));
    if (!order) return;
    orc_checkerboard_order(dim, N, 1, order);
    orc_steps_order(dim, N, L, kappa1, kappa2, mu, gamma, tau, P, Q, U, V, order, nsteps, 0);
    free(order);
}

/* The same checkerboard steps with the points of one colour split over
 * OpenMP threads.  Points of one colour have no neighbour of their own colour
 * (N even), so each colour's updates are independent of one another and the
 * result is bitwise the serial one; a test checks that on every run. */
void orc_steps_checkerboard_omp(int dim, int64_t N, double L, double kappa1, double kappa2,
                                double mu, double gamma, double tau,
                                double* P, double* Q, double* U, double* V,
                                int64_t nsteps, int nthreads)
{
    orc_ctx c;
    orc_setup(&c, dim, N, L, kappa1, kappa2, mu, gamma, tau / 2.0, 0);
    int64_t* order = (int64_t*)malloc((size_t)c.M * sizeof(int64_t));
    if (!order) return;
    orc_checkerboard_order(dim, N, 1, order);
    int64_t half = c.M / 2;
    const int64_t* red = order;
    const int64_t* black = order + half;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int64_t n = 0; n < nsteps; ++n) {
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < half; ++t) orc_base_point(&c, red[t], P, Q, U, V);
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < half; ++t) orc_base_point(&c, black[t], P, Q, U, V);
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < half; ++t) orc_adjoint_point(&c, black[t], P, Q, U, V);
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < half; ++t) orc_adjoint_point(&c, red[t], P, Q, U, V);
    }
    free(order);
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Discrete invariants, accumulated in long double:
 *   out[0] = E_h  = h^d sum [ 1/2 ( kappa1 |grad_h Psi|^2 + kappa2 |grad_h U|^2
 *                                   + V^2 + mu^2 U^2 ) - gamma |Psi|^2 U ]
 *            with grad_h the forward difference (Sec. 2; summation by parts
 *            turns -X^T D X into sum |grad_h X|^2);
 *   out[1] = S_E  = h^d sum of the absolute value of each term above (a scale
 *            for relative energy errors, since E_h has no fixed sign);
 *   out[2] = mass = h^d sum |Psi|^2 (the discrete norm of Sec. 2). */
void orc_invariants(int dim, int64_t N, double L, double kappa1, double kappa2,
                    double mu, double gamma,
                    const double* P, const double* Q, const double* U, const double* V,
                    double* out)
{
    orc_ctx c;
    orc_setup(&c, dim, N, L, 0.0, 0.0, 0.0, 0.0, 0.0, 0);
    double h = L / (double)N;
    long double hd = 1.0L;
    for (int a = 0; a < dim; ++a) hd *= (long double)h;
    long double e = 0.0L, scale = 0.0L, mass = 0.0L;
    for (int64_t i = 0; i < c.M; ++i) {
        int64_t nb[6];
        orc_neighbours(&c, i, nb);
        long double gp = 0.0L, gu = 0.0L;
        for (int a = 0; a < dim; ++a) {
            int64_t j = nb[2 * a + 1]; /* +e_a neighbour */
            long double dp = (long double)P[j] - P[i];
            long double dq = (long double)Q[j] - Q[i];
            long double du = (long double)U[j] - U[i];
            gp += dp * dp + dq * dq;
            gu += du * du;
        }
        long double hh = (long double)h * h;
        long double t1 = 0.5L * kappa1 * gp / hh;
        long double t2 = 0.5L * kappa2 * gu / hh;
        long double t3 = 0.5L * (long double)V[i] * V[i];
        long double t4 = 0.5L * (long double)mu * mu * U[i] * U[i];
        long double rho = (long double)P[i] * P[i] + (long double)Q[i] * Q[i];
        long double t5 = (long double)gamma * rho * U[i];
        e += t1 + t2 + t3 + t4 - t5;
        scale += fabsl(t1) + fabsl(t2) + t3 + t4 + fabsl(t5);
        mass += rho;
    }
    out[0] = (double)(e * hd);
    out[1] = (double)(scale * hd);
    out[2] = (double)(mass * hd);
}
