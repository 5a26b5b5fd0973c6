"""Pins of the FP64 CPU oracle against what arXiv 2502.09537 and mathematics fix.

None of these tests compares the oracle with itself re-typed.  Each pin is an
independent statement:
  * the semi-discrete ODE of Eq. (kgs-semi), integrated here with classical RK4:
    one DP-AVF2 step must agree with its exact flow to local order 3 (the
    composition of Eq. dp-comp is second order);
  * energy conservation for every update order (Lemma 3.1, Thm. 3.1, Eq. dp-comp),
    including the 4x4 order printed in the figure of Sec. 4.1;
  * order independence within a colour (Sec. 4.2): bitwise identical results;
  * time symmetry of the composition (Eq. dp-comp): tau then -tau returns the
    initial state;
  * the kappa1 = kappa2 = 0 closed form: pointwise phase rotation of Psi and the
    implicit-midpoint (Cayley) rotation of the (U,V) oscillator;
  * an exact standing soliton of Eq. (kgs), convergence order 2;
  * the energy's gradient term: summation by parts (Sec. 2) against the
    matrix form of E_h, and a single Fourier mode in closed form.
A final test plants each of five plausible mistakes in the oracle and checks that
at least one pin fails for every one of them.
"""
import math
import os

import numpy as np
import pytest

from paper_2502_09537_b300.inputs import Problem, coords, random_state

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers --
def lap_h(X, h):
    """Central-difference Laplacian of Sec. 2 on the periodic grid."""
    out = -2 * X.ndim * X
    for a in range(X.ndim):
        out = out + np.roll(X, 1, a) + np.roll(X, -1, a)
    return out / (h * h)


def kgs_semi_rhs(prob, z):
    """Right side of the semi-discrete system Eq. (kgs-semi)."""
    P, Q, U, V = z
    h = prob.h
    return np.array([
        -(prob.kappa1 / 2) * lap_h(Q, h) - prob.gamma * U * Q,
        (prob.kappa1 / 2) * lap_h(P, h) + prob.gamma * U * P,
        V,
        prob.kappa2 * lap_h(U, h) - prob.mu ** 2 * U + prob.gamma * (P * P + Q * Q),
    ])


def rk4_flow(prob, z, T, substeps):
    dt = T / substeps
    for _ in range(substeps):
        k1 = kgs_semi_rhs(prob, z)
        k2 = kgs_semi_rhs(prob, z + dt / 2 * k1)
        k3 = kgs_semi_rhs(prob, z + dt / 2 * k2)
        k4 = kgs_semi_rhs(prob, z + dt * k3)
        z = z + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return z


def copy_state(st):
    return tuple(np.array(a, dtype=np.float64, copy=True) for a in st)


def make_order(orc, kind, dim, N, seed=0):
    M = N ** dim
    if kind == "checkerboard":
        return orc.checkerboard_order(dim, N, True)
    if kind == "black_first":
        return orc.checkerboard_order(dim, N, False)
    if kind == "lexicographic":
        return np.arange(M, dtype=np.int64)
    if kind == "reverse":
        return np.arange(M, dtype=np.int64)[::-1].copy()
    if kind == "random":
        return np.random.Generator(np.random.PCG64(seed)).permutation(M).astype(np.int64)
    raise ValueError(kind)


def fig_ex_order():
    pts = np.loadtxt(os.path.join(GOLDEN, "fig_ex_order.txt"), dtype=np.int64, comments="#")
    return ((pts[:, 0] - 1) * 4 + (pts[:, 1] - 1)).astype(np.int64)


SMALL = {1: 16, 2: 8, 3: 6}


def local_error_ratio(orc, dim, kind="checkerboard", mut=0, taus=(0.02, 0.01, 0.005)):
    N = SMALL[dim]
    errs = []
    for tau in taus:
        prob = Problem(dim, N, 2 * math.pi * 1.3, 0.9, 1.1, 0.8, 1.2, tau)
        st = random_state(prob, 7, 0.5)
        ref = rk4_flow(prob, np.array(st), tau, 400)
        P, Q, U, V = copy_state(st)
        orc.steps_order(prob, P, Q, U, V, make_order(orc, kind, dim, N, 3), 1, mut)
        errs.append(np.abs(np.array([P, Q, U, V]) - ref).max())
    return errs[0] / errs[1], errs[1] / errs[2]


def energy_drift(orc, prob, st, order, nsteps, chunk, mut=0):
    P, Q, U, V = copy_state(st)
    E0, S0, _ = orc.invariants(prob, P, Q, U, V)
    worst = 0.0
    done = 0
    while done < nsteps:
        n = min(chunk, nsteps - done)
        orc.steps_order(prob, P, Q, U, V, order, n, mut)
        done += n
        E, S, _ = orc.invariants(prob, P, Q, U, V)
        # E_h has no fixed sign and the state may grow, so the error is taken
        # relative to the larger absolute-term scale of the two states.
        worst = max(worst, abs(E - E0) / max(S0, S))
    return worst


# Energy bar: the increment-form oracle stays below 2e-14 over 10^4 steps on
# every case here (a round-off random walk); 1e-13 leaves a margin of 5.
ENERGY_BAR = 1e-13


# ------------------------------------------------------------- the pins --
@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("kind", ["checkerboard", "lexicographic", "random"])
def test_local_error_order_three_vs_semidiscrete_flow(orc, dim, kind):
    """One DP-AVF2 step vs the exact flow of Eq. (kgs-semi): error ratio 8 per
    halving of tau (local order 3 of a second-order method, Eq. dp-comp)."""
    r1, r2 = local_error_ratio(orc, dim, kind)
    assert 7.0 < r1 < 9.0 and 7.0 < r2 < 9.0, (r1, r2)


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("kind", ["checkerboard", "black_first", "lexicographic",
                                  "reverse", "random"])
def test_energy_conserved_any_order(orc, dim, kind):
    """Thm. 3.1 and the composition theorem: E_h is conserved to round-off for
    every grid-point order, over 10^4 steps."""
    N = SMALL[dim]
    prob = Problem(dim, N, 2 * math.pi, 1.0, 1.0, 1.0, 1.0, 0.05)
    st = random_state(prob, 11 + dim, 0.6)
    drift = energy_drift(orc, prob, st, make_order(orc, kind, dim, N, 5), 10_000, 1000)
    assert drift <= ENERGY_BAR, drift


def test_energy_conserved_exp3_parameters(orc):
    """Negative kappa1 (Sec. 5.2 parameters): still conserved to round-off."""
    prob = Problem(3, 6, 20.0, -0.4, 0.1, 0.1, 0.2, 0.02)
    st = random_state(prob, 3, 0.8)
    drift = energy_drift(orc, prob, st, make_order(orc, "checkerboard", 3, 6), 10_000, 2000)
    assert drift <= ENERGY_BAR, drift


def test_energy_conserved_fig_ex_order(orc):
    """The 4x4 general order of the figure in Sec. 4.1 runs explicitly and
    conserves E_h."""
    order = fig_ex_order()
    assert sorted(order.tolist()) == list(range(16))
    prob = Problem(2, 4, 4.0, 1.0, 1.0, 1.0, 1.0, 0.1)
    st = random_state(prob, 21, 0.7)
    assert energy_drift(orc, prob, st, order, 10_000, 1000) <= ENERGY_BAR


@pytest.mark.parametrize("dim,N", [(1, 32), (2, 10), (3, 6)])
def test_within_colour_order_is_bitwise_irrelevant(orc, dim, N):
    """Sec. 4.2: no red point depends on another red point, so any order inside
    each colour gives bitwise the same result."""
    prob = Problem(dim, N, 7.0, 1.0, 1.3, 0.7, 1.1, 0.03)
    st = random_state(prob, 5, 0.5)
    base = orc.checkerboard_order(dim, N, True)
    half = base.size // 2
    rng = np.random.Generator(np.random.PCG64(9))
    shuffled = np.concatenate([rng.permutation(base[:half]), rng.permutation(base[half:])])
    a = copy_state(st)
    b = copy_state(st)
    orc.steps_order(prob, *a, base, 25)
    orc.steps_order(prob, *b, shuffled, 25)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    c = copy_state(st)
    orc.steps_checkerboard(prob, *c, 25)
    for x, y in zip(a, c):
        assert np.array_equal(x, y)


def test_colour_order_matters(orc):
    """Red-first and black-first are two different schemes (Sec. 4.2 fixes
    red first): results differ beyond round-off, while both conserve E_h."""
    prob = Problem(2, 8, 6.0, 1.0, 1.0, 1.0, 1.0, 0.05)
    st = random_state(prob, 5, 0.5)
    a = copy_state(st)
    b = copy_state(st)
    orc.steps_order(prob, *a, orc.checkerboard_order(2, 8, True), 10)
    orc.steps_order(prob, *b, orc.checkerboard_order(2, 8, False), 10)
    assert max(np.abs(x - y).max() for x, y in zip(a, b)) > 1e-6


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_time_reversible(orc, dim):
    """Eq. (dp-comp) is a symmetric composition: n steps with tau followed by n
    steps with -tau return the initial state up to round-off."""
    N = SMALL[dim]
    prob = Problem(dim, N, 5.0, 1.0, 1.0, 1.0, 1.0, 0.02)
    back = prob._replace(tau=-prob.tau)
    st = random_state(prob, 13, 0.5)
    s = copy_state(st)
    order = orc.checkerboard_order(dim, N, True)
    orc.steps_order(prob, *s, order, 50)
    assert max(np.abs(x - y).max() for x, y in zip(s, st)) > 1e-3
    orc.steps_order(back, *s, order, 50)
    assert max(np.abs(x - y).max() for x, y in zip(s, st)) < 1e-12


def kappa_zero_closed_form(prob, st, nsteps):
    """Exact DP-AVF2 solution when kappa1 = kappa2 = 0: points decouple.
    Psi: (i + g U) Psi' = (i - g U) Psi  =>  Psi' = Psi exp(2 i atan(g U)).
    (U,V): implicit midpoint for u'=v, v'=-mu^2 u + gamma|Psi|^2, i.e. the
    complex z = mu (U - U*) + i V, U* = gamma|Psi|^2/mu^2, is multiplied by
    exp(-2 i atan(mu s / 2)) per half step.  The base half uses U before its
    (U,V) update, the adjoint half U after it."""
    s = prob.tau / 2
    g = s * prob.gamma / 2
    P0, Q0, U0, V0 = st
    psi = P0 + 1j * Q0
    rho = np.abs(psi) ** 2
    ustar = prob.gamma * rho / prob.mu ** 2
    z0 = prob.mu * (U0 - ustar) + 1j * V0
    rot = np.exp(-2j * math.atan(prob.mu * s / 2))

    def U_after(m):  # U after m half-step (U,V) updates
        return (z0 * rot ** m).real / prob.mu + ustar

    phase = np.zeros_like(P0)
    for n in range(nsteps):
        phase += np.arctan(g * U_after(2 * n)) + np.arctan(g * U_after(2 * n + 2))
    psi_n = psi * np.exp(2j * phase)
    zn = z0 * rot ** (2 * nsteps)
    return psi_n.real, psi_n.imag, zn.real / prob.mu + ustar, zn.imag


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_kappa_zero_closed_form(orc, dim):
    N = SMALL[dim]
    prob = Problem(dim, N, 3.0, 0.0, 0.0, 0.9, 1.3, 0.07)
    st = random_state(prob, 17, 0.8)
    s = copy_state(st)
    orc.steps_checkerboard(prob, *s, 200)
    exact = kappa_zero_closed_form(prob, st, 200)
    for x, y in zip(s, exact):
        assert np.abs(x - y).max() < 1e-12


def soliton(prob, t):
    """Standing soliton of Eq. (kgs), kappas = mu = gamma = 1 (substitution
    gives omega = 1/2, B = 3/4, A^2 = 9/8):
    psi = (3 sqrt2 / 4) sech^2(x/2) e^{i t/2}, u = (3/4) sech^2(x/2), u_t = 0."""
    (x,) = coords(prob)
    s = 1.0 / np.cosh(x / 2) ** 2
    a = 3 * math.sqrt(2) / 4
    return a * s * math.cos(t / 2), a * s * math.sin(t / 2), 0.75 * s, 0.0 * s


def soliton_errors(orc, kind, Ns, tau_of_h, L=60.0, T=1.0):
    errs = []
    for N in Ns:
        h = L / N
        n = int(round(T / tau_of_h(h)))
        prob = Problem(1, N, L, 1.0, 1.0, 1.0, 1.0, T / n)
        st = copy_state(soliton(prob, 0.0))
        order = orc.checkerboard_order(1, N) if kind == "checkerboard" else np.arange(N)
        orc.steps_order(prob, *st, order, n)
        ex = soliton(prob, T)
        errs.append(max(np.abs(a - b).max() for a, b in zip(st, ex)))
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)], errs


def test_standing_soliton_order_two_checkerboard(orc):
    """Checkerboard order with tau ~ h^3: order 2 in h (its error has a
    (tau/h^2)^2 term, so tau ~ h does not converge)."""
    orders, errs = soliton_errors(orc, "checkerboard", [64, 128, 256, 512], lambda h: h ** 3 / 4)
    assert all(1.9 < o < 2.2 for o in orders), (orders, errs)
    assert errs[-1] < 1e-3


def test_standing_soliton_order_two_lexicographic(orc):
    orders, errs = soliton_errors(orc, "lexicographic", [64, 128, 256, 512], lambda h: h * h / 2)
    assert all(1.9 < o < 2.2 for o in orders), (orders, errs)


def _laplacian_matrix_1d(N):
    D = -2 * np.eye(N)
    for j in range(N):
        D[j, (j + 1) % N] += 1
        D[j, (j - 1) % N] += 1
    return D


@pytest.mark.parametrize("dim,N", [(1, 7), (2, 5), (3, 4)])
def test_energy_matches_matrix_form(orc, dim, N):
    """E_h of Sec. 2 in matrix form, 1/2(-k1 p'Dp - k1 q'Dq - k2 u'Du + v'v +
    mu^2 u'u) - gamma (p^2+q^2)'u with D the Kronecker-sum Laplacian, times h^d,
    equals the oracle's forward-difference form (summation by parts)."""
    prob = Problem(dim, N, 3.3, 0.7, 1.9, 1.3, 0.8, 0.1)
    h = prob.h
    D1 = _laplacian_matrix_1d(N) / h ** 2
    I1 = np.eye(N)
    D = np.zeros((N ** dim, N ** dim))
    for a in range(dim):
        term = np.ones((1, 1))
        for b in range(dim):
            term = np.kron(term, D1 if a == b else I1)
        D += term
    st = random_state(prob, 23, 0.9)
    p, q, u, v = (x.reshape(-1) for x in st)
    E = 0.5 * (-prob.kappa1 * p @ D @ p - prob.kappa1 * q @ D @ q - prob.kappa2 * u @ D @ u
               + v @ v + prob.mu ** 2 * u @ u) - prob.gamma * (p * p + q * q) @ u
    E *= h ** dim
    E_orc, S_orc, M_orc = orc.invariants(prob, *st)
    assert abs(E - E_orc) <= 1e-12 * S_orc
    assert abs(M_orc - h ** dim * np.sum(p * p + q * q)) <= 1e-13 * M_orc


def test_energy_fourier_mode_closed_form(orc):
    """P = cos(2 pi m x / L), Q = U = V = 0 in 1D: sum_j h |grad_h P|^2 equals
    (2N/h) sin^2(pi m/N), so E_h = kappa1 N sin^2(pi m/N) / h; and constants
    P = a, U = b give E_h = L (mu^2 b^2 / 2 - gamma a^2 b)."""
    N, L, m = 24, 5.0, 3
    prob = Problem(1, N, L, 1.7, 1.0, 0.6, 0.9, 0.1)
    (x,) = coords(prob)
    P = np.cos(2 * math.pi * m * x / L)
    Z = np.zeros(N)
    E, _, _ = orc.invariants(prob, P, Z.copy(), Z.copy(), Z.copy())
    assert E == pytest.approx(prob.kappa1 * N * math.sin(math.pi * m / N) ** 2 / prob.h, rel=1e-13)
    a, b = 0.8, -1.3
    E2, _, M2 = orc.invariants(prob, np.full(N, a), Z.copy(), np.full(N, b), Z.copy())
    assert E2 == pytest.approx(L * (prob.mu ** 2 * b * b / 2 - prob.gamma * a * a * b), rel=1e-13)
    assert M2 == pytest.approx(L * a * a, rel=1e-14)


def test_openmp_twin_is_bitwise_serial(orc):
    prob = Problem(2, 32, 9.0, 1.0, 1.0, 1.0, 1.0, 0.01)
    st = random_state(prob, 31, 0.5)
    a = copy_state(st)
    b = copy_state(st)
    orc.steps_checkerboard(prob, *a, 30)
    orc.steps_checkerboard_omp(prob, *b, 30, 4)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_mass_is_a_diagnostic_only(orc):
    """The paper claims no mass conservation; the scheme changes h^d sum |Psi|^2
    by far more than round-off while E_h stays exact."""
    prob = Problem(1, 64, 20.0, 1.0, 1.0, 1.0, 1.0, 0.05)
    st = random_state(prob, 2, 0.8)
    s = copy_state(st)
    E0, S0, M0 = orc.invariants(prob, *s)
    orc.steps_checkerboard(prob, *s, 200)
    E1, _, M1 = orc.invariants(prob, *s)
    assert abs(E1 - E0) / S0 < 1e-13
    assert abs(M1 - M0) / M0 > 1e-8


# ----------------------------------------------- planted mistakes caught --
MUTANTS = {
    "adjoint uses U^n on its right side (printed Eq. scheme1-adj)": 1,
    "adjoint half not reversed": 2,
    "base (U,V) uses |Psi^n|^2": 4,
    "Laplacian diagonal fixed at the 2D value": 8,
    "adjoint keeps the base variable order": 16,
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistakes_are_caught(orc, name):
    mut = MUTANTS[name]
    failures = []
    for dim in (1, 3):
        r1, r2 = local_error_ratio(orc, dim, "checkerboard", mut)
        if not (7.0 < r1 < 9.0 and 7.0 < r2 < 9.0):
            failures.append(f"local order dim={dim}: {r1:.2f} {r2:.2f}")
    prob = Problem(2, 8, 2 * math.pi, 1.0, 1.0, 1.0, 1.0, 0.05)
    st = random_state(prob, 13, 0.6)
    drift = energy_drift(orc, prob, st, make_order(orc, "checkerboard", 2, 8), 400, 100, mut)
    if drift > ENERGY_BAR:
        failures.append(f"energy drift {drift:.2e}")
    assert failures, f"planted mistake '{name}' passed every pin"
