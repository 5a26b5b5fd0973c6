"""Per-variable update orders in the oracle (the remark after Eq. dp-avf-kj-adj:
Psi and (U,V) may be updated in different orders), pinned against what the
scheme fixes: with one common order the two-sweep form is Algorithm 1's
per-point procedure exactly; with different orders the discrete energy is
still conserved (Thm. 3.1's argument is per variable) and a step with -tau
undoes a step with tau; and the planted wrong reading (the adjoint half
keeping Psi first) breaks that reversibility, so the pins have power."""
import numpy as np
import pytest

import oracle
from paper_2502_09537_b300 import orders
from paper_2502_09537_b300.inputs import Problem, random_state


def _copy(st):
    return [np.array(a, dtype=np.float64, copy=True) for a in st]


def _drift(prob, st, op, ou, nsteps, mut=0):
    s = _copy(st)
    E0, S0, _ = oracle.invariants(prob, *s)
    worst = 0.0
    for _ in range(nsteps // 100):
        oracle.steps_orders2(prob, *s, op, ou, 100, mut)
        E, S, _ = oracle.invariants(prob, *s)
        worst = max(worst, abs(E - E0) / max(S0, S))
    return worst


@pytest.mark.parametrize("dim,N", [(1, 16), (2, 8), (3, 6)])
@pytest.mark.parametrize("name", ["lex", "checkerboard", "random", "reverse"])
def test_one_common_order_is_the_interleaved_scheme(dim, N, name):
    prob = Problem(dim, N, 5.0, 1.1, 0.9, 1.2, 0.8, 0.03)
    st = random_state(prob, 2502_09537 + 300 + dim, 0.6)
    o = {"lex": orders.lexicographic(dim, N), "checkerboard": orders.checkerboard(dim, N),
         "random": orders.random_order(dim, N, 31 + dim), "reverse": orders.reverse_lexicographic(dim, N)}[name]
    a, b = _copy(st), _copy(st)
    oracle.steps_order(prob, *a, o, 25)
    oracle.steps_orders2(prob, *b, o, o, 25)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def _pair(dim, N, k):
    lex, rev = orders.lexicographic(dim, N), orders.reverse_lexicographic(dim, N)
    cb = orders.checkerboard(dim, N)
    r1, r2 = orders.random_order(dim, N, 41 + dim), orders.random_order(dim, N, 43 + dim)
    return [(lex, rev), (cb, r1), (r1, r2), (rev, cb)][k]


@pytest.mark.parametrize("dim,N", [(1, 24), (2, 10), (3, 6)])
@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_energy_conserved_with_different_orders(dim, N, k):
    prob = Problem(dim, N, 6.0, 1.0, 1.1, 0.9, 1.2, 0.05)
    st = random_state(prob, 2502_09537 + 310 + dim, 0.6)
    op, ou = _pair(dim, N, k)
    drift = _drift(prob, st, op, ou, 1000)
    assert drift <= 1e-13, drift


@pytest.mark.parametrize("dim,N", [(1, 24), (2, 10), (3, 6)])
def test_negative_tau_undoes_a_step_with_different_orders(dim, N):
    prob = Problem(dim, N, 6.0, 1.0, 1.1, 0.9, 1.2, 0.05)
    st = random_state(prob, 2502_09537 + 320 + dim, 0.6)
    op, ou = _pair(dim, N, 1)
    s = _copy(st)
    oracle.steps_orders2(prob, *s, op, ou, 40)
    moved = max(np.abs(x - y).max() for x, y in zip(s, st))
    oracle.steps_orders2(prob._replace(tau=-prob.tau), *s, op, ou, 40)
    back = max(np.abs(x - y).max() / np.abs(y).max() for x, y in zip(s, st))
    assert moved > 1e-3 and back <= 1e-12, (moved, back)


def _back(prob, st, op, ou, mut):
    s = _copy(st)
    oracle.steps_orders2(prob, *s, op, ou, 40, mut)
    oracle.steps_orders2(prob._replace(tau=-prob.tau), *s, op, ou, 40, mut)
    return max(np.abs(x - y).max() / np.abs(y).max() for x, y in zip(s, st))


def test_planted_wrong_adjoint_variable_order_breaks_reversibility():
    """Keeping Psi first in the adjoint half gives another DP-AVF scheme --
    every order conserves the energy, so that pin cannot see it -- but not
    the adjoint of the base half: the step is no longer undone by -tau."""
    prob = Problem(2, 10, 6.0, 1.0, 1.1, 0.9, 1.2, 0.05)
    st = random_state(prob, 2502_09537 + 330, 0.6)
    op, ou = _pair(2, 10, 0)
    assert _drift(prob, st, op, ou, 1000, oracle.MUT_NO_ADJ_SWAP) <= 1e-13
    assert _back(prob, st, op, ou, 0) <= 1e-12
    assert _back(prob, st, op, ou, oracle.MUT_NO_ADJ_SWAP) > 1e-3
