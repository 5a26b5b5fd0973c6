"""Degenerate cases and exact structural properties of the DP-AVF2 scheme on
the GPU path (C ABI through the Python binding), each against a fact the
scheme fixes rather than against another implementation:

- the zero state is a fixed point (Eq. scheme1 with Psi = U = V = 0 has no
  source term);
- the step is time-reversible: Phi*_{tau/2} o Phi_{tau/2} with -tau is the
  inverse of the step with tau (Phi* is the adjoint of Phi, Sec. 3), so
  stepping forward then backward returns the initial state to round-off;
- a negative tau is still the same scheme (matches the oracle run with -tau);
- kappa1 = kappa2 = 0 decouples the points: the Psi update is a Cayley
  transform (i - r) Psi' = (i + r) Psi, so |Psi| is pointwise invariant;
- gamma = 0 decouples Psi from (U, V): r and the (U,V) source lose their
  coupling terms exactly, so each field's trajectory is bitwise independent
  of the other field's initial data.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2502_09537_b300.inputs import Problem, random_state  # noqa: E402
from paper_2502_09537_b300.solver import KGS_FP32, KGS_FP64, KGS_OPT_KERNEL, Solver  # noqa: E402

FP64_BAR = 1e-12


def copy_state(st):
    return [np.array(a, dtype=np.float64, copy=True) for a in st]


def run(prob, st, nsteps, precision=KGS_FP64, kernel=0):
    with Solver.from_problem(prob, precision) as s:
        s.set_option(KGS_OPT_KERNEL, kernel)
        s.set_state(*copy_state(st))
        s.step(nsteps)
        return s.get_state(), s.invariants()


def rel_err(a, b):
    return max(np.abs(x - y).max() / max(np.abs(y).max(), 1e-300) for x, y in zip(a, b))


@pytest.mark.parametrize("precision", [KGS_FP64, KGS_FP32])
@pytest.mark.parametrize("dim,N,kernel", [(1, 64, 0), (2, 66, 1), (2, 64, 6), (3, 18, 1), (3, 64, 5)])
def test_zero_state_is_a_fixed_point(dim, N, kernel, precision):
    prob = Problem(dim, N, 9.0, 1.1, 0.8, 1.3, 0.7, 0.01)
    zero = [np.zeros((N,) * dim) for _ in range(4)]
    st, inv = run(prob, zero, 25, precision, kernel)
    for a in st:
        assert not a.any()
        assert not np.signbit(a).any()
    assert inv == (0.0, 0.0, 0.0)


@pytest.mark.parametrize("dim,N,tau", [(1, 128, 2e-3), (2, 48, 1e-2), (3, 16, 5e-3)])
def test_step_with_negative_tau_inverts_the_step(dim, N, tau):
    prob = Problem(dim, N, 8.0, 1.2, 0.9, 1.1, 0.8, tau)
    st = random_state(prob, 2502_09537 + 200 + dim, 0.6)
    with Solver.from_problem(prob) as s:
        s.set_state(*copy_state(st))
        s.step(30)
        mid = s.get_state()
        s.set_tau(-tau)
        s.step(30)
        back = s.get_state()
    moved = rel_err(mid, st)
    err = rel_err(back, st)
    print(f"{dim}D: moved {moved:.2e}, back to {err:.2e}")
    assert moved > 1e-4           # the forward run did change the state
    assert err <= 1e-13


@pytest.mark.parametrize("dim,N", [(2, 24), (3, 10)])
def test_negative_tau_matches_oracle(orc, dim, N):
    prob = Problem(dim, N, 6.0, 0.9, 1.2, 1.0, 1.1, -0.01)
    st = random_state(prob, 2502_09537 + 210 + dim, 0.6)
    gpu, _ = run(prob, st, 40)
    ref = copy_state(st)
    orc.steps_checkerboard(prob, *ref, 40)
    assert rel_err(gpu, ref) <= FP64_BAR


@pytest.mark.parametrize("dim,N", [(1, 64), (2, 24), (3, 10)])
def test_kappa_zero_keeps_psi_modulus_pointwise(orc, dim, N):
    prob = Problem(dim, N, 6.0, 0.0, 0.0, 1.3, 0.9, 0.02)
    st = random_state(prob, 2502_09537 + 220 + dim, 0.7)
    gpu, _ = run(prob, st, 200)
    mod0 = np.hypot(st[0], st[1])
    mod1 = np.hypot(gpu[0], gpu[1])
    drift = np.abs(mod1 - mod0).max() / mod0.max()
    print(f"{dim}D kappa = 0: pointwise |Psi| drift {drift:.2e} over 200 steps")
    assert drift <= 1e-13
    ref = copy_state(st)
    orc.steps_checkerboard(prob, *ref, 200)
    assert rel_err(gpu, ref) <= FP64_BAR


@pytest.mark.parametrize("precision", [KGS_FP64, KGS_FP32])
@pytest.mark.parametrize("dim,N", [(2, 26), (3, 12)])
def test_gamma_zero_decouples_psi_from_u(dim, N, precision):
    prob = Problem(dim, N, 7.0, 1.1, 0.8, 1.2, 0.0, 0.01)
    a = random_state(prob, 2502_09537 + 230 + dim, 0.6)
    b = random_state(prob, 2502_09537 + 240 + dim, 0.6)
    psi_a_uv_b = [a[0], a[1], b[2], b[3]]
    psi_b_uv_a = [b[0], b[1], a[2], a[3]]
    ra, _ = run(prob, a, 60, precision)
    rb, _ = run(prob, b, 60, precision)
    rab, _ = run(prob, psi_a_uv_b, 60, precision)
    rba, _ = run(prob, psi_b_uv_a, 60, precision)
    # Psi follows its own initial data only, (U, V) theirs
    assert np.array_equal(rab[0], ra[0]) and np.array_equal(rab[1], ra[1])
    assert np.array_equal(rab[2], rb[2]) and np.array_equal(rab[3], rb[3])
    assert np.array_equal(rba[0], rb[0]) and np.array_equal(rba[1], rb[1])
    assert np.array_equal(rba[2], ra[2]) and np.array_equal(rba[3], ra[3])
    # and the runs did move
    assert not np.array_equal(ra[0], a[0]) and not np.array_equal(ra[2], a[2])
    assert math.isfinite(float(np.abs(ra[0]).max()))


@pytest.mark.parametrize("precision", [KGS_FP64, KGS_FP32])
def test_changing_tau_between_graph_replays(precision):
    """kgs_set_tau between two runs long enough to replay the captured step
    graph: the second run uses the new tau (bitwise what a fresh handle with
    that tau computes from the same state), not the graph's old constants."""
    prob = Problem(2, 64, 9.0, 1.1, 0.9, 1.2, 0.8, 0.01)
    st = random_state(prob, 2502_09537 + 250, 0.6)
    with Solver.from_problem(prob, precision) as s:
        s.set_state(*copy_state(st))
        s.step(40)
        mid = s.get_state()
        s.set_tau(0.004)
        s.step(40)
        got = s.get_state()
    want, _ = run(prob._replace(tau=0.004), mid, 40, precision)
    for x, y in zip(got, want):
        assert np.array_equal(x, y)
    first, _ = run(prob, st, 40, precision)
    for x, y in zip(mid, first):
        assert np.array_equal(x, y)
