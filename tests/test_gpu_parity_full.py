"""Parity with the FP64 oracle over whole configurations, for every path.

* The 2D configuration (2048^2, 1000 steps) and the 3D configuration (512^3,
  200 steps) on the GPU against the oracle's OpenMP twin (bitwise equal to the
  serial oracle, tested on the CPU), per field at the FP64 bar 1e-12 in
  max-norm after every step of the run.
* The 3D configuration's regime (tau/h^2 = 0.328) at reduced N over its 200
  steps, where the serial oracle is quick.
* FP32 state against the FP64 oracle in 3D (the reduced regime cases and the
  full 512^3 grid), bounded by what float32 rounding allows (below).
* Batched instances (kgs_batch_step) and served requests (serve.Server)
  against the oracle, instance by instance.

FP32 bound.  With u = 2^-24 (float32 unit roundoff), the FP32 path starts
from the state rounded to float32 (one rounding, u of the field's max-norm)
and each step adds an increment to every state value at most four times (two
colour passes, each a fused adjoint-then-base pair of half-updates), each
addition rounded once (u); the increments' own rounding errors are of order
tau times u and fit in the margin.  Errors injected at one step are carried
to the end by the scheme; how much the run amplifies a perturbation of the
initial state, A, is measured on the oracle itself (the same run from the
float32-rounded initial state; A = its max-norm difference / u, at least 1).
So the FP32 max-norm error per field is bounded by (1 + 4 n) u max(A, 1),
and the energy drift by the same figure (E_h is a smooth function of the
state; a relative state error e moves it by at most about 2e of S_E, and
the bound already counts every rounding as worst-case aligned).  Where the
amplification run would double a long oracle run (512^3), the A measured
on the reduced cases at the same tau/h^2 is used.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2502_09537_b300 import inputs, serve  # noqa: E402
from paper_2502_09537_b300.inputs import Problem, random_state  # noqa: E402
from paper_2502_09537_b300.solver import KGS_FP32, KGS_FP64, Batch, Solver  # noqa: E402

FP64_BAR = 1e-12
U32 = 2.0 ** -24
C3_TAU_OVER_H2 = 5e-4 / (20.0 / 512) ** 2   # 0.32768


def copy_state(st):
    return tuple(np.array(a, dtype=np.float64, copy=True) for a in st)


def field_errs(a, b):
    return [float(np.abs(x - y).max() / max(np.abs(y).max(), 1e-300)) for x, y in zip(a, b)]


def oracle_run(orc, prob, st, nsteps):
    out = copy_state(st)
    if prob.points * nsteps < 3e7:
        orc.steps_checkerboard(prob, *out, nsteps)
    else:
        orc.steps_checkerboard_omp(prob, *out, nsteps, orc.max_threads())
    return out


def gpu_run(prob, st, nsteps, precision=KGS_FP64):
    with Solver.from_problem(prob, precision) as s:
        s.set_state(*st)
        E0, S0, _ = s.invariants()
        s.step(nsteps)
        E1, S1, _ = s.invariants()
        return s.get_state(), abs(E1 - E0) / max(S0, S1)


def fp32_bound(nsteps, amplification):
    return (1 + 4 * nsteps) * U32 * max(amplification, 1.0)


def amplification(orc, prob, st, nsteps, ref):
    """How much the run amplifies a float32-sized perturbation of its initial
    state: the oracle from the float32-rounded state against ref (the oracle
    from the exact state), divided by u."""
    rounded = tuple(np.asarray(a, dtype=np.float32).astype(np.float64) for a in st)
    pert = oracle_run(orc, prob, rounded, nsteps)
    return max(field_errs(pert, ref)) / U32


# ------------------------------------------------------------------ 2D full --
def test_2d_configuration_all_1000_steps_match_oracle(orc):
    """2048^2, tau = 1e-3, 1000 steps (tau/h^2 = 2.62): every field within 1e-12
    of the oracle after the whole run."""
    w = inputs.gauss_2d(2048, 1000)
    ref = oracle_run(orc, w.prob, w.state, w.nsteps)
    got, drift = gpu_run(w.prob, copy_state(w.state), w.nsteps)
    errs = field_errs(got, ref)
    print(f"2D 2048^2 x 1000: per-field max-norm rel diff {['%.2e' % e for e in errs]}, drift {drift:.1e}")
    assert max(errs) <= FP64_BAR
    assert drift <= 1e-12


# ------------------------------------------------------ 3D regime, reduced --
@pytest.mark.parametrize("N", [64, 96])
def test_3d_regime_200_steps_fp64_and_fp32_match_oracle(orc, N):
    """The 3D configuration's data and tau/h^2 = 0.328 at N = 64 and 96, all
    200 steps: FP64 within 1e-12 per field; FP32 within its rounding bound."""
    w = inputs.gauss_3d(N, 200)
    prob = w.prob._replace(tau=C3_TAU_OVER_H2 * w.prob.h ** 2)
    ref = oracle_run(orc, prob, w.state, 200)
    got, drift = gpu_run(prob, copy_state(w.state), 200)
    errs = field_errs(got, ref)
    assert max(errs) <= FP64_BAR
    assert drift <= 1e-12
    A = amplification(orc, prob, w.state, 200, ref)
    got32, drift32 = gpu_run(prob, copy_state(w.state), 200, KGS_FP32)
    errs32 = field_errs(got32, ref)
    bound = fp32_bound(200, A)
    print(f"3D N={N} tau/h^2=0.328 x 200: fp64 {max(errs):.2e}; amplification {A:.2f}; "
          f"fp32 per field {['%.2e' % e for e in errs32]}, drift {drift32:.2e}, bound {bound:.2e}")
    assert max(errs32) <= bound
    assert drift32 <= bound


# ------------------------------------------------------------------ 3D full --
@pytest.fixture(scope="module")
def c3_full(orc):
    """The 3D configuration at full size (512^3, tau = 5e-4, 200 steps): the
    initial state and the oracle's result (OpenMP twin, a few minutes)."""
    w = inputs.gauss_3d(512, 200)
    ref = oracle_run(orc, w.prob, w.state, w.nsteps)
    return w, ref


@pytest.mark.slow
def test_3d_configuration_all_200_steps_fp64_matches_oracle(c3_full):
    w, ref = c3_full
    got, drift = gpu_run(w.prob, w.state, w.nsteps)
    errs = field_errs(got, ref)
    print(f"3D 512^3 x 200 fp64: per-field {['%.2e' % e for e in errs]}, drift {drift:.1e}")
    assert max(errs) <= FP64_BAR
    assert drift <= 1e-12


@pytest.mark.slow
def test_3d_configuration_fp32_within_rounding_bound_of_oracle(orc, c3_full):
    """FP32 state on the full 3D configuration against the FP64 oracle, with
    the amplification measured at N = 96 in the same regime (tau/h^2 = 0.328,
    200 steps; the full grid's own would double the oracle run)."""
    w, ref = c3_full
    small = inputs.gauss_3d(96, 200)
    sp = small.prob._replace(tau=C3_TAU_OVER_H2 * small.prob.h ** 2)
    sref = oracle_run(orc, sp, small.state, 200)
    A = amplification(orc, sp, small.state, 200, sref)
    got, drift = gpu_run(w.prob, w.state, w.nsteps, KGS_FP32)
    errs = field_errs(got, ref)
    bound = fp32_bound(w.nsteps, A)
    print(f"3D 512^3 x 200 fp32: per-field {['%.2e' % e for e in errs]}, drift {drift:.2e}, "
          f"bound {bound:.2e} (amplification {A:.2f})")
    assert max(errs) <= bound
    assert drift <= bound


# -------------------------------------------------------- batch and serve --
MIX = [
    (Problem(1, 1030, 80.0, 1.0, 1.0, 1.0, 1.0, 1e-3), KGS_FP64, 60),
    (Problem(2, 130, 40.0, 1.3, 0.7, 1.1, 0.9, 5e-4), KGS_FP64, 45),
    (Problem(3, 22, 20.0, 0.6, 1.9, 0.8, 1.5, 5e-4), KGS_FP64, 60),
    (Problem(3, 34, 20.0, -0.4, 0.1, 0.1, 0.2, 1e-2), KGS_FP64, 30),
    (Problem(2, 64, 40.0, 1.9, 1.2, 0.6, 0.7, 5e-4), KGS_FP32, 60),
    (Problem(3, 34, 20.0, 1.7, 0.5, 1.4, 1.2, 5e-4), KGS_FP32, 45),
    (Problem(1, 600, 80.0, 1.0, 1.0, 1.0, 1.0, 1e-3), KGS_FP32, 60),
    (Problem(2, 4, 3.0, 1.0, 1.0, 1.0, 1.0, 1e-2), KGS_FP64, 17),
]


def check_against_oracle(orc, prob, precision, st, nsteps, got):
    ref = oracle_run(orc, prob, st, nsteps)
    errs = field_errs(got, ref)
    if precision == KGS_FP64:
        assert max(errs) <= FP64_BAR, (prob, errs)
    else:
        bound = fp32_bound(nsteps, amplification(orc, prob, st, nsteps, ref))
        assert max(errs) <= bound, (prob, errs, bound)
    return max(errs)


def test_batch_instances_match_oracle(orc):
    """A mixed batch (1D/2D/3D, FP64 and FP32, negative kappa1, per-instance
    step counts) stepped by kgs_batch_step: every instance against the oracle."""
    states = [random_state(p, 900 + k, 0.6) for k, (p, _, _) in enumerate(MIX)]
    with Batch(1 << 28) as b:
        ids = [b.add(p, prec) for p, prec, _ in MIX]
        for i, st in zip(ids, states):
            b.set_state(i, *copy_state(st))
        b.step_each([n for _, _, n in MIX])
        for i, (p, prec, n), st in zip(ids, MIX, states):
            e = check_against_oracle(orc, p, prec, st, n, b.get_state(i))
            print(f"batch dim={p.dim} N={p.N} {'fp64' if prec == KGS_FP64 else 'fp32'} x {n}: {e:.2e}")


def test_served_requests_match_oracle(orc):
    """Requests served with continuous batching (a small budget and slot cap
    force staggered admission): every result against the oracle."""
    reqs = []
    for k, (p, prec, n) in enumerate(MIX):
        st = random_state(p, 950 + k, 0.5)
        reqs.append(serve.Request(k, p, n, lambda st=st: copy_state(st), prec, 0.0))
    srv = serve.Server(1_500_000, quantum=7, max_slots=3, max_wait=0.5)
    for r in reqs:
        srv.submit(r)
    results = {r.rid: r for r in srv.run()}
    srv.close()
    assert sorted(results) == list(range(len(reqs)))
    for req in reqs:
        e = check_against_oracle(orc, req.prob, req.precision, req.state(), req.nsteps,
                                 results[req.rid].state)
        print(f"serve rid={req.rid} dim={req.prob.dim}: {e:.2e}")
