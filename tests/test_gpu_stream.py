"""The streamed-plane kernel (KGS_OPT_KERNEL = 7: a float32 3D step's black
and red passes in one launch walking axis 0, planes staged by TMA tensor
loads on a packed layout with ghost copies) against the one-launch-per-pass
kernel -- bitwise, for grids of one, two and three tiles per axis, several
run lengths and split calls -- and against the FP64 oracle in the 3D
configuration's regime; its bounded waits report KGS_ERR_TIMEOUT without
losing the context; grids and precisions it does not take run the passes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2502_09537_b300 import inputs  # noqa: E402
from paper_2502_09537_b300.inputs import Problem, random_state  # noqa: E402
from paper_2502_09537_b300.solver import KGS_FP32, KGS_FP64, KGS_OPT_KERNEL, Solver  # noqa: E402

STREAM = 7


def run(prob, st, splits, kernel, precision=KGS_FP32, chunk=0):
    from paper_2502_09537_b300.solver import KGS_OPT_STREAM_CHUNK
    with Solver.from_problem(prob, precision) as s:
        s.set_option(KGS_OPT_KERNEL, kernel)
        s.set_option(KGS_OPT_STREAM_CHUNK, chunk)
        s.set_state(*[np.array(a, copy=True) for a in st])
        for n in splits:
            s.step(n)
        return s.get_state(), s.invariants()


@pytest.mark.parametrize("N", [64, 128, 192])
@pytest.mark.parametrize("splits", [[1], [2], [7], [3, 4]])
@pytest.mark.parametrize("chunk", [-1, 0, 5, 128])
def test_streamed_planes_are_bitwise_the_pass_kernel(N, splits, chunk):
    """Both work orders: contiguous shares (chunk -1) and round-robin chunks
    (the default 64 planes; a ragged last chunk for 5; whole tiles for 128
    at N <= 128)."""
    prob = Problem(3, N, 20.0, 1.1, 0.9, 1.2, 0.8, 5e-4 * (512 / N) ** 2)
    st = random_state(prob, 2502_09537 + 300 + N, 0.5)
    want, inv_want = run(prob, st, [sum(splits)], 1)
    got, inv_got = run(prob, st, splits, STREAM, chunk=chunk)
    for x, y in zip(got, want):
        assert np.array_equal(x, y)
    assert inv_got == inv_want


def test_streamed_planes_one_row_last_tile():
    """N = 320 = 11 x 29 + 1: the last row of tiles holds a single row (the
    ring rows are its neighbours on both sides; most of its box is
    zero-filled beyond the grid)."""
    prob = Problem(3, 320, 20.0, 1.1, 0.9, 1.2, 0.8, 5e-4 * (512 / 320) ** 2)
    st = random_state(prob, 2502_09537 + 320, 0.5)
    want, inv_want = run(prob, st, [3], 1)
    got, inv_got = run(prob, st, [1, 2], STREAM)
    for x, y in zip(got, want):
        assert np.array_equal(x, y)
    assert inv_got == inv_want


def test_streamed_planes_negative_kappa1_and_bumps():
    """The Sec. 5.2 parameters (kappa1 < 0) on its ellipsoid data."""
    w = inputs.paper_exp3_ellipsoids_3d(64, 0.01, 9)
    want, _ = run(w.prob, w.state, [9], 1)
    got, _ = run(w.prob, w.state, [9], STREAM)
    for x, y in zip(got, want):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("prob,precision", [
    (Problem(3, 96, 20.0, 1.0, 1.0, 1.0, 1.0, 5e-4), KGS_FP32),   # N not a multiple of 64
    (Problem(3, 64, 20.0, 1.0, 1.0, 1.0, 1.0, 5e-4), KGS_FP64),   # float64 state
    (Problem(2, 128, 40.0, 1.0, 1.0, 1.0, 1.0, 5e-4), KGS_FP32),  # 2D
])
@pytest.mark.parametrize("kernel", [STREAM, STREAM + 1])
def test_grids_it_does_not_take_run_the_passes(prob, precision, kernel):
    """Kernels 7 and 8 (one and two steps per launch) on grids neither takes."""
    st = random_state(prob, 77, 0.5)
    want, _ = run(prob, st, [5], 1, precision)
    got, _ = run(prob, st, [5], kernel, precision)
    for x, y in zip(got, want):
        assert np.array_equal(x, y)


def test_streamed_planes_fp32_within_rounding_bound_of_oracle(orc):
    """The 3D configuration's data and tau/h^2 = 0.328 at N = 128 over its 200
    steps: float32 state through this kernel against the FP64 oracle, bounded
    by (1 + 4 n) u A (u = 2^-24, A the run's measured amplification of a
    float32-sized perturbation of the initial state, at least 1)."""
    w = inputs.gauss_3d(128, 200)
    prob = w.prob._replace(tau=(5e-4 / (20.0 / 512) ** 2) * w.prob.h ** 2)
    ref = tuple(np.array(a, copy=True) for a in w.state)
    orc.steps_checkerboard_omp(prob, *ref, 200, orc.max_threads())
    pert = tuple(np.asarray(a, dtype=np.float32).astype(np.float64) for a in w.state)
    orc.steps_checkerboard_omp(prob, *pert, 200, orc.max_threads())
    u = 2.0 ** -24

    def errs(a, b):
        return [float(np.abs(x - y).max() / np.abs(y).max()) for x, y in zip(a, b)]

    A = max(1.0, max(errs(pert, ref)) / u)
    with Solver.from_problem(prob, KGS_FP32) as s:
        s.set_option(KGS_OPT_KERNEL, STREAM)
        s.set_state(*[np.array(a, copy=True) for a in w.state])
        E0, S0, _ = s.invariants()
        s.step(200)
        E1, S1, _ = s.invariants()
        got = s.get_state()
    e = errs(got, ref)
    drift = abs(E1 - E0) / max(S0, S1)
    bound = (1 + 4 * 200) * u * A
    print(f"streamed fp32 N=128: per field {['%.2e' % x for x in e]}, drift {drift:.2e}, bound {bound:.2e}")
    assert max(e) <= bound and drift <= bound


def test_streamed_planes_wait_timeout_is_reported_and_the_context_survives():
    """The test hook makes every CTA wait once on a barrier that nothing
    completes: the wait ends after its 2 s limit, the CTA waits for its own
    loads in flight and leaves, the handle reports KGS_ERR_TIMEOUT at the next
    synchronising call and from then on, and a new handle still works."""
    from paper_2502_09537_b300.solver import KGS_ERR_TIMEOUT, KGS_OPT_TEST_BARRIER_STALL, KGSError
    prob = Problem(3, 64, 20.0, 1.0, 1.0, 1.0, 1.0, 5e-4)
    st = random_state(prob, 2502_09537 + 310, 0.5)
    with Solver.from_problem(prob, KGS_FP32) as s:
        s.set_option(KGS_OPT_KERNEL, STREAM)
        s.set_option(KGS_OPT_TEST_BARRIER_STALL, 1)
        s.set_state(*[np.array(a, copy=True) for a in st])
        s.step(2)
        with pytest.raises(KGSError) as ei:
            s.invariants()
        assert ei.value.status == KGS_ERR_TIMEOUT
        with pytest.raises(KGSError) as ei:
            s.step(1)
        assert ei.value.status == KGS_ERR_TIMEOUT
    want, _ = run(prob, st, [4], 1)
    got, _ = run(prob, st, [4], STREAM)
    for x, y in zip(got, want):
        assert np.array_equal(x, y)
