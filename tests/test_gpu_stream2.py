"""Two steps per launch (KGS_OPT_KERNEL = 8: a float32 3D step pair's four
colour passes chained plane by plane in one launch, a four-row halo staged
by TMA tensor loads) against the one-launch-per-pass kernel -- bitwise, for
grids of one, two and three tiles per axis with short last tiles, odd and
even run lengths (an odd one ends with a one-step launch) and split calls --
and against the FP64 oracle in the 3D configuration's regime; its bounded
waits report KGS_ERR_TIMEOUT without losing the context."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2502_09537_b300 import inputs  # noqa: E402
from paper_2502_09537_b300.inputs import Problem, random_state  # noqa: E402
from paper_2502_09537_b300.solver import KGS_FP32, KGS_OPT_KERNEL, Solver  # noqa: E402

STREAM2 = 8


def run(prob, st, splits, kernel, chunk=0):
    from paper_2502_09537_b300.solver import KGS_OPT_STREAM_CHUNK
    with Solver.from_problem(prob, KGS_FP32) as s:
        s.set_option(KGS_OPT_KERNEL, kernel)
        s.set_option(KGS_OPT_STREAM_CHUNK, chunk)
        s.set_state(*[np.array(a, copy=True) for a in st])
        l0 = s.launch_count
        for n in splits:
            s.step(n)
        launches = s.launch_count - l0
        return s.get_state(), s.invariants(), launches


@pytest.mark.parametrize("N", [64, 128, 192])
@pytest.mark.parametrize("splits", [[1], [2], [7], [3, 4], [2, 2, 4]])
@pytest.mark.parametrize("chunk", [-1, 0, 5, 128])
def test_two_step_launches_are_bitwise_the_pass_kernel(N, splits, chunk):
    """N = 64, 128, 192 hold 23 + 23 + 18, 5 x 23 + 13 and 8 x 23 + 8 rows
    of tiles; chunk -1: contiguous shares, 5: ragged last chunks, 128: whole
    tile columns at N <= 128."""
    prob = Problem(3, N, 20.0, 1.1, 0.9, 1.2, 0.8, 5e-4 * (512 / N) ** 2)
    st = random_state(prob, 2502_09537 + 800 + N, 0.5)
    want, inv_want, _ = run(prob, st, [sum(splits)], 1)
    got, inv_got, _ = run(prob, st, splits, STREAM2, chunk=chunk)
    for x, y in zip(got, want):
        assert np.array_equal(x, y)
    assert inv_got == inv_want


@pytest.mark.parametrize("N", [320, 576])
def test_two_step_launches_short_last_tiles(N):
    """N = 320 = 13 x 23 + 21 and N = 576 = 25 x 23 + 1 (a last row of tiles
    one row high: its halo rows reach past both of its sides)."""
    prob = Problem(3, N, 20.0, 1.1, 0.9, 1.2, 0.8, 5e-4 * (512 / N) ** 2)
    st = random_state(prob, 2502_09537 + N, 0.5)
    want, inv_want, _ = run(prob, st, [4], 1)
    got, inv_got, _ = run(prob, st, [1, 3], STREAM2)
    for x, y in zip(got, want):
        assert np.array_equal(x, y)
    assert inv_got == inv_want


def test_launch_counts():
    """n steps: the R_base pass, the conversions in and out, n / 2 two-step
    launches and, for odd n, one one-step launch."""
    prob = Problem(3, 64, 20.0, 1.0, 1.0, 1.0, 1.0, 5e-4)
    st = random_state(prob, 2502_09537 + 811, 0.5)
    for n, want in ((6, 3 + 3), (7, 4 + 3), (1, 1 + 3), (2, 1 + 3)):
        _, _, launches = run(prob, st, [n], STREAM2)
        assert launches == want, (n, launches)


def test_two_step_launches_are_the_default_for_fp32_3d():
    """KGS_OPT_KERNEL 0 (auto) takes two steps per launch for a float32 3D
    grid it fits from N = 128: kernel 8's launch count, and bitwise the state
    of kernels 8 and 7; at N = 64 (three tiles) it makes one launch per pass."""
    prob = Problem(3, 128, 20.0, 1.0, 1.0, 1.0, 1.0, 5e-4)
    st = random_state(prob, 2502_09537 + 311, 0.5)
    runs = [run(prob, st, [6], k) for k in (0, STREAM2, 7)]
    assert runs[0][2] == runs[1][2] == 6 / 2 + 3
    assert runs[2][2] == 6 + 3
    for r in runs[1:]:
        for x, y in zip(runs[0][0], r[0]):
            assert np.array_equal(x, y)
    small = Problem(3, 64, 20.0, 1.0, 1.0, 1.0, 1.0, 5e-4)
    st = random_state(small, 2502_09537 + 312, 0.5)
    auto, pas = run(small, st, [6], 0), run(small, st, [6], 1)
    assert auto[2] == pas[2]
    for x, y in zip(auto[0], pas[0]):
        assert np.array_equal(x, y)


def test_two_step_launches_negative_kappa1_and_bumps():
    """The Sec. 5.2 parameters (kappa1 < 0) on its ellipsoid data."""
    w = inputs.paper_exp3_ellipsoids_3d(64, 0.01, 9)
    want, _, _ = run(w.prob, w.state, [9], 1)
    got, _, _ = run(w.prob, w.state, [9], STREAM2)
    for x, y in zip(got, want):
        assert np.array_equal(x, y)


def test_two_step_launches_fp32_within_rounding_bound_of_oracle(orc):
    """The 3D configuration's data and tau/h^2 = 0.328 at N = 128 over its 200
    steps through this kernel against the FP64 oracle, bounded by
    (1 + 4 n) u A (u = 2^-24, A the run's measured amplification of a
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
        s.set_option(KGS_OPT_KERNEL, STREAM2)
        s.set_state(*[np.array(a, copy=True) for a in w.state])
        E0, S0, _ = s.invariants()
        s.step(200)
        E1, S1, _ = s.invariants()
        got = s.get_state()
    e = errs(got, ref)
    drift = abs(E1 - E0) / max(S0, S1)
    bound = (1 + 4 * 200) * u * A
    print(f"two-step fp32 N=128: per field {['%.2e' % x for x in e]}, drift {drift:.2e}, bound {bound:.2e}")
    assert max(e) <= bound and drift <= bound


def test_two_step_wait_timeout_is_reported_and_the_context_survives():
    """The test hook makes every CTA wait once on a barrier that nothing
    completes: the wait ends after its 2 s limit, the CTA waits for its own
    loads in flight and leaves, the handle reports KGS_ERR_TIMEOUT, and a new
    handle still works."""
    from paper_2502_09537_b300.solver import KGS_ERR_TIMEOUT, KGS_OPT_TEST_BARRIER_STALL, KGSError
    prob = Problem(3, 64, 20.0, 1.0, 1.0, 1.0, 1.0, 5e-4)
    st = random_state(prob, 2502_09537 + 810, 0.5)
    with Solver.from_problem(prob, KGS_FP32) as s:
        s.set_option(KGS_OPT_KERNEL, STREAM2)
        s.set_option(KGS_OPT_TEST_BARRIER_STALL, 1)
        s.set_state(*[np.array(a, copy=True) for a in st])
        s.step(2)
        with pytest.raises(KGSError) as ei:
            s.invariants()
        assert ei.value.status == KGS_ERR_TIMEOUT
    want, _, _ = run(prob, st, [4], 1)
    got, _, _ = run(prob, st, [4], STREAM2)
    for x, y in zip(got, want):
        assert np.array_equal(x, y)


def test_largest_grid_both_streamed_kernels_are_the_pass_kernel():
    """N = 1024, the largest grid the streamed kernels take (4.3e9 float4 of
    packed state, tensor-map strides of 8.7 GB per colour): two and three
    steps (one two-step launch; two and one), compared on the device with the
    pass kernel's state bit for bit.  Inputs are drawn on the device; one
    handle exists at a time (about 61 GB each with the packed copies)."""
    N = 1024
    prob = Problem(3, N, 20.0, 1.1, 0.9, 1.2, 0.8, 5e-4 * (512 / N) ** 2)
    g = torch.Generator(device="cuda")
    g.manual_seed(2502_09537 + N)
    init = [0.5 * (torch.rand((N,) * 3, dtype=torch.float64, device="cuda", generator=g) - 0.5)
            for _ in range(4)]

    def final(kernel, nsteps):
        out = [torch.empty_like(a) for a in init]
        with Solver.from_problem(prob, KGS_FP32) as s:
            s.set_option(KGS_OPT_KERNEL, kernel)
            s.set_state(*init)
            s.step(nsteps)
            s.get_state(out)
            torch.cuda.synchronize()
        return out

    for nsteps in (2, 3):
        want = final(1, nsteps)
        for kernel in (STREAM2, 7):
            got = final(kernel, nsteps)
            for x, y in zip(got, want):
                assert torch.equal(x, y), (kernel, nsteps)
            del got
        del want
        torch.cuda.empty_cache()
