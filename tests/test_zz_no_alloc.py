"""kgs_invariants_noalloc through the C ABI against the handle-based
kgs_invariants, on two calls in a row.

The allocation-free entry point serves callers that cannot allocate device
memory where they need the energy (their GPU memory is owned by their own
arena or budget, or they cannot pay cudaMalloc's implicit synchronisation, or
they cannot create a kgs handle, whose creation allocates).  Its reduction
scratch is one fixed array inside libkgs shared by every call, so the second
call here uses a smaller grid than the first: a stale partial sum left by the
first call would show up as a wrong result.  Tolerance: the one the other
invariant tests use (1e-13 of the energy's absolute-term scale).

This file is named to be collected last.
"""
import ctypes

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2502_09537_b300.inputs import Problem, random_state  # noqa: E402
from paper_2502_09537_b300.solver import Solver, load_library  # noqa: E402

KGS_ERR_RANGE = -7
KGS_NOALLOC_MAX_POINTS = 33554432
TOL = 1e-13


def noalloc_invariants(lib, prob, dev, stream):
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.kgs_invariants_noalloc(prob.dim, prob.N, prob.L, prob.kappa1, prob.kappa2, prob.mu,
                                    prob.gamma, *[d.data_ptr() for d in dev], out.data_ptr(),
                                    stream.cuda_stream)
    assert st == 0, lib.kgs_last_error()
    stream.synchronize()
    return out.cpu().tolist()


def handle_invariants(prob, dev, stream):
    with Solver.from_problem(prob) as s:
        s.set_state(*dev, stream=stream)
        return s.invariants(stream=stream)


def test_noalloc_matches_handle_invariants_twice():
    lib = load_library()
    stream = torch.cuda.Stream()
    cases = [Problem(2, 1024, 40.0, 1.0, 1.2, 0.9, 1.1, 1e-3),   # 256 partial triples
             Problem(3, 24, 10.0, -0.4, 0.1, 0.1, 0.2, 1e-2)]    # then 4
    for k, prob in enumerate(cases):
        st = random_state(prob, 900 + k, 0.7)
        dev = [torch.from_numpy(a).cuda() for a in st]
        torch.cuda.synchronize()
        want = handle_invariants(prob, dev, stream)
        got = noalloc_invariants(lib, prob, dev, stream)
        scale = want[1]
        assert abs(got[0] - want[0]) <= TOL * scale, (k, got, want)
        assert abs(got[1] - want[1]) <= TOL * scale, (k, got, want)
        assert abs(got[2] - want[2]) <= TOL * want[2], (k, got, want)


def test_noalloc_rejects_grids_beyond_its_limit():
    lib = load_library()
    small = [torch.zeros(8, dtype=torch.float64, device="cuda") for _ in range(5)]
    N = 2048  # 2048^3 points > KGS_NOALLOC_MAX_POINTS: refused before any work
    assert N ** 3 > KGS_NOALLOC_MAX_POINTS
    st = lib.kgs_invariants_noalloc(3, N, 1.0, 1.0, 1.0, 1.0, 1.0,
                                    *[t.data_ptr() for t in small], None)
    assert st == KGS_ERR_RANGE
    assert b"limit" in lib.kgs_last_error()
    assert lib.kgs_last_status() == KGS_ERR_RANGE
