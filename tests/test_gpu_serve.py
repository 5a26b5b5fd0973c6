"""Continuous batching: results in the mix equal results alone (bitwise), with
staggered admission forced by a small memory budget and a slot cap, and
requests of different sizes, dimensions, precisions and step counts."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2502_09537_b300 import serve  # noqa: E402
from paper_2502_09537_b300.inputs import Problem, random_state  # noqa: E402
from paper_2502_09537_b300.solver import KGS_FP32, KGS_FP64, Solver  # noqa: E402


def make_requests():
    specs = [
        (Problem(2, 96, 40.0, 1.2, 0.8, 1.1, 0.9, 5e-4), KGS_FP64, 37),
        (Problem(3, 20, 20.0, 0.7, 1.6, 0.8, 1.4, 5e-4), KGS_FP32, 11),
        (Problem(1, 600, 80.0, 1.0, 1.0, 1.0, 1.0, 1e-3), KGS_FP64, 53),
        (Problem(2, 64, 40.0, 1.9, 1.1, 0.6, 0.7, 5e-4), KGS_FP32, 29),
        (Problem(3, 16, 20.0, 1.5, 0.6, 1.2, 1.1, 5e-4), KGS_FP64, 8),
        (Problem(2, 130, 40.0, 0.6, 0.9, 1.4, 1.8, 5e-4), KGS_FP64, 64),
        (Problem(2, 48, 40.0, 1.0, 1.0, 1.0, 1.0, 5e-4), KGS_FP64, 5),
        (Problem(3, 24, 20.0, 1.1, 1.3, 0.9, 0.6, 5e-4), KGS_FP32, 21),
    ]
    reqs = []
    for k, (p, prec, n) in enumerate(specs):
        st = random_state(p, 800 + k, 0.5)
        reqs.append(serve.Request(k, p, n, lambda st=st: tuple(a.copy() for a in st), prec, 0.0))
    return reqs


def solo(req):
    with Solver.from_problem(req.prob, req.precision) as s:
        s.set_state(*req.state())
        s.step(req.nsteps)
        return s.get_state()


@pytest.mark.parametrize("budget,slots,quantum,turn_work", [(1 << 30, 64, 10, 0.0), (700_000, 3, 7, 0.0),
                                                              (1 << 30, 64, 10, 2e5)])
def test_results_in_the_mix_equal_results_alone(budget, slots, quantum, turn_work):
    reqs = make_requests()
    srv = serve.Server(budget, quantum=quantum, max_slots=slots, turn_work=turn_work, max_wait=0.5)
    for r in reqs:
        srv.submit(r)
    results = srv.run()
    srv.close()
    assert sorted(r.rid for r in results) == list(range(len(reqs)))
    if slots == 3:
        # the small budget forced later admissions: some request was admitted
        # after another had completed
        first_done = min(r.finished for r in results)
        assert any(r.admitted >= first_done for r in results)
    by_id = {r.rid: r for r in results}
    for req in reqs:
        got = by_id[req.rid].state
        for x, y in zip(got, solo(req)):
            assert np.array_equal(x, y)
        assert by_id[req.rid].energy_drift < (1e-12 if req.precision == KGS_FP64 else 1e-4)


def test_request_larger_than_the_budget_is_refused():
    from paper_2502_09537_b300.solver import KGSError
    srv = serve.Server(100_000)
    big = serve.Request(0, Problem(2, 128, 40.0, 1, 1, 1, 1, 5e-4), 10, lambda: None)
    with pytest.raises(KGSError):
        srv.submit(big)
    srv.close()
