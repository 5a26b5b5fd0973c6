"""Asynchronous host state transfers (KGS_HOST_ASYNC): queued on a stream,
they give bitwise the state of the synchronous calls, and two handles fed
and read on copy streams while the other computes (the end-to-end benchmark's
pipeline) give every solve's result unchanged."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2502_09537_b300.inputs import Problem, random_state  # noqa: E402
from paper_2502_09537_b300.solver import (KGS_ERR_ARG, KGS_FP32, KGS_FP64, KGSError,  # noqa: E402
                                          Solver)


def pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


def pinned_empty(shape):
    return torch.empty(shape, dtype=torch.float64).pin_memory().numpy()


@pytest.mark.parametrize("dim,N,precision", [(3, 64, KGS_FP64), (3, 64, KGS_FP32), (2, 128, KGS_FP64)])
def test_async_transfers_equal_the_synchronous_ones(dim, N, precision):
    prob = Problem(dim, N, 20.0, 1.0, 0.9, 1.1, 0.8, 5e-4)
    st = random_state(prob, 2502_09537 + 900 + N, 0.5)
    with Solver.from_problem(prob, precision) as s:
        s.set_state(*st)
        s.step(5)
        want = s.get_state()
    stream = torch.cuda.Stream()
    host_in = [pinned(a) for a in st]
    host_out = [pinned_empty(a.shape) for a in st]
    with Solver.from_problem(prob, precision) as s:
        s.set_state(*host_in, stream=stream, asynchronous=True)
        s.step(5, stream=stream)
        s.get_state(host_out, stream=stream, asynchronous=True)
        stream.synchronize()
    for x, y in zip(host_out, want):
        assert np.array_equal(x, y)


def test_two_handles_pipelined_on_copy_streams():
    """Solve i on one handle while the next input goes into the other handle
    on an upload stream and the previous result comes back on a download
    stream, ordered by events: each result equals its serial solve."""
    prob = Problem(3, 64, 20.0, 1.0, 0.9, 1.1, 0.8, 5e-4)
    inputs = [random_state(prob, 2502_09537 + 950 + i, 0.5) for i in range(4)]
    want = []
    with Solver.from_problem(prob, KGS_FP32) as s:
        for st in inputs:
            s.set_state(*st)
            s.step(7)
            want.append(s.get_state())
    comp, up, down = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    host_in = [[pinned(a) for a in st] for st in inputs]
    host_out = [[pinned_empty(a.shape) for a in st] for st in inputs]
    hs = [Solver.from_problem(prob, KGS_FP32), Solver.from_problem(prob, KGS_FP32)]
    try:
        loaded, done, read = {}, {}, {}

        def upload(i):
            h = hs[i % 2]
            if i - 2 in read:
                up.wait_event(read[i - 2])  # the handle's previous result is out
            h.set_state(*host_in[i], stream=up, asynchronous=True)
            loaded[i] = torch.cuda.Event()
            loaded[i].record(up)

        upload(0)
        for i in range(len(inputs)):
            if i + 1 < len(inputs):
                upload(i + 1)
            comp.wait_event(loaded[i])
            hs[i % 2].step(7, stream=comp)
            done[i] = torch.cuda.Event()
            done[i].record(comp)
            down.wait_event(done[i])
            hs[i % 2].get_state(host_out[i], stream=down, asynchronous=True)
            read[i] = torch.cuda.Event()
            read[i].record(down)
        down.synchronize()
    finally:
        for h in hs:
            h.close()
    for got, ref in zip(host_out, want):
        for x, y in zip(got, ref):
            assert np.array_equal(x, y)


def test_bad_where_is_refused():
    prob = Problem(2, 16, 10.0, 1.0, 1.0, 1.0, 1.0, 1e-3)
    st = random_state(prob, 5, 0.5)
    with Solver.from_problem(prob, KGS_FP64) as s:
        ptrs = [a.ctypes.data for a in st]
        assert s._lib.kgs_set_state(s._h, *ptrs, 3, None) == KGS_ERR_ARG
        with pytest.raises(KGSError):
            s.get_state()  # no state set yet
