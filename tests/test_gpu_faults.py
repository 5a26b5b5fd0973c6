"""Out-of-memory paths, made to fail on purpose on the host: KGS_DEVICE_BUDGET
caps what one handle may allocate, so an allocation past it fails as if the
device were full -- without exhausting a shared device.  The creation that
does not fit returns NULL with KGS_ERR_OOM; a kernel option whose buffers do
not fit makes kgs_step return KGS_ERR_OOM before any work, the state stays
as it was, and the same handle steps with the plain passes afterwards."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2502_09537_b300.inputs import Problem, random_state  # noqa: E402
from paper_2502_09537_b300.solver import (KGS_FP32, KGS_OPT_KERNEL, KGSError,  # noqa: E402
                                          Solver)

KGS_ERR_OOM = -3


@pytest.fixture
def budget():
    def set_budget(nbytes):
        os.environ["KGS_DEVICE_BUDGET"] = str(int(nbytes))
    yield set_budget
    os.environ.pop("KGS_DEVICE_BUDGET", None)


def test_creation_past_the_budget_is_refused(budget):
    prob = Problem(3, 64, 20.0, 1.0, 1.0, 1.0, 1.0, 5e-4)   # 64^3 float32: 4 MB of state
    budget(1 << 20)
    with pytest.raises(KGSError) as ei:
        Solver.from_problem(prob, KGS_FP32)
    assert ei.value.status == KGS_ERR_OOM
    budget(32 << 20)   # state, staging and the streamed kernel's packed copies (~16.3 MB)
    with Solver.from_problem(prob, KGS_FP32) as s:
        s.set_state(*random_state(prob, 5, 0.5))
        s.step(2)


def test_option_buffers_past_the_budget_fail_cleanly_and_the_handle_goes_on(budget):
    """The streamed-plane kernel's two packed copies (about 10 MB at 64^3) do
    not fit in 12 MB next to the 6.4 MB of state and staging: kgs_step
    returns KGS_ERR_OOM, the state is the one set, and with one launch per
    colour pass the same handle steps bitwise as a handle without a budget."""
    prob = Problem(3, 64, 20.0, 1.0, 1.0, 1.0, 1.0, 5e-4)
    st = random_state(prob, 6, 0.5)
    budget(12 << 20)
    with Solver.from_problem(prob, KGS_FP32) as s:
        s.set_state(*[a.copy() for a in st])
        before = s.get_state()
        s.set_option(KGS_OPT_KERNEL, 7)
        with pytest.raises(KGSError) as ei:
            s.step(3)
        assert ei.value.status == KGS_ERR_OOM
        for x, y in zip(s.get_state(), before):
            assert np.array_equal(x, y)
        s.set_option(KGS_OPT_KERNEL, 1)
        s.step(3)
        got = s.get_state()
    os.environ.pop("KGS_DEVICE_BUDGET", None)
    with Solver.from_problem(prob, KGS_FP32) as s:
        s.set_option(KGS_OPT_KERNEL, 1)
        s.set_state(*[a.copy() for a in st])
        s.step(3)
        want = s.get_state()
    for x, y in zip(got, want):
        assert np.array_equal(x, y)
