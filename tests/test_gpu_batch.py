"""Batched instances through the C ABI (kgs_batch_*): each instance of a mixed
batch (dimensions, sizes, parameters, precisions) is bitwise equal to the same
problem stepped alone, for uniform and per-instance step counts, graph replay,
and arena reuse after removals."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2502_09537_b300.inputs import Problem, random_state  # noqa: E402
from paper_2502_09537_b300.solver import (KGS_BATCH_OPT_GRAPH, KGS_FP32, KGS_FP64,  # noqa: E402
                                          Batch, KGSError, Solver)

MIX = [
    (Problem(2, 130, 40.0, 1.3, 0.7, 1.1, 0.9, 5e-4), KGS_FP64),
    (Problem(3, 22, 20.0, 0.6, 1.9, 0.8, 1.5, 5e-4), KGS_FP64),
    (Problem(2, 64, 40.0, 1.9, 1.2, 0.6, 0.7, 5e-4), KGS_FP32),
    (Problem(1, 1030, 80.0, 1.0, 1.0, 1.0, 1.0, 1e-3), KGS_FP64),
    (Problem(3, 34, 20.0, 1.7, 0.5, 1.4, 1.2, 5e-4), KGS_FP32),
    (Problem(2, 256, 40.0, 0.5, 0.9, 1.3, 1.9, 5e-4), KGS_FP64),
    (Problem(2, 4, 3.0, 1.0, 1.0, 1.0, 1.0, 1e-2), KGS_FP64),
]


def solo(prob, precision, st, nsteps):
    with Solver.from_problem(prob, precision) as s:
        s.set_state(*[a.copy() for a in st])
        s.step(nsteps)
        return s.get_state(), s.invariants()


def test_batch_equals_solo_runs():
    states = [random_state(p, 500 + k, 0.6) for k, (p, _) in enumerate(MIX)]
    with Batch(1 << 28) as b:
        ids = [b.add(p, prec) for p, prec in MIX]
        for i, st in zip(ids, states):
            b.set_state(i, *[a.copy() for a in st])
        b.step(12)
        b.step(12)          # replays the captured graph
        for i, (p, prec), st in zip(ids, MIX, states):
            want, inv = solo(p, prec, st, 24)
            got = b.get_state(i)
            for x, y in zip(got, want):
                assert np.array_equal(x, y)
            assert b.invariants(i) == inv


@pytest.mark.parametrize("graph", [0, 1])
def test_batch_per_instance_step_counts(graph):
    counts = [5, 0, 17, 1, 9, 17, 3]
    states = [random_state(p, 600 + k, 0.6) for k, (p, _) in enumerate(MIX)]
    with Batch(1 << 28) as b:
        b.set_option(KGS_BATCH_OPT_GRAPH, graph)
        ids = [b.add(p, prec) for p, prec in MIX]
        for i, st in zip(ids, states):
            b.set_state(i, *[a.copy() for a in st])
        b.step_each(counts)
        for i, (p, prec), st, n in zip(ids, MIX, states, counts):
            want, _ = solo(p, prec, st, n) if n else ((tuple(st)), None)
            for x, y in zip(b.get_state(i), want):
                assert np.array_equal(x, y)


def test_batch_arena_reuse_and_budget():
    p_big = Problem(2, 512, 40.0, 1, 1, 1, 1, 5e-4)      # 8 MB in FP64
    p_small = Problem(2, 128, 40.0, 1, 1, 1, 1, 5e-4)    # 0.5 MB
    with Batch(20 << 20) as b:                            # 20 MB budget
        a = b.add(p_big)
        c = b.add(p_big)
        with pytest.raises(KGSError):
            b.add(p_big)                                  # over budget
        b.remove(a)
        d = b.add(p_small)                                # fits in the hole
        assert d == a                                     # index reused
        e = b.add(p_small)
        st = random_state(p_small, 7, 0.5)
        b.set_state(d, *[x.copy() for x in st])
        b.set_state(e, *[x.copy() for x in st])
        b.set_state(c, *[x.copy() for x in random_state(p_big, 8, 0.5)])
        b.step(6)
        want, _ = solo(p_small, KGS_FP64, st, 6)
        for got in (b.get_state(d), b.get_state(e)):
            for x, y in zip(got, want):
                assert np.array_equal(x, y)
        assert b.free_bytes() > 0


def test_autotuned_options_are_bitwise_neutral():
    """Whatever the tuner picks, the state is the default's, bit for bit."""
    from paper_2502_09537_b300 import tune
    prob = Problem(3, 40, 20.0, 1.0, 1.0, 1.0, 1.0, 5e-4)
    st = random_state(prob, 9, 0.5)
    for prec in (KGS_FP64, KGS_FP32):
        opts = tune.Tuner(None).tune(prob, prec, nsteps=4)
        want, _ = solo(prob, prec, st, 9)
        with Solver.from_problem(prob, prec) as s:
            tune.apply(s, opts)
            s.set_state(*[a.copy() for a in st])
            s.step(9)
            for x, y in zip(s.get_state(), want):
                assert np.array_equal(x, y)


def test_tuned_batch_lists_are_bitwise_the_defaults():
    """The 96-instance batch specification with every N divided by 8 (even,
    >= 8): the autotuner's per-list CTAs per SM (timed on the GPU) leave every
    instance's state bitwise that of the library defaults."""
    from paper_2502_09537_b300 import inputs, tune
    specs = []
    for p, _, _ in inputs.batched_instances():
        n = max(8, (p.N // 8) & ~1)
        specs.append((p._replace(N=n), KGS_FP64 if len(specs) % 3 else KGS_FP32))
    states = [random_state(p, 1000 + k, 0.5) for k, (p, _) in enumerate(specs)]
    results = []
    for tuned in (False, True):
        with Batch(1 << 30) as b:
            ids = [b.add(p, prec) for p, prec in specs]
            for i, st in zip(ids, states):
                b.set_state(i, *[a.copy() for a in st])
            if tuned:
                chosen = tune.Tuner(None).tune_batch_lists(b, specs, nsteps=2)
                assert set(chosen) == {"fp64_2d", "fp64_3d", "fp32_2d", "fp32_3d"}
                for i, st in zip(ids, states):  # tuning stepped them: start again
                    b.set_state(i, *[a.copy() for a in st])
            b.step(7)
            results.append([b.get_state(i) for i in ids])
    for got, want in zip(results[1], results[0]):
        for x, y in zip(got, want):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("graph", [1, 0])
def test_persistent_launch_is_bitwise_the_per_pass_launches(graph):
    """KGS_BATCH_OPT_PERSISTENT: a step call is one cooperative launch running
    every colour pass of every instance (both precisions, 1D/2D/3D, per-instance
    step counts, a 4-point grid) with a grid barrier between passes; every
    instance's state is bitwise that of the per-pass launches, on repeated
    calls (graph replay) and after a change of step counts (a new graph)."""
    from paper_2502_09537_b300.solver import KGS_BATCH_OPT_PERSISTENT
    states = [random_state(p, 700 + k, 0.6) for k, (p, _) in enumerate(MIX)]
    plans = [[5, 0, 17, 1, 9, 17, 3], [4, 4, 4, 4, 4, 4, 4]]
    results = []
    for persistent in (0, 1):
        with Batch(1 << 28) as b:
            b.set_option(KGS_BATCH_OPT_GRAPH, graph)
            b.set_option(KGS_BATCH_OPT_PERSISTENT, persistent)
            ids = [b.add(p, prec) for p, prec in MIX]
            for i, st in zip(ids, states):
                b.set_state(i, *[a.copy() for a in st])
            l0 = b.launch_count
            b.step_each(plans[0])
            b.step_each(plans[0])
            b.step_each(plans[1])
            if persistent:
                assert b.launch_count - l0 == 3   # one launch per call
            results.append([b.get_state(i) for i in ids])
    for got, want in zip(results[1], results[0]):
        for x, y in zip(got, want):
            assert np.array_equal(x, y)


def test_persistent_launch_barrier_timeout_is_reported():
    """The test hook makes the persistent launch's grid barrier wait for CTAs
    that do not exist: the wait ends after its 2 s limit, every CTA leaves,
    the batch reports KGS_ERR_TIMEOUT from its next call on, and a new batch
    steps correctly."""
    from paper_2502_09537_b300.solver import (KGS_BATCH_OPT_PERSISTENT, KGS_BATCH_OPT_TEST_STALL,
                                              KGS_ERR_TIMEOUT)
    p, prec = MIX[1]
    st = random_state(p, 77, 0.5)
    with Batch(1 << 26) as b:
        b.set_option(KGS_BATCH_OPT_PERSISTENT, 1)
        b.set_option(KGS_BATCH_OPT_TEST_STALL, 1)
        i = b.add(p, prec)
        b.set_state(i, *[a.copy() for a in st])
        b.step(3)
        with pytest.raises(KGSError) as ei:
            b.invariants(i)
        assert ei.value.status == KGS_ERR_TIMEOUT
    want, _ = solo(p, prec, st, 3)
    with Batch(1 << 26) as b:
        b.set_option(KGS_BATCH_OPT_PERSISTENT, 1)
        i = b.add(p, prec)
        b.set_state(i, *[a.copy() for a in st])
        b.step(3)
        for x, y in zip(b.get_state(i), want):
            assert np.array_equal(x, y)
