"""Autotuner logic on CPU with an injected timer and fake solvers (no GPU)."""
import json

import numpy as np

from paper_2502_09537_b300 import tune
from paper_2502_09537_b300.inputs import Problem
from paper_2502_09537_b300.solver import (KGS_BATCH_OPT_CTAS_PER_SM, KGS_FP32, KGS_FP64,
                                          KGS_OPT_KERNEL, KGS_OPT_THREADS, KGS_OPT_TILE_T2)


class FakeSolver:
    def __init__(self):
        self.opts = {}

    def set_option(self, k, v):
        if k == KGS_OPT_KERNEL and v == 3 and self.opts.get("reject_tile"):
            raise RuntimeError("no")
        self.opts[k] = v

    def step(self, n, stream=None):
        pass

    def close(self):
        pass


def fake_timer_preferring(pred):
    def timer(s, n):
        return 1.0 if pred(s.opts) else 2.0
    return timer


def test_bucket_rounds_up_to_power_of_two():
    assert tune.bucket(Problem(2, 2048, 1, 1, 1, 1, 1, 1), KGS_FP64) == (2, 2048, 64)
    assert tune.bucket(Problem(3, 96, 1, 1, 1, 1, 1, 1), KGS_FP32) == (3, 128, 32)
    assert tune.bucket(Problem(1, 6, 1, 1, 1, 1, 1, 1), KGS_FP64) == (1, 8, 64)


def test_candidates_respect_shared_memory():
    p3 = Problem(3, 512, 20, 1, 1, 1, 1, 5e-4)
    for prec, elem in ((KGS_FP64, 8), (KGS_FP32, 4)):
        for o in tune.candidates(p3, prec):
            if o.get(KGS_OPT_KERNEL) == 3:
                T2 = o[KGS_OPT_TILE_T2]
                assert tune._tile_fits(3, elem, o.get(5, 1), T2, o[8], o[9])
    small = Problem(1, 512, 80, 1, 1, 1, 1, 1e-3)
    assert {KGS_OPT_KERNEL: 2} in tune.candidates(small, KGS_FP64)
    big = Problem(2, 2048, 40, 1, 1, 1, 1, 1e-3)
    assert {KGS_OPT_KERNEL: 2} not in tune.candidates(big, KGS_FP64)


def test_tuner_picks_fastest_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    prob = Problem(2, 2048, 40, 1, 1, 1, 1, 1e-3)
    t = tune.Tuner(path, timer=fake_timer_preferring(
        lambda o: o.get(KGS_OPT_KERNEL) == 1 and o.get(KGS_OPT_THREADS) == 512),
        make_solver=lambda p, prec: FakeSolver())
    best = t.tune(prob, KGS_FP64)
    assert best == {KGS_OPT_KERNEL: 1, KGS_OPT_THREADS: 512}
    saved = json.load(open(path))
    assert saved["2:2048:64"] == {"1": 1, "3": 512}
    # a new tuner reads the cache and does not time again
    t2 = tune.Tuner(path, timer=lambda s, n: 1 / 0, make_solver=lambda p, prec: FakeSolver())
    assert t2.tune(Problem(2, 1500, 40, 1, 1, 1, 1, 1e-3), KGS_FP64) == best


def test_tuner_skips_shapes_a_problem_rejects():
    def make(p, prec):
        s = FakeSolver()
        s.opts["reject_tile"] = True
        return s
    t = tune.Tuner(None, timer=fake_timer_preferring(lambda o: o.get(KGS_OPT_KERNEL) == 3),
                   make_solver=make)
    best = t.tune(Problem(3, 512, 20, 1, 1, 1, 1, 5e-4), KGS_FP32)
    assert best[KGS_OPT_KERNEL] == 1


def test_tune_batch_sets_best_cta_count():
    class FakeBatch:
        def __init__(self):
            self.c = None

        def set_option(self, k, v):
            assert k == KGS_BATCH_OPT_CTAS_PER_SM
            self.c = v

    b = FakeBatch()
    t = tune.Tuner(None)
    best = t.tune_batch(b, 10, timer=lambda bb, n: abs(bb.c - 4) + 1.0)
    assert best == 4 and b.c == 4


def test_tune_batch_lists_coordinate_descent_and_cache(tmp_path):
    """Each list (precision x dimension) of a batch gets its own CTAs per SM:
    the fake timer rewards FP64 2D lists at 4 and FP32 3D lists at 16 (each
    list's choice alone matters); the choice is set, returned and cached, and
    a second tuner reads it without timing."""
    class FakeBatch:
        def __init__(self):
            self.opt = {}
            self.steps = 0

        def set_option(self, k, v):
            self.opt[k] = v

        def step(self, n, stream=None):
            self.steps += 1

    def timer(b, n):
        return (abs(b.opt.get(tune.list_option(KGS_FP64, 2), 8) - 4)
                + abs(b.opt.get(tune.list_option(KGS_FP32, 3), 8) - 16) + 1.0)

    members = [(Problem(2, 512, 40, 1, 1, 1, 1, 5e-4), KGS_FP64),
               (Problem(2, 256, 40, 1, 1, 1, 1, 5e-4), KGS_FP64),
               (Problem(3, 64, 20, 1, 1, 1, 1, 5e-4), KGS_FP32)]
    path = str(tmp_path / "t.json")
    b = FakeBatch()
    chosen = tune.Tuner(path).tune_batch_lists(b, members, timer=timer)
    assert chosen == {"fp64_2d": 4, "fp32_3d": 16}
    assert b.opt[tune.list_option(KGS_FP64, 2)] == 4 and b.opt[tune.list_option(KGS_FP32, 3)] == 16
    assert b.steps == 8  # one warm-up call per timed value, 4 values x 2 lists
    b2 = FakeBatch()
    again = tune.Tuner(path).tune_batch_lists(b2, members, timer=lambda bb, n: 1 / 0)
    assert again == chosen and b2.opt == b.opt and b2.steps == 0
    for p, d in ((KGS_FP64, 1), (KGS_FP64, 3), (KGS_FP32, 2)):
        assert tune.list_name_of_option(tune.list_option(p, d)) == tune.list_name(p, d)


def test_serving_request_generator_matches_the_workload_shape():
    from paper_2502_09537_b300 import serve
    reqs = serve.poisson_requests(rate=50.0, count=300, seed=5)
    arr = [r.arrival for r in reqs]
    assert all(b > a for a, b in zip(arr, arr[1:]))
    gaps = np.diff([0.0] + arr)
    assert 0.5 / 50 < gaps.mean() < 2.0 / 50          # exponential, mean 1/rate
    for r in reqs:
        lo, hi = {1: (256, 8192), 2: (128, 2048), 3: (64, 384)}[r.prob.dim]
        assert lo <= r.prob.N <= hi and r.prob.N % 2 == 0
        assert 100 <= r.nsteps <= 10000
    assert {r.prob.dim for r in reqs} == {1, 2, 3}
    assert {r.precision for r in reqs} == {32, 64}
