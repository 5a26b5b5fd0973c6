"""The benchmark's roofline accounting, on the CPU: FP64-pipe flops per
point-update as the colour passes issue them, the algorithmic flop and byte
counts, and which launches carry an ncu traffic figure.  These are hand counts
of the pointwise code (kgs_point.cuh: update_point), pinned here so that a
change of the kernels' arithmetic has to change them too."""
import argparse
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_fp64_pipe_flops_per_point_update(bench):
    # black pass: 2 prepares (FMA r = alpha - g U: 2 flops each), 2 Psi applies
    # (6 FMAs: 12), one (U,V) source (mul + 2 FMAs: 5), two (U,V) steps (3 FMAs
    # + 1 add: 7) = 47; red pass: 1 prepare, 2 applies, 2 sources, 2 steps = 50,
    # less the V additions that run on the integer pipes (2 in 1D/2D, 1 in 3D)
    assert bench.flops_per_point_update(1) == (47 + 48) / 2
    assert bench.flops_per_point_update(2) == 47.5
    assert bench.flops_per_point_update(3) == 48.0
    assert bench.flops_per_point_update_unfused(2) == 52


def test_algorithmic_counts(bench):
    # neighbour sums 3(2d - 1) + 57.5 (beta S, B' S_U, prepares, applies, sources, steps)
    assert bench.algorithmic_flops_per_point_update(2) == 66.5
    assert bench.algorithmic_flops_per_point_update(3) == 72.5
    # read and write the four fields once per step
    assert bench.bytes_per_point_update(8) == 64
    assert bench.bytes_per_point_update(4) == 32


def _args(**kw):
    base = dict(order="checkerboard", kernel=0, grid_n=0, workload="2d", precision="fp64")
    base.update(kw)
    return argparse.Namespace(**base)


def test_traffic_only_for_the_captured_launches(bench):
    T = bench.NCU_TRAFFIC
    assert bench.traffic_of(_args()) == T[("2d", "fp64", "pass")]
    assert bench.traffic_of(_args(kernel=1, workload="3d", precision="fp32")) == T[("3d", "fp32", "pass")]
    # auto on a float32 3D grid streams two steps per launch (kernel 8); kernel 7 one
    assert bench.kernel_name(_args(workload="3d", precision="fp32")) == "stream2"
    assert bench.kernel_name(_args(kernel=8, workload="3d", precision="fp32")) == "stream2"
    assert bench.traffic_of(_args(workload="3d", precision="fp32")) == T.get(("3d", "fp32", "stream2"))
    assert bench.traffic_of(_args(kernel=7, workload="3d", precision="fp32")) == T[("3d", "fp32", "stream")]
    assert bench.temporal_depth(_args(workload="3d", precision="fp32")) == 2
    assert bench.temporal_depth(_args(kernel=7, workload="3d", precision="fp32")) == 1
    assert bench.bytes_per_point_update(4, 2) == 16
    assert bench.kernel_name(_args(kernel=7, workload="3d", precision="fp64")) == "pass"
    assert bench.traffic_of(_args(workload="3d")) == T[("3d", "fp64", "pass")]
    assert bench.traffic_of(_args(kernel=6)) is None          # another kernel
    assert bench.traffic_of(_args(kernel=5)) is None
    assert bench.traffic_of(_args(grid_n=256)) is None        # another grid size
    assert bench.traffic_of(_args(order="lex")) is None       # another update order
    assert bench.traffic_of(_args(workload="1d")) is None     # never captured
    for v in T.values():
        assert v is None or v > 0


def test_fp64_peak_from_unit_counts(bench):
    # 148 SMs x 2 FP64 FMA lanes per cycle x 2 flops x 2032 MHz
    assert abs(bench.FP64_PEAK_TFLOPS - 1.202944) < 1e-9
