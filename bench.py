#!/usr/bin/env python
"""Benchmark of the DP-AVF2 checkerboard solver (arXiv 2502.09537) on one B300.

Workload (default): the 2D KGS problem on [-20,20)^2 with N = 2048^2 points,
kappa1 = kappa2 = mu = gamma = 1, tau = 1e-3, 1000 DP-AVF2 steps in float64,
psi0 = (1+i) exp(-r^2), u0 = exp(-r^2), v0 = 0 plus seeded Gaussian noise
(sigma 1e-4); the discrete energy is evaluated every 100 steps.  One benchmark
step = one such solve: load the initial state (already in HBM), 1000 steps,
10 energy/mass evaluations.  Metric: grid-point updates per second
(N^d x steps / time).  Multi-GPU: every rank solves its own instance (the
instances are independent), value = all ranks' point-updates / max time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload 2d|1d|3d] [--precision fp64|fp32]

The reference arm (--impl reference) times the CPU oracle (oracle/, the
OpenMP checkerboard twin, bitwise equal to the serial oracle) on the host's
cores on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "point-updates/s & %HBM roofline, FP64 vs FP32 @stated err; serve p50/p99 latency"
UNIT = "point-updates/s"
ENERGY_EVERY = 100


def flops_per_point_update_unfused(dim: int) -> float:
    """FP64-pipe flops of one point-update in a general order (kgs_set_order):
    no fusion, every point takes one base update (prepare 2, apply 12, source
    5, step 7) and one adjoint update per step: 2 x 26 = 52."""
    return 2 * (2 + 12 + 5 + 7)


def flops_per_point_update(dim: int) -> float:
    """FP64-pipe flops of one point-update (one point, one full DP-AVF2 step)
    as the FP64 colour passes execute them (kgs_point.cuh), FMA = 2, add/mul
    = 1.  Per pass: Psi prepare r = alpha - g U (2), Psi apply 12, (U,V)
    source 5 (|Psi|^2 3, E'|Psi|^2 + B'S_U 2), one (U,V) step 7 (three FMAs
    and the V addition).  Black pass: 2 prepares + 2 applies + 1 source + 2
    steps = 47 flops (25 instructions); red pass: 1 prepare + 2 applies + 2
    sources + 2 steps = 50 (27), of which the V additions run on the integer
    pipes, both in 1D/2D (48 flops, 25 instructions), one in 3D (49, 26).  A
    point-update is the mean: 47.5 in 1D/2D, 48 in 3D.  The neighbour sums,
    beta S, B' S_U, 2r and 1/(1 + r^2) run on the integer pipes too."""
    black = 2 * 2 + 2 * 12 + 5 + 2 * 7
    red = 2 + 2 * 12 + 2 * 5 + 2 * 7 - (2 if dim <= 2 else 1)
    return (black + red) / 2


def algorithmic_flops_per_point_update(dim: int) -> float:
    """All flops of the method per point-update, wherever they run, counting
    a reciprocal as one: neighbour sums 3(2d-1), beta S 2, B' S_U 1, Psi
    prepare 6 (r 2, 2r 1, 1 + r^2 2, reciprocal 1), Psi apply 12, (U,V)
    source 5, (U,V) step 7.  Black pass 3 + 2x6 + 2x12 + 5 + 2x7 = 58, red
    pass 3 + 6 + 2x12 + 2x5 + 2x7 = 57."""
    return 3 * (2 * dim - 1) + 57.5


# DRAM bytes per launch of the dominant kernel (a fused colour pass) from the
# ncu captures summarised in profiles/ (dram__bytes_read.sum + write.sum), for
# the kernels as they are now; None where no capture of the current kernel exists.
NCU_TRAFFIC = {("2d", "fp64"): 117.52e6 + 25.74e6,     # pass_kernel_fp64_kgs2d_N2048.md (RED_FUSED)
               ("3d", "fp64"): 3.7645e9 + 2.1086e9,    # pass_kernel_fp64_kgs3d_N256.md (512^3 launch)
               ("3d", "fp32"): 1.8822e9 + 1.0321e9}    # pass_kernel_fp32_kgs3d_N512.md (512^3 launch)

def traffic_of(args):
    """DRAM bytes per pass launch from the ncu captures above: only for the
    launches they were taken on (the default one-per-pass kernel on the
    workload's full grid, checkerboard order); None otherwise."""
    if args.order != "checkerboard" or args.kernel not in (0, 1) or args.grid_n:
        return None
    return NCU_TRAFFIC.get((args.workload, args.precision))


# FP64 pipe of the B300: 2 FMA per cycle per SM (ncu: peak_sustained of
# sm__sass_thread_inst_executed_op_dfma_pred_on), 148 SMs, 2032 MHz maximum SM
# clock -> 2 x 2 x 148 x 2.032e9 = 1.203e12 flop/s.
FP64_PEAK_TFLOPS = 2 * 2 * 148 * 2.032e9 / 1e12


def bytes_per_point_update(elem: int) -> int:
    """Algorithmic HBM bytes of one point-update: read and write the four
    fields once (the two colour passes of a step each touch their own half)."""
    return 2 * 4 * elem


def make_workload(name: str, n: int = 0):
    """The benchmark configuration; n overrides the points per direction."""
    from paper_2502_09537_b300 import inputs
    if name == "2d":
        return inputs.gauss_2d(n or 2048, 1000)
    if name == "1d":
        return inputs.soliton_1d(n or 512, 2000)
    if name == "3d":
        return inputs.gauss_3d(n or 512, 200)
    raise ValueError(name)


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def cpu_baseline(work, seconds_target: float = 12.0):
    """The oracle (OpenMP checkerboard twin, all host cores) on a bounded
    sample of the workload: the full grid for a few steps."""
    import oracle
    threads = oracle.max_threads()
    st = tuple(np.array(a, copy=True) for a in work.state)
    t0 = time.perf_counter()
    oracle.steps_checkerboard_omp(work.prob, *st, 1, threads)
    t1 = time.perf_counter() - t0
    n = max(1, min(work.nsteps, int(seconds_target / max(t1, 1e-6))))
    t0 = time.perf_counter()
    oracle.steps_checkerboard_omp(work.prob, *st, n, threads)
    dt = time.perf_counter() - t0
    return {"value": work.prob.points * n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{work.name}: full grid, {n} of {work.nsteps} steps "
                      f"(OpenMP checkerboard twin, bitwise equal to the serial oracle)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    work = make_workload(args.workload)
    threads = oracle.max_threads()
    st = tuple(np.array(a, copy=True) for a in work.state)
    t0 = time.perf_counter()
    oracle.steps_checkerboard_omp(work.prob, *st, 1, threads)
    t1 = max(time.perf_counter() - t0, 1e-6)
    per_step = max(1, min(work.nsteps, int(4.0 / t1)))
    times = []
    for k in range(args.warmup + args.steps):
        st = tuple(np.array(a, copy=True) for a in work.state)
        t0 = time.perf_counter()
        oracle.steps_checkerboard_omp(work.prob, *st, per_step, threads)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = work.prob.points * per_step * len(times) / total
    sample = (f"{work.name}: full grid, {per_step} of {work.nsteps} steps per timed step "
              f"(OpenMP checkerboard twin, bitwise equal to the serial oracle)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": work.name, "dim": work.prob.dim, "N": work.prob.N,
                   "steps_per_solve": work.nsteps, "precision": "fp64", "sample_steps": per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_batch(args):
    """The 96-instance batch: 64 2D grids N in {128..2048} and 32 3D grids N in
    {64..256}, random parameters, tau = 5e-4, 500 steps, every instance in the
    chosen precision, stepped by kgs_batch_step (one launch per colour pass over
    all instances, replayed from a CUDA graph).  One benchmark step = load every
    initial state from HBM, 500 steps."""
    import torch
    from paper_2502_09537_b300 import build as kbuild
    from paper_2502_09537_b300 import inputs
    from paper_2502_09537_b300.solver import KGS_FP32, KGS_FP64, Batch
    kbuild.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    precision = KGS_FP64 if args.precision == "fp64" else KGS_FP32
    elem = 8 if precision == KGS_FP64 else 4
    specs = inputs.batched_instances()
    nsteps = specs[0][1]
    total_bytes = sum(p.points * 4 * elem for p, _, _ in specs)
    b = Batch(int(total_bytes * 1.05) + (64 << 20))
    init, ids = [], []
    for p, _, fn in specs:
        ids.append(b.add(p, precision))
        init.append([torch.from_numpy(a).cuda() for a in fn()])
    torch.cuda.synchronize()
    points = sum(p.points for p, _, _ in specs)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one():
        for i, st in zip(ids, init):
            b.set_state(i, *st, stream=stream)
        b.step(nsteps, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one()
        stream.synchronize()
        if dist:
            dist.barrier()
        times, kern = [], []
        l0 = b.launch_count
        with ClockSampler(local) as clk:
            for _ in range(args.steps):
                flush.zero_()
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(stream)
                for i, st in zip(ids, init):
                    b.set_state(i, *st, stream=stream)
                e1.record(stream)
                b.step(nsteps, stream=stream)
                e2.record(stream)
                stream.synchronize()
                times.append(e0.elapsed_time(e2))
                kern.append(e1.elapsed_time(e2))
        launches = b.launch_count - l0
    from paper_2502_09537_b300.dist import max_over_ranks
    total_ms = max_over_ranks(sum(times), device="cuda")
    value = world * points * nsteps * args.steps / (total_ms * 1e-3)
    step_launches = 2 * nsteps + 1  # one pass launch per colour pass (one precision)
    pass_ms = sum(kern) / (args.steps * step_launches)
    upd_per_launch = points * nsteps / step_launches
    peaks = measured_peaks()
    if precision == KGS_FP64:
        mean_dim_flops = sum(p.points * flops_per_point_update(p.dim) for p, _, _ in specs) / points
        achieved = upd_per_launch * mean_dim_flops / (pass_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "derived: 148 SMs x 2 FP64 FMA/cycle x 2 flops x 2032 MHz",
                "work": "FP64-pipe flops (neighbour sums, beta S, B'S_U, 2r, 1/(1+r^2) and the red pass's V additions -- both in 1D/2D, one in 3D -- run on the integer pipes)"}
    else:
        achieved = upd_per_launch * bytes_per_point_update(elem) / (pass_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks.get("hbm_gbs", 6400.0),
                "unit": "GB/s", "frac": achieved / peaks.get("hbm_gbs", 6400.0), "traffic": None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
    # end to end: host states in and out
    host_in = [[torch.from_numpy(a.cpu().numpy()).pin_memory().numpy() for a in st] for st in init]
    host_out = [[np.empty_like(a) for a in st] for st in host_in]
    with torch.cuda.stream(stream):
        stream.synchronize()
        t0 = time.perf_counter()
        for i, st in zip(ids, host_in):
            b.set_state(i, *st, stream=stream)
        b.step(nsteps, stream=stream)
        for i, out in zip(ids, host_out):
            b.get_state(i, out, stream=stream)
        e2e_s = time.perf_counter() - t0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if elem == 8 else "f32",
        "data": "synthetic",
        "config": {"workload": "kgs_batch96", "instances": len(specs), "points": points,
                   "steps_per_solve": nsteps, "precision": args.precision,
                   "l2": "256 MB buffer written between timed steps",
                   "parallelism": f"{world} independent batch(es), one per GPU"},
        "roofline": roof,
        "e2e": {"value": world * points * nsteps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": points * 32, "d2h_bytes_per_step": points * 32},
        "gpu_launches": launches, "clocks": clk.summary(),
        "kernel_ms_per_launch": pass_ms,
    }
    b.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if int(os.environ.get("RANK", "0")) == 0:
        print(json.dumps(line))


def run_serve(args):
    """Continuous-batching serving: Poisson arrivals of solve requests (dim in
    {1,2,3}, N in [256,8192] / [128,2048]^2 / [64,384]^3, steps uniform in
    [100, --max-steps], FP32 or FP64 each, parameters as the batched workload),
    admitted by a 150 GB device-memory budget, states resident on the device.
    One benchmark step = serving --requests requests from their arrival to
    their result on the host; value = point-updates/s over the step, with
    p50/p99 request latency and the worst per-request energy drift."""
    import torch
    from paper_2502_09537_b300 import build as kbuild
    from paper_2502_09537_b300 import serve
    kbuild.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    budget = 150 * (1 << 30)
    stream = torch.cuda.Stream()
    lat, pts, wall, drift_max, turns = [], 0, 0.0, 0.0, 0
    launches = 0
    with torch.cuda.stream(stream):
        with ClockSampler(local) as clk:
            for k in range(args.warmup + args.steps):
                reqs = serve.poisson_requests(args.rate, args.requests, seed=SEED_SERVE + 1000 * rank + k,
                                              step_range=(100, args.max_steps))
                srv = serve.Server(budget, quantum=100, stream=stream, keep_state=True,
                                   turn_work=args.turn_work)
                for r in reqs:
                    srv.submit(r)
                l0 = srv.batch.launch_count
                t0 = time.perf_counter()
                res = srv.run()
                dt = time.perf_counter() - t0
                if k >= args.warmup:
                    wall += dt
                    pts += srv.point_updates
                    lat += [r.latency for r in res]
                    drift_max = max(drift_max, max(r.energy_drift for r in res))
                    turns += srv.turns
                    launches += srv.batch.launch_count - l0
                srv.close()
    from paper_2502_09537_b300.dist import max_over_ranks
    wall = max_over_ranks(wall, device="cuda")
    value = world * pts / wall
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": "kgs_serve", "rate_per_s": args.rate,
                   "requests_per_step": args.requests, "step_range": [100, args.max_steps],
                   "budget_bytes": budget, "quantum_steps": 100, "turn_work": args.turn_work,
                   "l2": "inputs are built per request on the host (cold)",
                   "parallelism": f"{world} independent server(s), one per GPU"},
        "latency_s": {"p50": serve.percentile(lat, 50), "p99": serve.percentile(lat, 99)},
        "requests_per_s": world * len(lat) / wall,
        "energy_drift_max": drift_max,
        "e2e": {"value": value, "unit": UNIT,
                "note": "each request's state goes host->device at admission and back at completion "
                        "inside the timed region"},
        "gpu_launches": launches, "clocks": clk.summary(), "turns": turns,
    }
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


SEED_SERVE = 2502_09537 + 4


def solve(s, stream, init, nsteps, per_chunk_events=None, step_launches=None):
    """One benchmark step: load the initial state, nsteps DP-AVF2 steps with the
    energy evaluated every ENERGY_EVERY steps.  Returns the invariants seen.
    With per_chunk_events, CUDA events bracket each kgs_step call on the stream
    and step_launches[0] accumulates the kernels those calls launched."""
    s.set_state(*init, stream=stream)
    seen = [s.invariants(stream=stream)]
    done = 0
    while done < nsteps:
        n = min(ENERGY_EVERY, nsteps - done)
        if per_chunk_events is not None:
            a, b = per_chunk_events.pop(0)
            l0 = s.launch_count
            a.record(stream)
            s.step(n, stream=stream)
            b.record(stream)
            step_launches[0] += s.launch_count - l0
        else:
            s.step(n, stream=stream)
        done += n
        seen.append(s.invariants(stream=stream))
    return seen


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="2d", choices=["2d", "1d", "3d", "batch", "serve"])
    ap.add_argument("--rate", type=float, default=50.0, help="serving: request arrival rate (1/s)")
    ap.add_argument("--requests", type=int, default=48, help="serving: requests per timed step")
    ap.add_argument("--turn-work", type=float, default=5e9,
                    help="serving: point-updates per turn, shortest remaining work first (0: all)")
    ap.add_argument("--max-steps", type=int, default=1000,
                    help="serving: upper end of the per-request step range (workload: 10000)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--threads", type=int, default=0, help="colour-pass CTA size (tuning)")
    ap.add_argument("--kernel", type=int, default=0,
                    help="KGS_OPT_KERNEL: 0 auto, 1 pass, 2 shared memory, 3 tile, 4 persistent, "
                         "5 slab-pipelined passes, 6 wave (a step's two passes in one launch)")
    ap.add_argument("--slab-planes", type=int, default=0, help="KGS_OPT_SLAB_PLANES (slab and wave kernels)")
    ap.add_argument("--wave-lag", type=int, default=0, help="KGS_OPT_WAVE_LAG (wave kernel)")
    ap.add_argument("--wave-chunk", type=int, default=0, help="KGS_OPT_WAVE_CHUNK (wave kernel)")
    ap.add_argument("--pdl", type=int, default=-1, help="KGS_OPT_PDL (-1: the library default)")
    ap.add_argument("--ppt", type=int, default=0, help="points per thread (tuning)")
    ap.add_argument("--order", default="checkerboard", choices=["checkerboard", "lex", "block", "lex-rev"],
                    help="update order: the checkerboard (Algorithm 3), the lexicographic "
                         "wavefront (Eq. order1), Algorithm 2's block order (2D, 16 blocks), or "
                         "lex-rev: Psi in the lexicographic order and (U,V) in its reverse "
                         "(per-variable orders, kgs_set_orders)")
    ap.add_argument("--order-mode", type=int, default=0,
                    help="KGS_OPT_ORDER_MODE for a general order: 0 auto, 1 one launch per level "
                         "(colour-split layout), 2 one persistent launch per step, 3 one launch per "
                         "level on a natural-order copy")
    ap.add_argument("--steps-per-solve", type=int, default=0,
                    help="DP-AVF2 steps per benchmark step (default: the workload's)")
    ap.add_argument("--grid-n", type=int, default=0,
                    help="points per direction instead of the workload's (small cases for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return

    import torch
    from paper_2502_09537_b300 import build as kbuild
    from paper_2502_09537_b300.solver import KGS_FP32, KGS_FP64, Solver, probe_fma_rate
    kbuild.build()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    work = make_workload(args.workload, args.grid_n)
    if args.steps_per_solve:
        work = work._replace(nsteps=args.steps_per_solve)
    prob = work.prob
    precision = KGS_FP64 if args.precision == "fp64" else KGS_FP32
    elem = 8 if precision == KGS_FP64 else 4
    stream = torch.cuda.Stream()
    init_dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in work.state]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    nchunks = (work.nsteps + ENERGY_EVERY - 1) // ENERGY_EVERY
    s = Solver.from_problem(prob, precision)
    from paper_2502_09537_b300.solver import KGS_OPT_PPT, KGS_OPT_THREADS
    if args.threads:
        s.set_option(KGS_OPT_THREADS, args.threads)
    if args.kernel:
        from paper_2502_09537_b300.solver import KGS_OPT_KERNEL
        s.set_option(KGS_OPT_KERNEL, args.kernel)
    if args.ppt:
        s.set_option(KGS_OPT_PPT, args.ppt)
    if args.slab_planes:
        from paper_2502_09537_b300.solver import KGS_OPT_SLAB_PLANES
        s.set_option(KGS_OPT_SLAB_PLANES, args.slab_planes)
    if args.wave_lag:
        from paper_2502_09537_b300.solver import KGS_OPT_WAVE_LAG
        s.set_option(KGS_OPT_WAVE_LAG, args.wave_lag)
    if args.wave_chunk:
        from paper_2502_09537_b300.solver import KGS_OPT_WAVE_CHUNK
        s.set_option(KGS_OPT_WAVE_CHUNK, args.wave_chunk)
    if args.pdl >= 0:
        from paper_2502_09537_b300.solver import KGS_OPT_PDL
        s.set_option(KGS_OPT_PDL, args.pdl)
    if args.order_mode:
        from paper_2502_09537_b300.solver import KGS_OPT_ORDER_MODE
        s.set_option(KGS_OPT_ORDER_MODE, args.order_mode)
    if args.order == "lex-rev":
        from paper_2502_09537_b300 import orders
        s.set_orders(orders.lexicographic(prob.dim, prob.N), orders.reverse_lexicographic(prob.dim, prob.N))
    elif args.order != "checkerboard":
        from paper_2502_09537_b300 import orders
        s.set_order(orders.lexicographic(prob.dim, prob.N) if args.order == "lex"
                    else orders.block_split_2d(prob.N, 16))
    torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            solve(s, stream, init_dev, work.nsteps)
        stream.synchronize()
        if dist:
            dist.barrier()
        iter_ms, kern_ms = [], []
        step_launches = [0]
        launches0 = s.launch_count
        drift = 0.0
        with ClockSampler(local) as clk:
            for _ in range(args.steps):
                flush.zero_()
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(nchunks)]
                kev = list(ev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                seen = solve(s, stream, init_dev, work.nsteps, per_chunk_events=kev,
                             step_launches=step_launches)
                e1.record(stream)
                stream.synchronize()
                iter_ms.append(e0.elapsed_time(e1))
                kern_ms.append(sum(a.elapsed_time(b) for a, b in ev))
                E0, S0, _ = seen[0]
                drift = max(drift, max(abs(E - E0) / max(S0, S) for E, S, _ in seen))
        launches = s.launch_count - launches0
    from paper_2502_09537_b300.dist import max_over_ranks
    total_ms = max_over_ranks(sum(iter_ms), device="cuda")
    pts_per_step = prob.points * work.nsteps
    value = world * pts_per_step * args.steps / (total_ms * 1e-3)

    # end to end through the C ABI with host buffers (pinned)
    host_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in work.state]
    host_out = [torch.empty(a.shape, dtype=torch.float64).pin_memory().numpy() for a in work.state]
    with torch.cuda.stream(stream):
        e2e_ms = []
        for _ in range(max(1, min(args.steps, 3))):
            flush.zero_()
            stream.synchronize()
            t0 = time.perf_counter()
            solve(s, stream, host_in, work.nsteps)
            s.get_state(host_out, stream=stream)
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_value = world * pts_per_step * len(e2e_ms) / (sum(e2e_ms) * 1e-3)

    # roofline of the dominant kernel (the colour-pass / tile kernel that runs
    # inside kgs_step): algorithmic work per launch / average launch duration,
    # both over the timed region
    pass_ms = sum(kern_ms) / step_launches[0]
    upd_per_launch = prob.points * work.nsteps * args.steps / step_launches[0]
    peaks = measured_peaks()
    if precision == KGS_FP64:
        fma_rate, _ = probe_fma_rate(64, 2048, 8, stream)
        fpu = (flops_per_point_update(prob.dim) if args.order == "checkerboard"
               else flops_per_point_update_unfused(prob.dim))
        flops_per_launch = upd_per_launch * fpu
        achieved = flops_per_launch / (pass_ms * 1e-3) / 1e12
        peak = FP64_PEAK_TFLOPS
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": traffic_of(args),
                "peak_source": "derived: 148 SMs x 2 FP64 FMA/cycle x 2 flops x 2032 MHz",
                "probe_tflops": 2 * fma_rate / 1e12,
                "work": "FP64-pipe flops (neighbour sums, beta S, B'S_U, 2r, 1/(1+r^2) and the red pass's V additions -- both in 1D/2D, one in 3D -- run on the integer pipes)",
                "flops_per_point_update": fpu,
                "algorithmic_flops_per_point_update": algorithmic_flops_per_point_update(prob.dim),
                "algorithmic_tflops": upd_per_launch * algorithmic_flops_per_point_update(prob.dim)
                / (pass_ms * 1e-3) / 1e12,
                "hbm_frac": bytes_per_point_update(elem) * upd_per_launch / (pass_ms * 1e-3)
                / 1e9 / peaks.get("hbm_gbs", 6400.0)}
    else:
        bytes_per_launch = upd_per_launch * bytes_per_point_update(elem)
        achieved = bytes_per_launch / (pass_ms * 1e-3) / 1e9
        peak = peaks.get("hbm_gbs", 6400.0)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": traffic_of(args),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "ms_per_step_median": float(np.median(iter_ms)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if elem == 8 else "f32",
        "data": "synthetic",
        "config": {"workload": work.name, "dim": prob.dim, "N": prob.N, "L": prob.L,
                   "threads": args.threads or 256, "kernel": args.kernel, "order": args.order,
                   "order_mode": args.order_mode,
                   "slab_planes": args.slab_planes, "wave_lag": args.wave_lag,
                   "wave_chunk": args.wave_chunk,
                   "tau": prob.tau, "steps_per_solve": work.nsteps, "precision": args.precision,
                   "energy_every": ENERGY_EVERY,
                   "l2": "256 MB buffer written between timed steps",
                   "parallelism": f"{world} independent instance(s), one per GPU"},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": 4 * prob.points * 8, "d2h_bytes_per_step": 4 * prob.points * 8},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "energy_drift": drift,
        "kernel_ms_per_launch": pass_ms,
        "kernel_launches_per_solve": step_launches[0] / args.steps,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:  # the oracle baseline: N = 1 only
        line["cpu_baseline"] = cpu_baseline(work)
    s.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
