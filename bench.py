#!/usr/bin/env python
"""Benchmark of the DP-AVF2 checkerboard solver (arXiv 2502.09537) on one B300.

Workload (default): the 3D KGS problem on [-10,10)^3 with N = 512^3 points
(134M points, 4.3 GB of float64 state), kappa1 = kappa2 = mu = gamma = 1,
tau = 5e-4, 200 DP-AVF2 steps, psi0 = (1+i) exp(-|x|^2), u0 = exp(-|x|^2),
v0 = 0 plus seeded Gaussian noise (sigma 1e-4); the discrete energy is
evaluated every 100 steps.  One benchmark step = one such solve: load the
initial state (already in HBM), 200 steps, 3 energy/mass evaluations.
Metric: grid-point updates per second (N^d x steps / time).  `value` is the
float64 solve; the line also carries the same workload with float32 state
(its rate, roofline, speed-up, and its max-norm error and energy drift
against the float64 run), the 96-instance batch in both precisions and a
serving run at 50 requests/s (one timed step each).  Multi-GPU: every rank
solves its own instance (the instances are independent), value = all ranks'
point-updates / max time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload 3d|2d|1d|batch|serve] [--precision fp64|fp32]

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


# DRAM bytes per launch of the dominant kernel: the sum dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture of that launch on the workload's
# full grid (2D: a RED_FUSED pass of the 2048^2 grid; 3D: a launch of the
# 512^3 grid, one-pass metrics), for the kernels as they are now, keyed by
# (workload, precision, kernel: "pass" = one launch per colour pass, "stream"
# = a step's two passes per launch, "stream2" = a step pair's four passes per
# launch); None where no capture exists.
NCU_TRAFFIC = {("2d", "fp64", "pass"): 117.52e6 + 25.74e6,
               ("3d", "fp64", "pass"): 3.7645e9 + 2.1086e9,
               ("3d", "fp32", "pass"): 1.8822e9 + 1.0321e9,
               ("3d", "fp32", "stream"): 2.4073e9 + 2.1756e9,
               ("3d", "fp32", "stream2"): 2.5981e9 + 2.1786e9}


# Issue-slot view of the float64 colour passes: the fraction of peak each
# pipe issued at (sm__inst_executed_pipe_{fp64,alu,fma}, smsp__issue_active;
# ncu --set full, active cycles, mean of the black and red passes), from the
# captures of the current kernels: 2D on the 2048^2 launches, 3D on 256^3
# launches.  The FP64 pipe binds; the integer ALU pipe, which carries the
# exact neighbour sums and the Psi weight, is close behind.
NCU_PIPES = {("2d", "fp64", "pass"): {"fp64": 0.874, "alu": 0.746, "fma": 0.129, "issue_active": 0.611},
             ("3d", "fp64", "pass"): {"fp64": 0.864, "alu": 0.825, "fma": 0.131, "issue_active": 0.652}}


def kernel_name(args, precision=None):
    """The dominant kernel of a solve: what KGS_OPT_KERNEL selects (0 = the
    library's automatic choice, which streams float32 3D grids whose N is a
    multiple of 64 from 128 to 1024, two steps per launch ("stream2"), and
    makes one launch per pass otherwise; "stream": one step per launch)."""
    precision = precision or args.precision
    n = args.grid_n or {"1d": 512, "2d": 2048, "3d": 512}.get(args.workload, 0)
    streams = args.workload == "3d" and precision == "fp32" and n % 64 == 0 and 64 <= n <= 1024
    if args.kernel == 8 or (args.kernel == 0 and streams and n >= 128):
        return "stream2" if streams else "pass"
    if args.kernel == 7:
        return "stream" if streams else "pass"
    return "pass" if args.kernel in (0, 1) else None


def traffic_of(args, precision=None):
    """DRAM bytes per launch of the dominant kernel from the ncu captures
    above: only for the launches they were taken on (the workload's full grid,
    checkerboard order, the kernel captured); None otherwise."""
    if args.order != "checkerboard" or args.grid_n:
        return None
    k = kernel_name(args, precision)
    if k is None:
        return None
    return NCU_TRAFFIC.get((args.workload, precision or args.precision, k))


# Issue-active fraction of the two-step streamed kernel (smsp__issue_active,
# ncu --set full of one 256^3 launch of the current kernel).
NCU_ISSUE_STREAM2 = 0.656


# FP64 pipe of the B300: 2 FMA per cycle per SM (ncu: peak_sustained of
# sm__sass_thread_inst_executed_op_dfma_pred_on), 148 SMs, 2032 MHz maximum SM
# clock -> 2 x 2 x 148 x 2.032e9 = 1.203e12 flop/s.
FP64_PEAK_TFLOPS = 2 * 2 * 148 * 2.032e9 / 1e12


def bytes_per_point_update(elem: int, depth: int = 1) -> float:
    """Algorithmic HBM bytes of one point-update: read and write the four
    fields once per launch (the two colour passes of a step each touch their
    own half), over the `depth` steps a launch applies."""
    return 2 * 4 * elem / depth


def temporal_depth(args, precision=None) -> int:
    """Steps per launch of the dominant kernel."""
    return 2 if kernel_name(args, precision) == "stream2" else 1


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


def init_dist():
    """(world, rank, local, dist module or None) from the torchrun environment;
    sets the device and joins an NCCL group when there are several ranks."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local, dist


def batch_leg(precision_name, steps, warmup, world, local, dist, tuned=True, persistent=False):
    """The 96-instance batch: 64 2D grids N in {128..2048} and 32 3D grids N in
    {64..256}, random parameters, tau = 5e-4, 500 steps, every instance in the
    chosen precision, stepped by kgs_batch_step (one launch per colour pass,
    dimension and mode over all instances, replayed from a CUDA graph), with the
    autotuner's persistent-CTA choice.  One benchmark step = load every initial
    state from HBM, 500 steps.  Returns the measurement as a dict."""
    import torch
    from paper_2502_09537_b300 import inputs, tune
    from paper_2502_09537_b300.solver import KGS_FP32, KGS_FP64, Batch
    precision = KGS_FP64 if precision_name == "fp64" else KGS_FP32
    elem = 8 if precision == KGS_FP64 else 4
    specs = inputs.batched_instances()
    nsteps = specs[0][1]
    total_bytes = sum(p.points * 4 * elem for p, _, _ in specs)
    b = Batch(int(total_bytes * 1.05) + (64 << 20))
    if persistent:
        from paper_2502_09537_b300.solver import KGS_BATCH_OPT_PERSISTENT
        b.set_option(KGS_BATCH_OPT_PERSISTENT, 1)
    init, ids = [], []
    for p, _, fn in specs:
        ids.append(b.add(p, precision))
        init.append([torch.from_numpy(a).cuda() for a in fn()])
    torch.cuda.synchronize()
    points = sum(p.points for p, _, _ in specs)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def load():
        for i, st in zip(ids, init):
            b.set_state(i, *st, stream=stream)

    load()  # the tuner steps the batch: every instance needs a state
    tuned_opts = tune.Tuner(tune.default_cache_path()).tune_batch_lists(
        b, [(p, precision) for p, _, _ in specs], stream=stream) if tuned and not persistent else {}

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            load()
            b.step(nsteps, stream=stream)
        stream.synchronize()
        if dist:
            dist.barrier()
        times, kern = [], []
        l0 = b.launch_count
        with ClockSampler(local) as clk:
            for _ in range(steps):
                flush.zero_()
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(stream)
                load()
                e1.record(stream)
                b.step(nsteps, stream=stream)
                e2.record(stream)
                stream.synchronize()
                times.append(e0.elapsed_time(e2))
                kern.append(e1.elapsed_time(e2))
        launches = b.launch_count - l0
    from paper_2502_09537_b300.dist import max_over_ranks
    total_ms = max_over_ranks(sum(times), device="cuda")
    value = world * points * nsteps * steps / (total_ms * 1e-3)
    # the colour passes of one precision: a launch per pass, dimension and mode
    pass_ms = sum(kern) / max(launches, 1)
    upd_per_launch = points * nsteps * steps / max(launches, 1)
    peaks = measured_peaks()
    if precision == KGS_FP64:
        mean_dim_flops = sum(p.points * flops_per_point_update(p.dim) for p, _, _ in specs) / points
        achieved = upd_per_launch * mean_dim_flops / (pass_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "derived: 148 SMs x 2 FP64 FMA/cycle x 2 flops x 2032 MHz",
                "work": "FP64-pipe flops of the colour passes"}
    else:
        achieved = upd_per_launch * bytes_per_point_update(elem) / (pass_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks.get("hbm_gbs", 6400.0),
                "unit": "GB/s", "frac": achieved / peaks.get("hbm_gbs", 6400.0), "traffic": None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs of measured"}
    # end to end: host states in and out (pinned), one solve
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
    b.close()
    return {
        "value": value, "ms_per_step": total_ms / steps, "steps": steps, "warmup": warmup,
        "dtype": "f64" if elem == 8 else "f32",
        "config": {"workload": "kgs_batch96", "instances": len(specs), "points": points,
                   "steps_per_solve": nsteps, "precision": precision_name,
                   "tuned": tuned_opts, "persistent_launch": bool(persistent),
                   "l2": "256 MB buffer written between timed steps"},
        "roofline": roof,
        "e2e": {"value": world * points * nsteps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": points * 32, "d2h_bytes_per_step": points * 32},
        "gpu_launches": launches, "clocks": clk.summary(), "kernel_ms_per_launch": pass_ms,
    }


def run_batch(args):
    world, rank, local, dist = init_dist()
    from paper_2502_09537_b300 import build as kbuild
    kbuild.build()
    leg = batch_leg(args.precision, args.steps, args.warmup, world, local, dist, tuned=not args.untuned,
                    persistent=args.batch_persistent)
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": world, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "data": "synthetic"}
    line.update(leg)
    line["config"]["parallelism"] = f"{world} independent batch(es), one per GPU"
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def serve_leg(rate, requests, steps, warmup, max_steps, turn_work, world, rank, local, tuned=True):
    """Continuous-batching serving: Poisson arrivals of solve requests (dim in
    {1,2,3}, N in [256,8192] / [128,2048]^2 / [64,384]^3, steps uniform in
    [100, max_steps], FP32 or FP64 each, parameters as the batched workload),
    admitted by a 150 GB device-memory budget, states resident on the device.
    One benchmark step = serving `requests` requests from their arrival to
    their result on the host; value = point-updates/s over the step, with
    p50/p99 request latency and the worst per-request energy drift."""
    import torch
    from paper_2502_09537_b300 import serve
    budget = 150 * (1 << 30)
    stream = torch.cuda.Stream()
    batch_options, chosen = {}, {}
    if tuned:
        # the autotuner's per-list launch shapes, timed on a mix drawn from the
        # request distribution (capped at 8 GB of state)
        from paper_2502_09537_b300 import tune
        mix, used = [], 0
        for r in serve.poisson_requests(rate, 32, seed=SEED_SERVE - 1, step_range=(100, max_steps)):
            nb = serve.state_bytes(r.prob, r.precision)
            if used + nb <= (8 << 30):
                mix.append((r.prob, r.precision))
                used += nb
        batch_options = serve.tuned_batch_options(tune.Tuner(tune.default_cache_path()), mix, stream=stream)
        chosen = {tune.list_name_of_option(k): v for k, v in batch_options.items()}
    lat, pts, wall, drift_max, turns = [], 0, 0.0, 0.0, 0
    service = []
    launches = 0
    with torch.cuda.stream(stream):
        with ClockSampler(local) as clk:
            for k in range(warmup + steps):
                reqs = serve.poisson_requests(rate, requests, seed=SEED_SERVE + 1000 * rank + k,
                                              step_range=(100, max_steps))
                srv = serve.Server(budget, quantum=100, stream=stream, keep_state=True,
                                   turn_work=turn_work, batch_options=batch_options)
                for r in reqs:
                    srv.submit(r)
                l0 = srv.batch.launch_count
                t0 = time.perf_counter()
                res = srv.run()
                dt = time.perf_counter() - t0
                if k >= warmup:
                    wall += dt
                    pts += srv.point_updates
                    lat += [r.latency for r in res]
                    service += [r.finished - r.admitted for r in res]
                    drift_max = max(drift_max, max(r.energy_drift for r in res))
                    turns += srv.turns
                    launches += srv.batch.launch_count - l0
                srv.close()
    from paper_2502_09537_b300.dist import max_over_ranks
    wall = max_over_ranks(wall, device="cuda")
    value = world * pts / wall
    return {
        "value": value, "ms_per_step": 1e3 * wall / steps, "steps": steps, "warmup": warmup,
        "dtype": "f64+f32",
        "config": {"workload": "kgs_serve", "rate_per_s": rate,
                   "requests_per_step": requests, "step_range": [100, max_steps],
                   "budget_bytes": budget, "quantum_steps": 100, "turn_work": turn_work,
                   "tuned_batch_options": chosen,
                   "l2": "inputs are built per request on the host (cold)"},
        "latency_s": {"p50": serve.percentile(lat, 50), "p99": serve.percentile(lat, 99)},
        "residence_s": {"p50": serve.percentile(service, 50), "p99": serve.percentile(service, 99)},
        "requests_per_s": world * len(lat) / wall,
        "energy_drift_max": drift_max,
        "e2e": {"value": value, "unit": UNIT,
                "note": "each request's state goes host->device at admission and back at completion "
                        "inside the timed region"},
        "gpu_launches": launches, "clocks": clk.summary(), "turns": turns,
    }


def run_serve(args):
    world, rank, local, dist = init_dist()
    from paper_2502_09537_b300 import build as kbuild
    kbuild.build()
    rates = [float(r) for r in str(args.rate).split(",")]
    for rate in rates:
        leg = serve_leg(rate, args.requests, args.steps, args.warmup, args.max_steps, args.turn_work,
                        world, rank, local)
        line = {"metric": METRIC, "unit": UNIT, "n_gpus": world, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "data": "synthetic"}
        line.update(leg)
        line["config"]["parallelism"] = f"{world} independent server(s), one per GPU"
        if rank == 0:
            print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


SEED_SERVE = 2502_09537 + 4


def solve(s, stream, init, nsteps, per_chunk_events=None, step_launches=None):
    """One benchmark step: load the initial state, nsteps DP-AVF2 steps with the
    energy evaluated every ENERGY_EVERY steps.  Returns the invariants seen.
    With per_chunk_events, CUDA events bracket each kgs_step call on the stream
    and step_launches[0] accumulates the kernels those calls launched."""
    s.set_state(*init, stream=stream)
    return advance(s, stream, nsteps, per_chunk_events, step_launches)


def advance(s, stream, nsteps, per_chunk_events=None, step_launches=None):
    """The steps of one solve from the state the solver holds, with the energy
    evaluated every ENERGY_EVERY steps (each evaluation waits for the stream)."""
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


def configure(s, args, prob):
    """Apply the command line's kernel options and update order to a solver."""
    from paper_2502_09537_b300 import solver as ks
    for flag, opt in ((args.threads, ks.KGS_OPT_THREADS), (args.kernel, ks.KGS_OPT_KERNEL),
                      (args.ppt, ks.KGS_OPT_PPT), (args.slab_planes, ks.KGS_OPT_SLAB_PLANES),
                      (args.wave_lag, ks.KGS_OPT_WAVE_LAG), (args.wave_chunk, ks.KGS_OPT_WAVE_CHUNK),
                      (args.order_mode, ks.KGS_OPT_ORDER_MODE),
                      (args.stream_chunk, ks.KGS_OPT_STREAM_CHUNK)):
        if flag:
            s.set_option(opt, flag)
    if args.stream_prefetch >= 0:
        s.set_option(ks.KGS_OPT_STREAM_PREFETCH, args.stream_prefetch)
    if args.pdl >= 0:
        s.set_option(ks.KGS_OPT_PDL, args.pdl)
    if args.order == "lex-rev":
        from paper_2502_09537_b300 import orders
        s.set_orders(orders.lexicographic(prob.dim, prob.N), orders.reverse_lexicographic(prob.dim, prob.N))
    elif args.order != "checkerboard":
        from paper_2502_09537_b300 import orders
        s.set_order(orders.lexicographic(prob.dim, prob.N) if args.order == "lex"
                    else orders.block_split_2d(prob.N, 16))


def solo_leg(args, work, precision_name, init_dev, flush, local, dist, world, steps, warmup):
    """Time `steps` solves of the workload (after `warmup` untimed ones) in one
    precision, CUDA events on the solver's stream; returns the measurement and
    the solver (open, holding the last solve's final state)."""
    import torch
    from paper_2502_09537_b300.solver import KGS_FP32, KGS_FP64, Solver, probe_fma_rate
    prob = work.prob
    precision = KGS_FP64 if precision_name == "fp64" else KGS_FP32
    elem = 8 if precision == KGS_FP64 else 4
    stream = torch.cuda.Stream()
    nchunks = (work.nsteps + ENERGY_EVERY - 1) // ENERGY_EVERY
    s = Solver.from_problem(prob, precision)
    configure(s, args, prob)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            solve(s, stream, init_dev, work.nsteps)
        stream.synchronize()
        if dist:
            dist.barrier()
        iter_ms, kern_ms = [], []
        step_launches = [0]
        launches0 = s.launch_count
        drift = 0.0
        with ClockSampler(local) as clk:
            for _ in range(steps):
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
    value = world * pts_per_step * steps / (total_ms * 1e-3)
    # roofline of the dominant kernel (the colour-pass kernels that run inside
    # kgs_step): algorithmic work per launch / average launch duration, both
    # over the timed region
    pass_ms = sum(kern_ms) / step_launches[0]
    upd_per_launch = pts_per_step * steps / step_launches[0]
    peaks = measured_peaks()
    if precision == KGS_FP64:
        fma_rate, _ = probe_fma_rate(64, 2048, 8, stream)
        fpu = (flops_per_point_update(prob.dim) if args.order == "checkerboard"
               else flops_per_point_update_unfused(prob.dim))
        achieved = upd_per_launch * fpu / (pass_ms * 1e-3) / 1e12
        peak = FP64_PEAK_TFLOPS
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": traffic_of(args, precision_name),
                "peak_source": "derived: 148 SMs x 2 FP64 FMA/cycle x 2 flops x 2032 MHz",
                "probe_tflops": 2 * fma_rate / 1e12,
                "work": "FP64-pipe flops (neighbour sums, beta S, B'S_U, 2r, 1/(1+r^2) and the red pass's V additions -- both in 1D/2D, one in 3D -- run on the integer pipes)",
                "flops_per_point_update": fpu,
                "algorithmic_flops_per_point_update": algorithmic_flops_per_point_update(prob.dim),
                "algorithmic_tflops": upd_per_launch * algorithmic_flops_per_point_update(prob.dim)
                / (pass_ms * 1e-3) / 1e12,
                "hbm_frac": bytes_per_point_update(elem) * upd_per_launch / (pass_ms * 1e-3)
                / 1e9 / peaks.get("hbm_gbs", 6400.0)}
        k = kernel_name(args, precision_name)
        if traffic_of(args, precision_name) is not None and (args.workload, precision_name, k) in NCU_PIPES:
            roof["pipes_ncu"] = dict(NCU_PIPES[(args.workload, precision_name, k)],
                                     note="fraction of each pipe's peak issue rate over active cycles, "
                                          "ncu capture of these launches")
    else:
        depth = temporal_depth(args, precision_name)
        achieved = upd_per_launch * bytes_per_point_update(elem, depth) / (pass_ms * 1e-3) / 1e9
        peak = peaks.get("hbm_gbs", 6400.0)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": traffic_of(args, precision_name),
                "peak_source": ("MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks
                                else "fallback 6.4 TB/s (of fallback)"),
                "bytes_per_point_update": bytes_per_point_update(elem, depth), "temporal_depth": depth}
    leg = {
        "value": value, "ms_per_step": total_ms / steps,
        "ms_per_step_median": float(np.median(iter_ms)), "steps": steps, "warmup": warmup,
        "dtype": "f64" if elem == 8 else "f32", "roofline": roof, "gpu_launches": launches,
        "clocks": clk.summary(), "energy_drift": drift, "kernel_ms_per_launch": pass_ms,
        "kernel_launches_per_solve": step_launches[0] / steps,
    }
    return leg, s, stream


def e2e_leg(s, stream, work, flush, world, steps, make_solver):
    """The same solves end to end through the C ABI with host buffers: every
    solve's initial state goes in from pinned host memory and its final state
    comes back to pinned host memory, inside the timed region.  Two handles
    take turns, as a caller streaming many problems would run them: while one
    computes, the next solve's input goes into the other on an upload stream
    and the previous solve's result comes back on a download stream
    (KGS_HOST_ASYNC transfers, ordered by events)."""
    import torch
    prob = work.prob
    n = max(1, steps)
    host_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in work.state]
    host_out = [[torch.empty(a.shape, dtype=torch.float64).pin_memory().numpy() for a in work.state]
                for _ in range(2)]
    other = make_solver()
    with torch.cuda.stream(stream):
        solve(other, stream, host_in, work.nsteps)  # untimed: first-use allocations and graphs
    hs = [s, other]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    flush.zero_()
    torch.cuda.synchronize()
    loaded, read = {}, {}

    def upload(i):
        if i - 2 in read:
            up.wait_event(read[i - 2])  # this handle's previous result is out
        hs[i % 2].set_state(*host_in, stream=up, asynchronous=True)
        loaded[i] = torch.cuda.Event()
        loaded[i].record(up)

    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        upload(0)
        for i in range(n):
            if i + 1 < n:
                upload(i + 1)
            stream.wait_event(loaded[i])
            advance(hs[i % 2], stream, work.nsteps)
            done = torch.cuda.Event()
            done.record(stream)
            down.wait_event(done)
            hs[i % 2].get_state(host_out[i % 2], stream=down, asynchronous=True)
            read[i] = torch.cuda.Event()
            read[i].record(down)
        down.synchronize()
    from paper_2502_09537_b300.dist import max_over_ranks
    e2e_s = max_over_ranks(time.perf_counter() - t0, device="cuda")  # the slowest rank's time
    other.close()
    del host_in, host_out
    return {"value": world * prob.points * work.nsteps * n / e2e_s, "unit": UNIT,
            "h2d_bytes_per_step": 4 * prob.points * 8, "d2h_bytes_per_step": 4 * prob.points * 8,
            "solves": n, "overlap": "two handles; copies of one solve overlap the other's compute"}


def final_state_dev(s, prob):
    import torch
    out = tuple(torch.empty((prob.N,) * prob.dim, dtype=torch.float64, device="cuda") for _ in range(4))
    s.get_state(out)
    torch.cuda.synchronize()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="3d", choices=["3d", "2d", "1d", "batch", "serve"],
                    help="3d (default): the 512^3 configuration in FP64 with an FP32 leg; 2d: "
                         "2048^2; 1d: the 512-point soliton; batch: the 96 instances; serve: "
                         "continuous batching")
    ap.add_argument("--rate", default="50", help="serving: request arrival rate(s) (1/s), comma-separated")
    ap.add_argument("--requests", type=int, default=48, help="serving: requests per timed step")
    ap.add_argument("--turn-work", type=float, default=5e9,
                    help="serving: point-updates per turn, shortest remaining work first (0: all)")
    ap.add_argument("--max-steps", type=int, default=10000,
                    help="serving: upper end of the per-request step range (the workload's 10000)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true", help="3d: skip the FP32 leg")
    ap.add_argument("--no-summaries", action="store_true",
                    help="3d: skip the compact batch and serve summaries")
    ap.add_argument("--untuned", action="store_true", help="batch: library defaults, no autotuner")
    ap.add_argument("--batch-persistent", action="store_true",
                    help="batch: one persistent cooperative launch per step call (KGS_BATCH_OPT_PERSISTENT)")
    ap.add_argument("--threads", type=int, default=0, help="colour-pass CTA size (tuning)")
    ap.add_argument("--kernel", type=int, default=0,
                    help="KGS_OPT_KERNEL: 0 auto, 1 pass, 2 shared memory, 3 tile, 4 persistent, "
                         "5 slab-pipelined passes, 6 wave (a step's two passes in one launch), "
                         "7 streamed planes (3D FP32: a step's two passes per axis-0 plane, TMA-staged), "
                         "8 streamed planes, two steps per launch (the 3D FP32 default)")
    ap.add_argument("--slab-planes", type=int, default=0, help="KGS_OPT_SLAB_PLANES (slab and wave kernels)")
    ap.add_argument("--stream-chunk", type=int, default=0, help="KGS_OPT_STREAM_CHUNK (streamed-plane kernel)")
    ap.add_argument("--stream-prefetch", type=int, default=-1,
                    help="KGS_OPT_STREAM_PREFETCH (streamed-plane kernel; -1: the library default)")
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
    kbuild.build()
    world, rank, local, dist = init_dist()

    work = make_workload(args.workload, args.grid_n)
    if args.steps_per_solve:
        work = work._replace(nsteps=args.steps_per_solve)
    prob = work.prob
    init_dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in work.state]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    leg, s, stream = solo_leg(args, work, args.precision, init_dev, flush, local, dist, world,
                              args.steps, args.warmup)

    def make_solver(precision_name):
        from paper_2502_09537_b300.solver import KGS_FP32, KGS_FP64, Solver
        h = Solver.from_problem(prob, KGS_FP64 if precision_name == "fp64" else KGS_FP32)
        configure(h, args, prob)
        return h

    e2e = e2e_leg(s, stream, work, flush, world, args.steps, lambda: make_solver(args.precision))
    line = {
        "metric": METRIC, "value": leg["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": leg["ms_per_step"],
        "ms_per_step_median": leg["ms_per_step_median"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": leg["dtype"],
        "data": "synthetic",
        "config": {"workload": work.name, "dim": prob.dim, "N": prob.N, "L": prob.L,
                   "threads": args.threads or 256, "kernel": args.kernel, "order": args.order,
                   "order_mode": args.order_mode,
                   "slab_planes": args.slab_planes, "wave_lag": args.wave_lag,
                   "wave_chunk": args.wave_chunk, "stream_chunk": args.stream_chunk,
                   "tau": prob.tau, "steps_per_solve": work.nsteps, "precision": args.precision,
                   "energy_every": ENERGY_EVERY,
                   "l2": "256 MB buffer written between timed steps",
                   "parallelism": f"{world} independent instance(s), one per GPU"},
        "roofline": leg["roofline"],
        "e2e": e2e,
        "gpu_launches": leg["gpu_launches"],
        "clocks": leg["clocks"],
        "energy_drift": leg["energy_drift"],
        "kernel_ms_per_launch": leg["kernel_ms_per_launch"],
        "kernel_launches_per_solve": leg["kernel_launches_per_solve"],
    }

    # FP32 state against FP64 on the same workload: its own timing and
    # roofline, the speed-up, and its max-norm error and energy drift against
    # the FP64 run (the FP64 path equals the FP64 oracle to 1e-12, tested)
    if args.precision == "fp64" and not args.no_fp32 and args.workload in ("3d", "2d"):
        ref = final_state_dev(s, prob)
        s.close()
        leg32, s32, stream32 = solo_leg(args, work, "fp32", init_dev, flush, local, dist, world,
                                        args.steps, min(args.warmup, 3))
        got = final_state_dev(s32, prob)
        e2e32 = e2e_leg(s32, stream32, work, flush, world, args.steps, lambda: make_solver("fp32"))
        s32.close()
        one_step = None
        if kernel_name(args, "fp32") == "stream2":
            # the one-step streamed kernel beside it: DRAM-bound where the
            # two-step one is bound by instruction issue
            args1 = argparse.Namespace(**vars(args))
            args1.kernel = 7
            leg1, s1, _ = solo_leg(args1, work, "fp32", init_dev, flush, local, dist, world,
                                   min(args.steps, 3), 1)
            s1.close()
            one_step = {"value": leg1["value"], "unit": UNIT, "kernel": 7, "roofline": leg1["roofline"],
                        "kernel_ms_per_launch": leg1["kernel_ms_per_launch"], "gpu_launches": leg1["gpu_launches"],
                        "clocks": leg1["clocks"]}
        errs = [float((a - b).abs().max() / b.abs().max()) for a, b in zip(got, ref)]
        del got, ref
        line["fp32"] = {
            "value": leg32["value"], "unit": UNIT, "ms_per_step": leg32["ms_per_step"],
            "speedup_vs_fp64": leg32["value"] / leg["value"],
            "max_norm_rel_err_vs_fp64": max(errs),
            "max_norm_rel_err_per_field": dict(zip(("P", "Q", "U", "V"), errs)),
            "energy_drift": leg32["energy_drift"], "roofline": leg32["roofline"], "e2e": e2e32,
            "gpu_launches": leg32["gpu_launches"], "clocks": leg32["clocks"],
            "kernel_ms_per_launch": leg32["kernel_ms_per_launch"],
            "kernel_launches_per_solve": leg32["kernel_launches_per_solve"],
            "note": "error of the FP32-state run against the FP64 run from the same initial state, "
                    "per field max|x32 - x64| / max|x64| after the whole solve",
        }
        if one_step is not None:
            roof = line["fp32"]["roofline"]
            roof["note"] = (
                "two steps per launch (temporal depth 2): one read and one write of the state per two "
                "steps, 16 B per point-update; bound by shared-memory latency and instruction issue, "
                f"not DRAM (ncu 256^3: {NCU_ISSUE_STREAM2:.0%} issue-active); one_step: the DRAM-bound "
                "one-step kernel; equivalent_*: the bandwidth a one-step kernel (32 B per point-update) "
                "would need for this kernel's rate")
            roof["equivalent_one_step_gbs"] = roof["achieved"] * 2
            roof["equivalent_one_step_frac"] = roof["frac"] * 2
            line["fp32"]["one_step"] = one_step
            line["gpu_launches"] += one_step["gpu_launches"]
        line["gpu_launches"] += leg32["gpu_launches"]
    else:
        s.close()

    if rank == 0 and world == 1 and not args.no_cpu_baseline:  # the oracle baseline: N = 1 only
        line["cpu_baseline"] = cpu_baseline(work)
    del init_dev
    torch.cuda.empty_cache()

    # compact summaries of the batched and served workloads (one timed step each)
    if args.workload == "3d" and not args.no_summaries and not args.grid_n:
        summ = {}
        for name in ("fp64", "fp32"):
            b = batch_leg(name, 1, 1, world, local, dist)
            summ[name] = {k: b[k] for k in ("value", "ms_per_step", "roofline", "gpu_launches",
                                            "kernel_ms_per_launch")}
            summ[name]["tuned"] = b["config"]["tuned"]
        summ["config"] = {"workload": "kgs_batch96", "instances": 96, "steps_per_solve": 500,
                          "timed_steps": 1, "warmup": 1}
        line["batch"] = summ
        sv = serve_leg(50.0, 16, 1, 0, 10000, args.turn_work, world, rank, local)
        line["serve"] = {k: sv[k] for k in ("value", "latency_s", "residence_s", "requests_per_s",
                                            "energy_drift_max", "gpu_launches", "turns")}
        line["serve"]["config"] = sv["config"]
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
