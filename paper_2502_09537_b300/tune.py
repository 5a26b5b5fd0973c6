"""Autotuner for libkgs launch shapes.

For a problem bucket -- (dimension, N rounded up to a power of two,
precision) -- it times every candidate launch shape on a representative
problem of that bucket and keeps the fastest:

  * the colour-pass kernel (one launch per pass) with 128, 256 or 512 threads
    per CTA, its persistent grid-stride variant and its slab-pipelined
    schedule (2D, 3D);
  * the temporally blocked tile kernel with a few tile shapes (tile extents,
    passes per launch, threads per CTA) that fit in shared memory;
  * the shared-memory resident kernel, when the grid fits in one CTA.

For a batch it chooses the number of persistent CTAs per SM, for the whole
batch or per list of instances (one precision and dimension: the instances
whose colour passes share a launch), by coordinate descent over the lists
with the whole batch's step timed.  Every option
computes bitwise the same state (the kernels share their pointwise code), so
tuning changes only speed.  Timing uses CUDA events around kgs_step on the
caller's stream after warm-up steps; a timer can be injected (the CPU tests
do).  Results are cached in memory and, if a path is given, in a JSON file.
"""
from __future__ import annotations

import json
import math
import os
from typing import Callable, Dict, List, Optional, Sequence, Tuple

from .solver import (KGS_BATCH_OPT_CTAS_LIST, KGS_BATCH_OPT_CTAS_PER_SM, KGS_FP64, KGS_OPT_KERNEL, KGS_OPT_THREADS,
                     KGS_OPT_TILE_LX, KGS_OPT_TILE_PASSES, KGS_OPT_TILE_T1, KGS_OPT_TILE_T2,
                     KGS_OPT_TILE_THREADS, KGS_OPT_STREAM_CHUNK)

SMEM_BYTES = 227 * 1024
Options = Dict[int, int]


def bucket(prob, precision: int) -> Tuple[int, int, int]:
    """(dim, N rounded up to a power of two, precision)."""
    return (prob.dim, 1 << max(2, math.ceil(math.log2(prob.N))), precision)


def _tile_fits(dim: int, elem: int, T1: int, T2: int, H: int, threads: int) -> bool:
    A1 = 1 if dim == 2 else T1 + 2 * H
    A2 = T2 + 2 * H
    smem = (2 * H + 2) * A1 * A2 * 4 * elem
    return (smem <= SMEM_BYTES and A1 * A2 <= 6 * threads and A1 * (A2 // 2) <= 4 * threads
            and T2 % 2 == 0)


def candidates(prob, precision: int) -> List[Options]:
    """Launch shapes worth timing for this problem."""
    elem = 8 if precision == KGS_FP64 else 4
    out: List[Options] = [{KGS_OPT_KERNEL: 1, KGS_OPT_THREADS: t} for t in (128, 256, 512)]
    out.append({KGS_OPT_KERNEL: 4})  # persistent grid-stride passes
    if prob.dim >= 2:
        out.append({KGS_OPT_KERNEL: 5})  # colour passes pipelined in L2-sized axis-0 slabs
    if prob.dim == 3 and precision != KGS_FP64 and prob.N % 64 == 0 and 64 <= prob.N <= 1024:
        # streamed planes: a step's two passes in one launch, in chunk orders,
        # and a step pair's four passes in one launch
        out += [{KGS_OPT_KERNEL: 7, KGS_OPT_STREAM_CHUNK: ch} for ch in (0, 32, 128, -1)]
        out += [{KGS_OPT_KERNEL: 8, KGS_OPT_STREAM_CHUNK: ch} for ch in (0, -1)]
    if prob.points <= SMEM_BYTES // (4 * elem):
        out.append({KGS_OPT_KERNEL: 2})
    if prob.dim == 2:
        shapes = [(1, 256, 8, 512, 64), (1, 512, 8, 1024, 64), (1, 128, 8, 256, 64)]
    elif prob.dim == 3:
        shapes = [(32, 32, 3, 512, 64), (32, 32, 2, 512, 64), (16, 16, 2, 512, 64)]
    else:
        shapes = []
    for T1, T2, H, thr, LX in shapes:
        if _tile_fits(prob.dim, elem, T1, T2, H, thr) and prob.N >= 16:
            o = {KGS_OPT_KERNEL: 3, KGS_OPT_TILE_T2: T2, KGS_OPT_TILE_PASSES: H,
                 KGS_OPT_TILE_THREADS: thr, KGS_OPT_TILE_LX: LX}
            if prob.dim == 3:
                o[KGS_OPT_TILE_T1] = T1
            out.append(o)
    return out


def list_option(precision: int, dim: int) -> int:
    """The batch option that sets one list's persistent CTAs per SM."""
    return KGS_BATCH_OPT_CTAS_LIST + 3 * (0 if precision == KGS_FP64 else 1) + dim - 1


def list_name(precision: int, dim: int) -> str:
    return "%s_%dd" % ("fp64" if precision == KGS_FP64 else "fp32", dim)


def list_name_of_option(option: int) -> str:
    """The list name of a KGS_BATCH_OPT_CTAS_LIST option."""
    k = option - KGS_BATCH_OPT_CTAS_LIST
    return list_name(KGS_FP64 if k < 3 else 0, k % 3 + 1)


def default_cache_path() -> Optional[str]:
    """The JSON cache named by KGS_TUNE_CACHE, or None (in-memory only)."""
    return os.environ.get("KGS_TUNE_CACHE") or None


def apply(solver, options: Options) -> None:
    for k, v in options.items():
        solver.set_option(k, v)


def cuda_event_timer(solver, nsteps: int, stream=None) -> float:
    """Milliseconds of solver.step(nsteps) on the stream, by CUDA events."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    solver.step(nsteps, stream=s)
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1)


class Tuner:
    def __init__(self, cache_path: Optional[str] = None,
                 timer: Callable = cuda_event_timer,
                 make_solver: Optional[Callable] = None):
        self.cache_path = cache_path
        self.timer = timer
        self.make_solver = make_solver
        self.cache: Dict[str, Options] = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                raw = json.load(f)
            self.cache = {k: {int(a): int(b) for a, b in v.items()} for k, v in raw.items()}

    def _save(self):
        if self.cache_path:
            tmp = self.cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump({k: {str(a): b for a, b in v.items()} for k, v in self.cache.items()},
                          f, indent=1, sort_keys=True)
            os.replace(tmp, self.cache_path)

    def _solver(self, prob, precision):
        if self.make_solver is not None:
            return self.make_solver(prob, precision)
        import numpy as np
        from .solver import Solver
        s = Solver.from_problem(prob, precision)
        st = [np.full((prob.N,) * prob.dim, 0.1) for _ in range(4)]
        s.set_state(*st)
        return s

    def tune(self, prob, precision: int = KGS_FP64, nsteps: Optional[int] = None,
             warmup: int = 2) -> Options:
        """Fastest launch options for the bucket of prob (measured once per bucket)."""
        key = "%d:%d:%d" % bucket(prob, precision)
        if key in self.cache:
            return dict(self.cache[key])
        if nsteps is None:  # about 5e8 point-updates per candidate, at least 4 steps
            nsteps = max(4, int(5e8 // prob.points))
        best, best_ms = None, float("inf")
        for opts in candidates(prob, precision):
            s = self._solver(prob, precision)
            try:
                apply(s, opts)
                s.step(warmup)
                ms = self.timer(s, nsteps)
            except Exception:
                continue  # a shape this problem cannot take
            finally:
                close = getattr(s, "close", None)
                if close:
                    close()
            if ms < best_ms:
                best, best_ms = opts, ms
        if best is None:
            best = {}
        self.cache[key] = dict(best)
        self._save()
        return dict(best)

    def tune_batch(self, batch, nsteps: int,
                   ctas: Sequence[int] = (2, 4, 8, 16), timer: Optional[Callable] = None) -> int:
        """Persistent CTAs per SM for a batch (times batch.step(nsteps) for each)."""
        t = timer or self.timer
        best, best_ms = ctas[0], float("inf")
        for c in ctas:
            batch.set_option(KGS_BATCH_OPT_CTAS_PER_SM, c)
            ms = t(batch, nsteps)
            if ms < best_ms:
                best, best_ms = c, ms
        batch.set_option(KGS_BATCH_OPT_CTAS_PER_SM, best)
        return best

    def tune_batch_lists(self, batch, members: Sequence[Tuple[object, int]], nsteps: int = 8,
                         values: Sequence[int] = (2, 4, 8, 16), warmup: int = 1,
                         timer: Optional[Callable] = None, stream=None) -> Dict[str, int]:
        """Persistent CTAs per SM of every list of a batch (members: the
        (problem, precision) of its live instances).  Lists are tuned one at a
        time, the others held at their current choice, each value timed over
        batch.step(nsteps) after `warmup` untimed calls (a changed option makes
        the next call capture a new graph).  The choice is set on the batch,
        cached per (list, total points rounded up to a power of two) and
        returned as {list name: CTAs per SM}."""
        t = timer or (lambda b, n: self.timer(b, n, stream) if self.timer is cuda_event_timer
                      else self.timer(b, n))
        points: Dict[Tuple[int, int], int] = {}
        for prob, prec in members:
            k = (prec, prob.dim)
            points[k] = points.get(k, 0) + prob.points
        chosen: Dict[str, int] = {}
        todo = []
        for (prec, dim), pts in sorted(points.items()):
            key = "batch:%s:%d" % (list_name(prec, dim), 1 << max(0, math.ceil(math.log2(pts))))
            if key in self.cache:
                v = int(self.cache[key][0])
                batch.set_option(list_option(prec, dim), v)
                chosen[list_name(prec, dim)] = v
            else:
                todo.append((prec, dim, key))
        for prec, dim, key in todo:
            best, best_ms = values[0], float("inf")
            for v in values:
                batch.set_option(list_option(prec, dim), v)
                for _ in range(warmup):
                    batch.step(nsteps, stream=stream)
                ms = t(batch, nsteps)
                if ms < best_ms:
                    best, best_ms = v, ms
            batch.set_option(list_option(prec, dim), best)
            chosen[list_name(prec, dim)] = best
            self.cache[key] = {0: best}
        if todo:
            self._save()
        return chosen
