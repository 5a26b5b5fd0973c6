"""Continuous-batching request loop for DP-AVF2 solves on one GPU.

A request is one KGS problem (dimension, N, parameters, time step), its
precision, a number of steps and an initial state.  The server owns one
kgs batch whose arena is the device-memory budget.  Each turn of the loop:

  1. admits waiting requests, in arrival order, while the arena has a free
     range for the request's state and a slot is free (a request that does
     not fit waits; later ones do not overtake it, so admission is FIFO);
  2. advances admitted requests by min(quantum, steps left) DP-AVF2 steps in
     one batched launch sequence (kgs_batch_step_each: requests of all sizes
     and precisions share each colour-pass launch).  Which requests a turn
     advances: all of them by default; with a work target, shortest remaining
     work first (point-updates left) until the turn holds that many
     point-updates -- enough to keep the GPU busy -- plus every request that
     has waited longer than the aging limit, so large requests are not
     starved.  Shortest-remaining-work-first lets small requests finish
     within the first turns instead of waiting out turns dominated by large
     ones, which lowers mean and median latency at about the same throughput;
  3. completes the requests with no steps left: reads their state and
     invariants back, records the latency (completion - arrival) and removes
     them, which returns their memory for the next admissions.

States stay on the device from admission to completion.  The batch steps
every instance exactly as a solo run would (the same pointwise code), so a
result does not depend on what else was in the mix (tests check bitwise).
"""
from __future__ import annotations

import collections
import concurrent.futures
import time
from dataclasses import dataclass, field
from typing import Callable, Deque, Dict, List, Optional, Sequence, Tuple

import numpy as np

from .solver import KGS_FP64, Batch, KGSError


@dataclass
class Request:
    rid: int
    prob: object              # inputs.Problem
    nsteps: int
    state: Callable[[], Tuple[np.ndarray, ...]]  # builds (P, Q, U, V) on the host
    precision: int = KGS_FP64
    arrival: float = 0.0      # seconds after the server's start


@dataclass
class Result:
    rid: int
    state: Tuple[np.ndarray, ...]
    energy0: float
    energy: float
    scale: float
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def energy_drift(self) -> float:
        return abs(self.energy - self.energy0) / self.scale


def state_bytes(prob, precision: int) -> int:
    return prob.points * 4 * (8 if precision == KGS_FP64 else 4)


@dataclass
class _Active:
    req: Request
    inst: int
    left: int
    energy0: float
    scale0: float
    admitted: float
    last_turn: float = 0.0  # when a turn last advanced it (admission time at first)


class Server:
    def __init__(self, budget_bytes: int, quantum: int = 100, max_slots: int = 256,
                 device: int = -1, clock: Callable[[], float] = time.perf_counter,
                 stream=None, keep_state: bool = True, prepare_ahead: int = 8,
                 turn_work: float = 0.0, max_wait: float = 5.0,
                 batch_options: Optional[Dict[int, int]] = None):
        self.batch = Batch(budget_bytes, device)
        # launch shapes (kgs_batch_set_option), e.g. the autotuner's per-list
        # persistent CTAs from tuned_batch_options
        for k, v in (batch_options or {}).items():
            self.batch.set_option(k, v)
        self.budget = budget_bytes
        self.quantum = quantum
        # shortest-remaining-work-first turns: point-updates per turn (0: advance
        # every admitted request each turn) and the aging limit in seconds
        self.turn_work = turn_work
        self.max_wait = max_wait
        self.max_slots = max_slots
        self.clock = clock
        self.stream = stream
        self.keep_state = keep_state
        self.pending: Deque[Request] = collections.deque()
        self.active: Dict[int, _Active] = {}
        self.results: List[Result] = []
        self.t0: Optional[float] = None
        self.turns = 0
        self.point_updates = 0
        # initial states of the next waiting requests are built on host threads
        # while the GPU steps the admitted ones (numpy releases the GIL)
        self.prepare_ahead = prepare_ahead
        self._pool = concurrent.futures.ThreadPoolExecutor(max_workers=4) if prepare_ahead else None
        self._prepared: Dict[int, concurrent.futures.Future] = {}

    def close(self):
        if self._pool is not None:
            self._pool.shutdown(wait=True)
            self._pool = None
        self.batch.close()

    def _prefetch(self):
        if self._pool is None:
            return
        for req in list(self.pending)[:self.prepare_ahead]:
            if req.rid not in self._prepared:
                self._prepared[req.rid] = self._pool.submit(req.state)

    def _initial_state(self, req: Request):
        fut = self._prepared.pop(req.rid, None)
        return fut.result() if fut is not None else req.state()

    def submit(self, req: Request):
        if state_bytes(req.prob, req.precision) + 256 > self.budget:
            # cannot fit even in an empty arena: it would wait forever
            raise KGSError(-3, f"request {req.rid} needs more memory than the budget")
        self.pending.append(req)

    def now(self) -> float:
        return self.clock() - self.t0

    def _admit(self):
        while self.pending and len(self.active) < self.max_slots:
            req = self.pending[0]
            if req.arrival > self.now():
                break
            if state_bytes(req.prob, req.precision) > self.batch.free_bytes():
                break  # FIFO: wait for memory
            inst = self.batch.add(req.prob, req.precision)
            self.batch.set_state(inst, *self._initial_state(req), stream=self.stream)
            E0, S0, _ = self.batch.invariants(inst, stream=self.stream)
            t = self.now()
            self.active[inst] = _Active(req, inst, req.nsteps, E0, S0, t, t)
            self.pending.popleft()

    def _turn_selection(self) -> List[int]:
        """Instances this turn advances (see the module docstring)."""
        items = [(i, a.req.prob.points, a.left, a.last_turn) for i, a in self.active.items()]
        return select_turn(items, self.quantum, self.turn_work, self.max_wait, self.now())

    def _complete(self, a: _Active):
        state = self.batch.get_state(a.inst, stream=self.stream) if self.keep_state else ()
        E, S, _ = self.batch.invariants(a.inst, stream=self.stream)
        self.batch.remove(a.inst)
        self.results.append(Result(a.req.rid, state, a.energy0, E, max(a.scale0, S),
                                   a.req.arrival, a.admitted, self.now()))

    def run(self, until_empty: bool = True) -> List[Result]:
        """Serve until every submitted request has completed."""
        if self.t0 is None:
            self.t0 = self.clock()
        while self.pending or self.active:
            self._prefetch()
            self._admit()
            if not self.active:
                # nothing on the device: wait for the next arrival
                nxt = self.pending[0].arrival
                while self.now() < nxt:
                    time.sleep(min(1e-3, max(0.0, nxt - self.now())))
                continue
            size = max(self.active) + 1
            counts = [0] * size
            for inst in self._turn_selection():
                counts[inst] = min(self.quantum, self.active[inst].left)
            self.batch.step_each(counts, stream=self.stream)
            self.turns += 1
            self._prefetch()  # host work overlaps the launches just queued
            for inst, a in list(self.active.items()):
                n = counts[inst]
                a.left -= n
                if n:
                    a.last_turn = self.now()
                self.point_updates += a.req.prob.points * n
                if a.left == 0:
                    self._complete(a)
                    del self.active[inst]
            if not until_empty:
                break
        return self.results


def tuned_batch_options(tuner, members, nsteps: int = 8, stream=None, device: int = -1) -> Dict[int, int]:
    """Per-list persistent CTAs per SM for serving a mix like `members` (a
    list of (problem, precision)): the tuner times them on a batch of those
    problems holding zero states (timing does not depend on the values), and
    the choice is returned as batch options for Server(batch_options=...)."""
    import torch
    from . import tune
    need = sum(state_bytes(p, prec) + 512 for p, prec in members)
    b = Batch(need + (16 << 20), device)
    try:
        for p, prec in members:
            i = b.add(p, prec)
            z = torch.zeros((p.N,) * p.dim, dtype=torch.float64, device="cuda")
            b.set_state(i, z, z, z, z, stream=stream)
        chosen = tuner.tune_batch_lists(b, members, nsteps=nsteps, stream=stream)
    finally:
        b.close()
    opts = {}
    for p, prec in members:
        name = tune.list_name(prec, p.dim)
        if name in chosen:
            opts[tune.list_option(prec, p.dim)] = chosen[name]
    return opts


def select_turn(items, quantum: int, turn_work: float, max_wait: float, now: float) -> List[int]:
    """Instances one turn advances.  items: (instance, points, steps left, time
    a turn last advanced it).  turn_work <= 0: all of them.  Otherwise in
    increasing remaining work (points x steps left; ties by instance) while
    the turn holds fewer than turn_work point-updates, and every instance not
    advanced for more than max_wait seconds."""
    if turn_work <= 0:
        return [i for i, _, _, _ in items]
    chosen, work = [], 0.0
    for inst, pts, left, last in sorted(items, key=lambda x: (x[1] * x[2], x[0])):
        if work < turn_work or now - last > max_wait:
            chosen.append(inst)
            work += min(quantum, left) * pts
    return chosen


def percentile(xs: Sequence[float], q: float) -> float:
    return float(np.percentile(np.asarray(xs, dtype=float), q)) if len(xs) else float("nan")


def poisson_requests(rate: float, count: int, seed: int, step_range=(100, 10000),
                     precisions=(KGS_FP64, 0)) -> List[Request]:
    """Requests shaped like the serving workload: dim uniform in {1,2,3}, N
    uniform (even) in [256,8192] (1D), [128,2048] (2D), [64,384] (3D), steps
    uniform in step_range, kappa1, kappa2 ~ U[0.5,2], mu ~ U[0.5,1.5],
    gamma ~ U[0.5,2], tau = 5e-4, FP64 or FP32 with equal probability (pass
    precisions=(KGS_FP64,) for FP64 only), Gaussian-bump initial data, and
    exponential inter-arrival times of mean 1/rate seconds."""
    from . import inputs
    from .solver import KGS_FP32
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate))
        dim = int(rng.integers(1, 4))
        lo, hi, L = {1: (256, 8192, 80.0), 2: (128, 2048, 40.0), 3: (64, 384, 20.0)}[dim]
        N = 2 * int(rng.integers(lo // 2, hi // 2 + 1))
        prob = inputs.Problem(dim, N, L, float(rng.uniform(0.5, 2)), float(rng.uniform(0.5, 2)),
                              float(rng.uniform(0.5, 1.5)), float(rng.uniform(0.5, 2)), 5e-4)
        nsteps = int(rng.integers(step_range[0], step_range[1] + 1))
        choices = [p if p else KGS_FP32 for p in precisions]
        precision = int(choices[int(rng.integers(0, len(choices)))])
        sub = int(rng.integers(0, 2 ** 62))

        def fn(prob=prob, sub=sub):
            return inputs.gaussian_bump(prob, np.random.Generator(np.random.PCG64(sub)))
        out.append(Request(k, prob, nsteps, fn, precision, t))
    return out
