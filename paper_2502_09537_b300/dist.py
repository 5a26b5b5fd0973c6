"""Host-side multi-GPU helpers: one process per GPU, independent work per rank.

The DP-AVF2 instances of a batch or a request stream are independent, so N
GPUs run N disjoint shares of them with no data-path collective (weak
scaling).  The only collectives are the timing ones a benchmark needs: a
barrier before and after the timed region and the maximum of the ranks'
elapsed times.  These helpers work on any torch.distributed backend (gloo on
CPU in the tests, NCCL on GPUs).
"""
from __future__ import annotations

import os
from typing import List, Sequence, Tuple, TypeVar

T = TypeVar("T")


def rank_world() -> Tuple[int, int]:
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def shard(items: Sequence[T], rank: int, world: int, weights: Sequence[float] = None) -> List[T]:
    """This rank's share of items.  Without weights, round-robin.  With
    weights (e.g. point-updates per instance), greedy longest-processing-time
    assignment: items in decreasing weight go to the least loaded rank, ties
    to the lowest rank -- deterministic, so every rank computes the same
    partition without communicating."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    if weights is None:
        return [x for k, x in enumerate(items) if k % world == rank]
    if len(weights) != len(items):
        raise ValueError("one weight per item")
    order = sorted(range(len(items)), key=lambda k: (-weights[k], k))
    load = [0.0] * world
    owner = [0] * len(items)
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[k] = r
        load[r] += weights[k]
    return [items[k] for k in range(len(items)) if owner[k] == rank]


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a float over the default process group (identity when
    torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
