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


# ---------------------------------------------------------------- one grid --
# One N^d grid (d = 2 or 3) shared by the ranks as slabs of axis-0 planes.
# A colour pass updates one colour from the other colour's values, and the
# only cross-slab reads are the neighbours on the planes just below and just
# above a slab: so before every colour pass each rank sends its first and last
# planes of (P, Q, U) to the ranks below and above (V is never read at another
# point), and the red-first colouring stays global because a rank's points
# keep their global indices.  The invariants need the plane above a slab (the
# forward differences) and then one all-reduce of three sums.  The per-pass
# compute is the caller's (the colour-pass kernels on a GPU); this module
# holds the partition, the exchange and the schedule.

# the fused colour passes of a run of n steps (the same sequence as kgs_step):
# red base, (black base+adjoint, red adjoint+next base) x (n - 1), black, red adjoint
PASS_RED_BASE, PASS_BLACK_FUSED, PASS_RED_FUSED, PASS_RED_ADJ = 0, 1, 2, 3


def fused_pass_sequence(nsteps: int) -> List[int]:
    if nsteps < 1:
        return []
    return ([PASS_RED_BASE] + [PASS_BLACK_FUSED, PASS_RED_FUSED] * (nsteps - 1)
            + [PASS_BLACK_FUSED, PASS_RED_ADJ])


def slab_planes(N: int, world: int) -> List[Tuple[int, int]]:
    """(first plane, plane count) of every rank's slab along axis 0, in rank
    order, as equal as possible and at least one plane each."""
    if world < 1 or world > N:
        raise ValueError("need 1 <= world <= N")
    base, extra = divmod(N, world)
    out, p = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((p, n))
        p += n
    return out


class Slab:
    """This rank's slab of an N^d periodic grid: global planes [p0, p0 + n),
    held in arrays of n + 2 planes whose first and last are the halo planes
    p0 - 1 and p0 + n (mod N).  Works with torch tensors on any
    torch.distributed backend (gloo on CPU, NCCL on GPUs)."""

    TAG_TO_LOWER, TAG_TO_UPPER = 7001, 7002

    def __init__(self, dim: int, N: int, rank: int, world: int, group=None):
        if dim not in (2, 3):
            raise ValueError("slabs cut 2D and 3D grids")
        self.dim, self.N, self.rank, self.world, self.group = dim, N, rank, world, group
        self.p0, self.n = slab_planes(N, world)[rank]
        self.lower, self.upper = (rank - 1) % world, (rank + 1) % world

    def local_shape(self) -> Tuple[int, ...]:
        return (self.n + 2,) + (self.N,) * (self.dim - 1)

    def take(self, full):
        """This rank's planes of a whole-grid array, with (unfilled) halo planes."""
        import torch
        out = torch.zeros(self.local_shape(), dtype=full.dtype, device=full.device)
        out[1:self.n + 1] = full[self.p0:self.p0 + self.n]
        return out

    def exchange(self, fields) -> None:
        """Fill the halo planes of each local field: plane 0 from the rank
        below (its last plane), plane n + 1 from the rank above (its first)."""
        import torch
        import torch.distributed as dist
        if self.world == 1:
            for f in fields:
                f[0] = f[self.n]
                f[self.n + 1] = f[1]
            return
        reqs, recvs = [], []
        for k, f in enumerate(fields):
            # one tag per field and direction: with two ranks the rank below
            # and the rank above are the same process
            to_lower, to_upper = self.TAG_TO_LOWER + 16 * k, self.TAG_TO_UPPER + 16 * k
            lo, hi = f[1].contiguous(), f[self.n].contiguous()
            got_lo, got_hi = torch.empty_like(lo), torch.empty_like(hi)
            reqs.append(dist.isend(lo, self.lower, group=self.group, tag=to_lower))
            reqs.append(dist.isend(hi, self.upper, group=self.group, tag=to_upper))
            reqs.append(dist.irecv(got_lo, self.lower, group=self.group, tag=to_upper))
            reqs.append(dist.irecv(got_hi, self.upper, group=self.group, tag=to_lower))
            recvs.append((f, got_lo, got_hi))
        for r in reqs:
            r.wait()
        for f, got_lo, got_hi in recvs:
            f[0] = got_lo
            f[self.n + 1] = got_hi

    def run(self, P, Q, U, V, nsteps: int, pass_fn) -> None:
        """nsteps DP-AVF2 steps of the whole grid: before every fused colour
        pass the halos of P, Q, U are exchanged, then pass_fn(mode, slab, P, Q,
        U, V) updates this slab's points of the pass's colour in place."""
        for mode in fused_pass_sequence(nsteps):
            self.exchange([P, Q, U])
            pass_fn(mode, self, P, Q, U, V)

    def invariants(self, P, Q, U, V, partial_fn) -> Tuple[float, float, float]:
        """(E_h, S_E, mass) of the whole grid: partial_fn(slab, P, Q, U, V)
        returns this slab's three sums (its planes, forward differences into
        the halo plane above), and one all-reduce adds them."""
        import torch
        import torch.distributed as dist
        self.exchange([P, Q, U, V])
        part = torch.tensor(list(partial_fn(self, P, Q, U, V)), dtype=torch.float64)
        if self.world > 1:
            dist.all_reduce(part, op=dist.ReduceOp.SUM, group=self.group)
        return float(part[0]), float(part[1]), float(part[2])
