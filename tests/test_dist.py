"""Multi-rank host logic with gloo on CPU, world size 2: the instance shards
are disjoint and cover the batch, every rank derives the same partition, and
the timing reduction returns the slowest rank's time."""
import os

import pytest
import torch.multiprocessing as mp

from paper_2502_09537_b300 import dist as kdist
from paper_2502_09537_b300 import inputs


def test_shard_round_robin_and_weighted():
    items = list(range(10))
    parts = [kdist.shard(items, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == items
    w = [p.points * n for p, n, _ in inputs.batched_instances()]
    ids = list(range(len(w)))
    parts = [kdist.shard(ids, r, 4, w) for r in range(4)]
    assert sorted(sum(parts, [])) == ids
    loads = [sum(w[k] for k in part) for part in parts]
    assert max(loads) / min(loads) < 1.1          # balanced by point-updates
    with pytest.raises(ValueError):
        kdist.shard(items, 3, 3)


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = [p.points * n for p, n, _ in inputs.batched_instances()]
    mine = kdist.shard(list(range(len(w))), rank, world, w)
    elapsed = 1.0 + rank          # rank 1 is the slower one
    slowest = kdist.max_over_ranks(elapsed)
    total = kdist.sum_over_ranks(len(mine))
    dist.barrier()
    out.put((rank, mine, slowest, total))
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, s0, t0), (r1, m1, s1, t1) = res
    assert set(m0).isdisjoint(m1) and sorted(m0 + m1) == list(range(96))
    assert s0 == s1 == 2.0
    assert t0 == t1 == 96
