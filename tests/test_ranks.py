"""Host logic of the multi-GPU runs (independent problems sharded over
ranks, no data collective), checked on the CPU, including two gloo ranks."""
import os
import socket

import numpy as np
import pytest

from paper_0707_3548_gb300 import inputs
from paper_0707_3548_gb300.ranks import max_over_ranks, shard_by_cost, sum_over_ranks


def _flops(shape):
    m, n = shape
    k = min(m, n)
    return 2.0 * max(m, n) * k * k - 2.0 * k ** 3 / 3.0


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shards_cover_every_instance_once_and_balance(world):
    costs = [_flops(s) for s in inputs.batch_shapes(500, seed=0)]
    shards = shard_by_cost(costs, world)
    assert len(shards) == world
    flat = sorted(a for s in shards for a in s)
    assert flat == list(range(len(costs)))
    loads = [sum(costs[a] for a in s) for s in shards]
    # longest-processing-time bound: no rank above the mean by more than one instance
    assert max(loads) <= sum(costs) / world + max(costs)
    assert shard_by_cost(costs, world) == shards              # deterministic


def test_more_ranks_than_instances():
    shards = shard_by_cost([3.0, 1.0], 4)
    assert sorted(len(s) for s in shards) == [0, 0, 1, 1]
    assert max_over_ranks(2.5) == 2.5 and sum_over_ranks(4.0) == 4.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = [_flops(s) for s in inputs.batch_shapes(200, seed=1)]
        shards = shard_by_cost(costs, world)
        mine = shards[rank]
        # every rank works on its own shard only; the job's totals
        units = float(len(mine))
        total = sum_over_ranks(units, dist)
        slowest = max_over_ranks(10.0 + rank, dist)
        import torch
        gathered = [torch.zeros(len(costs), dtype=torch.int64) for _ in range(world)]
        owner = torch.full((len(costs),), -1, dtype=torch.int64)
        owner[mine] = rank
        dist.all_gather(gathered, owner)
        merged = torch.stack(gathered).max(dim=0).values
        out.put((rank, total, slowest, bool((merged >= 0).all()),
                 int(((torch.stack(gathered) >= 0).sum(dim=0) == 1).all())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_shards_and_totals():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, slowest, covered, once in res:
        assert total == 200.0          # every instance processed by exactly one rank
        assert slowest == 11.0         # the job's time is the slower rank's
        assert covered and once
