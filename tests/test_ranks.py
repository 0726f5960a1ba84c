"""Host logic of the multi-GPU runs (independent problems sharded over
ranks, no data collective), checked on the CPU, including two gloo ranks."""
import os
import socket

import numpy as np
import pytest

from paper_0707_3548_gb300 import inputs
from paper_0707_3548_gb300.ranks import max_over_ranks, route_requests, shard_by_cost, sum_over_ranks


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


@pytest.mark.parametrize("world", [1, 2, 4])
def test_routing_keeps_repeat_requests_with_their_factor_and_balances(world):
    reqs, mats = inputs.serving_stream(400.0, 1.0, seed=0)
    ranks, owner = route_requests(reqs, world)
    assert len(ranks) == len(reqs) and all(0 <= r < world for r in ranks)
    first = {}
    for r, q in zip(ranks, reqs):
        first.setdefault(q["matrix"], r)
        assert r == first[q["matrix"]] == owner[q["matrix"]]   # repeat-A stays with the factor
    from paper_0707_3548_gb300.ranks import request_cost
    seen, loads = set(), [0.0] * world
    for r, q in zip(ranks, reqs):
        loads[r] += request_cost(q["m"], q["n"], q["nrhs"], q["matrix"] not in seen)
        seen.add(q["matrix"])
    biggest = max(request_cost(q["m"], q["n"], q["nrhs"], True) for q in reqs)
    assert max(loads) - min(loads) <= biggest                 # greedy balance
    assert route_requests(reqs, world)[0] == ranks             # deterministic


def _serve_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        reqs, _ = inputs.serving_stream(300.0, 1.0, seed=2)
        ranks, owner = route_requests(reqs, world)
        # this rank "serves" its requests: it records which it handled and
        # which matrices it factored (first sight) or reused (resident)
        served = torch.zeros(len(reqs), dtype=torch.int64)
        resident, reused_ok = set(), True
        for k, (r, q) in enumerate(zip(ranks, reqs)):
            if r != rank:
                continue
            served[k] = 1
            if q["matrix"] in resident:
                reused_ok = reused_ok and owner[q["matrix"]] == rank
            resident.add(q["matrix"])
        counts = served.clone()
        dist.all_reduce(counts, op=dist.ReduceOp.SUM)
        # a repeat-A request must reach the rank that holds its factor
        factored_here = torch.zeros(max(q["matrix"] for q in reqs) + 1, dtype=torch.int64)
        for mid in resident:
            factored_here[mid] = 1
        holders = factored_here.clone()
        dist.all_reduce(holders, op=dist.ReduceOp.SUM)
        out.put((rank, int(counts.min()), int(counts.max()), int(holders.max()), reused_ok,
                 int(served.sum())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_serve_each_request_once_with_resident_factors():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_serve_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    total = sum(r[5] for r in res)
    for rank, cmin, cmax, hmax, reused_ok, mine in res:
        assert cmin == 1 and cmax == 1      # every request served by exactly one rank
        assert hmax == 1                    # every matrix factored on one rank only
        assert reused_ok and mine > 0
    reqs, _ = inputs.serving_stream(300.0, 1.0, seed=2)
    assert total == len(reqs)
