"""Host-side helpers for running independent problems on several GPUs, one
process per GPU (replicas of one factorization, or the instances of a batch
or of a request stream sharded across ranks).  No method arithmetic lives
here and no collective touches the data: ranks only agree on the slowest
rank's time and on totals.

A single tiled factorization is not split across GPUs: every step would
broadcast V and T along tile rows and columns (the paper lists distributed
memory as future work), so it runs as independent replicas.
"""
import heapq


def shard_by_cost(costs, world):
    """Greedy longest-processing-time placement: instances in decreasing cost
    order, each to the rank with the least total so far (ties to the lower
    rank).  Returns one list of instance indices per rank, each in increasing
    index order.  Deterministic, so every rank computes the same shards."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda a: (-costs[a], a))
    heap = [(0.0, r) for r in range(world)]
    shards = [[] for _ in range(world)]
    for a in order:
        load, r = heapq.heappop(heap)
        shards[r].append(a)
        heapq.heappush(heap, (load + costs[a], r))
    return [sorted(s) for s in shards]


def max_over_ranks(value, dist=None, device=None):
    """The largest value over all ranks (the job's time is its slowest
    rank's); identity without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, dist=None, device=None):
    """The total of a per-rank count (units processed) over all ranks."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
