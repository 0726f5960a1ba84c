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


def request_cost(m, n, nrhs, fresh):
    """Work of one least-squares request in flops: the factorization
    2 m n^2 - 2 n^3 / 3 when its matrix is not resident on the rank, plus
    Q^T B and the back substitution (4 m n + n^2 per right-hand side)."""
    f = 2.0 * m * n * n - 2.0 * n ** 3 / 3.0 if fresh else 0.0
    return f + nrhs * (4.0 * m * n + n * n)


def route_requests(reqs, world):
    """Rank of every request of a served stream, in arrival order.

    A request whose matrix has been seen goes to the rank that factored it
    (its factorization stays resident there); a new matrix goes to the rank
    with the least work routed so far (ties to the lower rank).  Every rank
    computes the same routing from the same stream, so requests are
    partitioned with no message between ranks.  ``reqs`` are dicts with
    "matrix", "m", "n" and "nrhs" (as inputs.serving_stream makes them).
    Returns (rank per request, owning rank per matrix id)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    owner = {}
    out = []
    for q in reqs:
        mid = q["matrix"]
        fresh = mid not in owner
        if fresh:
            owner[mid] = min(range(world), key=lambda r: (load[r], r))
        r = owner[mid]
        load[r] += request_cost(q["m"], q["n"], q["nrhs"], fresh)
        out.append(r)
    return out, owner
