"""Sharding of independent analyses over ranks (one GPU per rank).

Candidates x input directions are independent wave analyses (the paper runs
its 708 analyses on 44 GPUs with no communication), so ranks exchange no data
on the hot path: each rank takes a DOF-balanced share of the analyses, and
only the wall time (max over ranks) and the final ERR table cross ranks.
"""
import heapq


def assign(costs, world):
    """Greedy longest-first partition of analyses over `world` ranks.

    ``costs``: per-analysis cost (e.g. DOF x steps).  Returns a list of index
    lists, one per rank; deterministic (ties broken by index and rank).
    """
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    shares = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shares[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(s) for s in shares]


def max_over_ranks(value, dist=None):
    """Maximum of a float over all ranks (the job's wall time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def gather_table(local, dist=None):
    """Merge per-rank {analysis index: result} dicts on every rank."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return dict(local)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, dict(local))
    out = {}
    for p in parts:
        out.update(p)
    return out
