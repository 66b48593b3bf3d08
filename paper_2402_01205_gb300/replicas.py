"""Replica placement for several GPUs (one process per GPU).

Time frames are independent (the paper distributes them round-robin over the
GPUs with no GPU intercommunication, Sec. 6), so multi-GPU runs are replicas:
each rank fits whole frames and no collective touches the data path.  Only
the benchmark's timing uses a collective (max over ranks).
"""
from __future__ import annotations


def shard_round_robin(n_items: int, rank: int, world: int) -> list:
    """Indices of the frames (or events) rank `rank` of `world` fits: round robin."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return list(range(rank, n_items, world))


def shard_balanced(sizes, rank: int, world: int) -> list:
    """Largest-first greedy assignment of items with the given sizes (clusters)
    to the least-loaded rank; returns this rank's item indices (deterministic)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += sizes[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank scalar over the default process group (timing only)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t)
    return float(t.item())
