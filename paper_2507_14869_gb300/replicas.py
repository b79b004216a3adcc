"""Data-parallel replicas over one process per GPU.

Chains, images and serving requests are independent (every draw is keyed
by its own chain id, sweep and site), so several GPUs run disjoint work with
no collective on the data path.  This module holds the host logic around
that: a deterministic longest-processing-time assignment of work items to
ranks, a chain-id scheme that keeps every replica's uniforms distinct, and
the two reductions a run reports through (the slowest rank's time, the
gathered per-item results).  It uses torch.distributed only when a process
group is initialised; the backend is whatever the caller chose (NCCL on
GPUs, gloo on the host).
"""
from __future__ import annotations

import heapq


def shard(costs, world: int):
    """Assign item indices to `world` ranks: items by decreasing cost (ties by
    index), each to the currently least-loaded rank (ties by rank).  Returns
    one list of item indices per rank, each in increasing order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(x) for x in out]


def chain_id(rank: int, local: int, per_rank: int) -> int:
    """Chain id of the local-th chain on `rank` when every rank runs
    `per_rank` chains: distinct over all ranks, below 2^24."""
    cid = rank * per_rank + local
    if not 0 <= local < per_rank or cid >= (1 << 24):
        raise ValueError("chain id out of range")
    return cid


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def max_time(t_local: float) -> float:
    """The slowest rank's time (the run's time under weak scaling)."""
    dist = _dist()
    if dist is None:
        return float(t_local)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather(local: dict) -> dict:
    """Union of every rank's {item index: result}."""
    dist = _dist()
    if dist is None:
        return dict(local)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, dict(local))
    out = {}
    for p in parts:
        for k, v in p.items():
            if k in out:
                raise ValueError(f"item {k} reported by two ranks")
            out[k] = v
    return out


def aggregate_rate(units_per_rank: float, t_local: float, world: int) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / max_time(t_local)
