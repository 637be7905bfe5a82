"""Host-side multi-process helpers (one process per GPU).

The solves shard by independent problems: lattices of an uneven batch (or
replicas of one workload) are assigned to ranks, each rank solves its share on
its own GPU, and no field data crosses ranks.  Only the timing and the
aggregate throughput are combined: the slowest rank's time bounds the job,
and the job's value is all ranks' work over that time.
"""
from __future__ import annotations

from typing import List, Sequence


def shard_by_cost(costs: Sequence[float], world: int) -> List[List[int]]:
    """Assign items (e.g. lattices, by site count x right-hand sides) to `world`
    ranks, largest first onto the least-loaded rank (longest-processing-time
    rule).  Returns the item indices of every rank, each list in ascending order;
    deterministic for equal costs (lower index first, lower rank first)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def job_time(local_seconds: float, group=None) -> float:
    """The job's time: the maximum over ranks of each rank's timed region."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(local_seconds)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def job_work(local_units: float, group=None) -> float:
    """The work all ranks did together (sum over ranks)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(local_units)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(local_units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())
