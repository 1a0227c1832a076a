"""Host-side sharding of the chi0 path over ranks (one process per GPU).

The path has no exchange step: q-points (and frequencies) are independent problems, so N
ranks take disjoint sets of q-points and no collective touches the data.  The only
collective is the benchmark's timing reduction (max over ranks).
"""
from __future__ import annotations

from typing import Sequence


def qpoint_shard(costs: Sequence[float], rank: int, world: int) -> list[int]:
    """Indices of the q-points rank `rank` computes: largest-first greedy onto the least
    loaded rank (deterministic, identical on every rank, disjoint and covering)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    owner = [0] * len(costs)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += costs[i]
    return [i for i in range(len(costs)) if owner[i] == rank]


def max_over_ranks(value: float, device=None) -> float:
    """Max of a float over all ranks of the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
