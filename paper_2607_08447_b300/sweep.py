"""Sharding of a detuning / gate-voltage sweep over ranks (one GPU each).

Sweep points are independent problems (the single-particle problem is
re-solved for every detuning point, Sec. II C of the paper), so a sweep
shards with no data-path collective: every rank solves its own subset and
only the timing is reduced.  The partition is greedy longest-processing-time
on the unknowns of each point, which balances uneven grid sizes.
"""
from __future__ import annotations

from typing import List, Sequence


def partition_sweep(costs: Sequence[float], world: int) -> List[List[int]]:
    """Indices of the sweep points per rank: largest cost first onto the
    least-loaded rank (ties to the lowest rank); each rank's list is sorted."""
    if world < 1:
        raise ValueError("world must be >= 1")
    loads = [0.0] * world
    shards: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        r = min(range(world), key=lambda q: (loads[q], q))
        shards[r].append(i)
        loads[r] += float(costs[i])
    return [sorted(s) for s in shards]


def shard_of(costs: Sequence[float], rank: int, world: int) -> List[int]:
    return partition_sweep(costs, world)[rank]
