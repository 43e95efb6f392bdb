"""Placement of independent sensor instances on ranks (one GPU each).

The batched and serving forms step instances that never exchange data, so
several GPUs share a set of instances without any collective in the step:
each rank owns whole instances.  The work of an instance is proportional to
its particle count (every substep touches every particle), so the set is
split by greedy bin packing, longest first (Graham's LPT rule): instances in
decreasing particle count, each to the rank with the fewest particles so far.
With that rule the most and least loaded ranks differ by at most the largest
instance: when the last instance went to the most loaded rank, that rank was
the least loaded, so its final load minus that instance is at most every
other rank's final load.
"""
from __future__ import annotations

import heapq


def bin_pack(sizes, world):
    """Split instances of the given sizes over `world` ranks, longest first.

    Returns (owners, loads): owners[r] lists the instance indices of rank r in
    increasing order, loads[r] their total size.  Ties go to the lower index
    and the lower rank, so every rank computes the same split."""
    if world < 1:
        raise ValueError("world must be at least 1")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    heap = [(0, r) for r in range(world)]
    owners = [[] for _ in range(world)]
    loads = [0] * world
    for i in order:
        load, r = heapq.heappop(heap)
        owners[r].append(i)
        loads[r] = load + sizes[i]
        heapq.heappush(heap, (loads[r], r))
    return [sorted(o) for o in owners], loads


def round_robin(n, world, rank):
    """Indices of n queries that rank `rank` of `world` serves (i % world)."""
    return list(range(rank, n, world))
