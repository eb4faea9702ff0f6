"""Sharding of independent grids across ranks (one process per GPU).

Grids share nothing, so a batch shards without any data-path collective:
each rank solves its own grids.  Assignment is the longest-processing-time
rule on vertex counts (largest grid first, to the least-loaded rank, ties by
rank), identical on every rank because it depends only on the grid sizes.
"""
from __future__ import annotations

import heapq


def assign(sizes, world: int):
    """Rank of every grid (list, same order as `sizes`)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda g: (-int(sizes[g]), g))
    heap = [(0, r) for r in range(world)]
    owner = [0] * len(sizes)
    for g in order:
        load, r = heapq.heappop(heap)
        owner[g] = r
        heapq.heappush(heap, (load + int(sizes[g]), r))
    return owner


def shard(dims_list, rank: int, world: int):
    """Indices of the grids (H, W) that `rank` of `world` solves."""
    owner = assign([h * w for h, w in dims_list], world)
    return [g for g, r in enumerate(owner) if r == rank]
