"""Sharding of independent voting problems across ranks (one GPU per rank).

Problems of a batch are independent (no exchange step), so ranks split them and
solve their share with no collective on the data path; only the small results
are gathered at the end.  The split is greedy by size: problems in decreasing n,
each to the least loaded rank (ties to the lower rank), which is deterministic
and balances sum(n) per rank.
"""
from __future__ import annotations

import heapq


def partition(sizes, world: int) -> list[list[int]]:
    """Problem indices per rank (each sorted ascending)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i)):
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]), r))
    return [sorted(x) for x in out]


def solve_sharded(solve_one, problems, rank: int, world: int, group=None):
    """Solve this rank's share with ``solve_one(problem) -> result`` and gather every
    rank's results; returns the list of results in problem order on every rank."""
    import torch.distributed as dist
    mine = partition([p.n for p in problems], world)[rank]
    local = {i: solve_one(problems[i]) for i in mine}
    if world == 1:
        return [local[i] for i in range(len(problems))]
    gathered = [None] * world
    dist.all_gather_object(gathered, local, group=group)
    merged = {}
    for part in gathered:
        merged.update(part)
    return [merged[i] for i in range(len(problems))]
