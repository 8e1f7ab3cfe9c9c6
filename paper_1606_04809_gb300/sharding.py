"""Placement of independent problem instances on ranks (one GPU per rank).

A single ASAGA instance needs one shared iterate with atomic adds, so it
does not split across GPUs; a batch of independent instances does.  Each
rank solves its own share with no exchange on the data path; only the
timing is reduced (max over ranks) at the end.  Shares are balanced by an
estimated cost per instance (nonzeros times expected epochs) with the
longest-processing-time rule: instances sorted by decreasing cost, each
given to the currently least-loaded rank (ties: lowest rank, then index).
"""
from __future__ import annotations

import heapq
from typing import Sequence


def shard_instances(costs: Sequence[float], world: int) -> list:
    """Instance indices of every rank, each list in increasing order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    shares = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shares[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(s) for s in shares]


def rank_instances(costs: Sequence[float], world: int, rank: int) -> list:
    return shard_instances(costs, world)[rank]


def instance_cost(p, epochs: float = 1.0) -> float:
    """Work estimate of one instance: nonzeros (at least n) times epochs."""
    return float(max(p.nnz, p.n)) * float(epochs)
