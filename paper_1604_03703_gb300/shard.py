"""Sharding of a batch of independent matrices over ranks (one GPU each).

The matrices of a batch are independent problems, so N GPUs process
disjoint subsets with no data-path collective: longest-processing-time-first
(LPT) assignment on the O(n^3) cost of a dense eigensolve, computed by every
rank from the same sizes (deterministic, so no communication is needed to
agree on it).  Results stay on the rank that computed them; `gather_order`
gives the permutation that puts a host-side concatenation back in batch
order."""
from __future__ import annotations

import heapq
from typing import List, Sequence


def lpt_partition(sizes: Sequence[int], world: int) -> List[List[int]]:
    """Indices of the matrices assigned to each of `world` ranks: largest
    cost first onto the least-loaded rank (ties: lower rank, lower index)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]) ** 3, i))
    heap = [(0, r) for r in range(world)]
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]) ** 3, r))
    for p in parts:
        p.sort()
    return parts


def loads(sizes: Sequence[int], parts: List[List[int]]) -> List[int]:
    return [sum(int(sizes[i]) ** 3 for i in p) for p in parts]


def gather_order(parts: List[List[int]]) -> List[int]:
    """Position in the rank-by-rank concatenation of each batch index."""
    flat = [i for p in parts for i in p]
    pos = [0] * len(flat)
    for k, i in enumerate(flat):
        pos[i] = k
    return pos
