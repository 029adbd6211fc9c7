"""Sharding of reference groups across ranks (one process per GPU).

Reference groups are independent (Sec. III.A of the paper): each group needs only the
data segment and its own kernels, so ranks take whole groups and the online path needs no
collective.  Groups are assigned longest-processing-time first: sorted by estimated cost,
each goes to the rank with the least work so far (ties to the lowest rank).  The cost of a
group is its number of templates times the segment length, plus the reconstruction work of
its neighbours, which grows with their kernel lengths.

Host logic only (no GPU): it is exercised by multi-process ``gloo`` tests on the CPU.
"""
from __future__ import annotations

import heapq
from typing import List, Sequence


def group_cost(n: int, kernel_lengths: Sequence[int], block: int = 16384, part: int = 4096) -> float:
    """Relative cost of one group: (1 + K) n for the matched filter and peaks, plus the
    overlap-save work of each neighbour: per output block of B - Lp samples, one block
    transform (~ log2 B) and P_j = ceil(L_j / Lp) spectral products."""
    import math
    recon = sum(math.log2(block) + max(1, -(-int(L) // part)) for L in kernel_lengths)
    return float(n) * (1 + len(kernel_lengths) + recon / math.log2(block) * block / (block - part))


def assign(costs: Sequence[float], world: int) -> List[List[int]]:
    """Partition group indices into `world` lists, longest processing time first."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    out: List[List[int]] = [[] for _ in range(world)]
    order = sorted(range(len(costs)), key=lambda g: (-costs[g], g))
    for g in order:
        load, r = heapq.heappop(heap)
        out[r].append(g)
        heapq.heappush(heap, (load + costs[g], r))
    for r in range(world):
        out[r].sort()
    return out


def my_groups(costs: Sequence[float], world: int, rank: int) -> List[int]:
    """The groups of `rank` (every rank computes the same assignment, no communication)."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return assign(costs, world)[rank]
