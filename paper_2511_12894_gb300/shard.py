"""Sharding of reference groups across ranks (one process per GPU).

Reference groups are independent (Sec. III.A of the paper): each group needs only the
data segment and its own kernels, so ranks take whole groups and the online path needs no
collective.  Groups are assigned longest-processing-time first: sorted by estimated cost,
each goes to the rank with the least work so far (ties to the lowest rank).  The cost of a
group is its number of templates times the segment length, plus the reconstruction work of
its neighbours, which grows with their kernel lengths.  A single group is split by its
neighbours instead (contiguous runs, every rank filtering the one reference).

The one exchange is the final gather of the window peaks: every rank's rows go to rank 0,
which places them in the global row order (references first, then the neighbours of each
group in group order, as one process would produce them).

Host logic plus one torch.distributed gather; exercised by multi-process ``gloo`` tests on
the CPU.
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


def split_neighbours(k: int, world: int, rank: int) -> range:
    """Contiguous run of a single group's k neighbours for `rank` (sizes differ by at most one)."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    q, r = divmod(k, world)
    lo = rank * q + min(rank, r)
    return range(lo, lo + q + (1 if rank < r else 0))


def global_rows(group_sizes: Sequence[int], groups: Sequence[int]) -> List[int]:
    """Global row indices, in local order, of the neighbour rows of `groups` (a rank's groups in
    the order it computes them), where the neighbours of group g occupy rows
    [sum(group_sizes[:g]), sum(group_sizes[:g + 1]))."""
    starts = [0]
    for k in group_sizes:
        starts.append(starts[-1] + int(k))
    out: List[int] = []
    for g in groups:
        out.extend(range(starts[g], starts[g + 1]))
    return out


def gather_rows(local, rows_of_rank: Sequence[Sequence[int]], total_rows: int, rank: int, world: int, dist):
    """Gather every rank's rows of `local` ([len(rows_of_rank[rank]), ...] tensor) to rank 0.

    Rank 0 returns a [total_rows, ...] tensor with each rank's row i at rows_of_rank[r][i];
    the other ranks return None.  Ranks hold different row counts, so every rank pads to the
    largest count before the collective (torch.distributed.gather wants equal shapes)."""
    import torch
    counts = [len(r) for r in rows_of_rank]
    if local.shape[0] != counts[rank]:
        raise ValueError("local rows do not match this rank's assignment")
    width = tuple(local.shape[1:])
    mx = max(counts) if counts else 0
    buf = torch.zeros((mx,) + width, dtype=local.dtype, device=local.device)
    buf[: counts[rank]] = local
    bufs = [torch.empty_like(buf) for _ in range(world)] if rank == 0 else None
    dist.gather(buf, gather_list=bufs, dst=0)
    if rank != 0:
        return None
    out = torch.zeros((total_rows,) + width, dtype=local.dtype, device=local.device)
    for r in range(world):
        if counts[r]:
            idx = torch.as_tensor(list(rows_of_rank[r]), dtype=torch.long, device=local.device)
            out[idx] = bufs[r][: counts[r]]
    return out
