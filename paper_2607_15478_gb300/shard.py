"""Sharding independent alignments across ranks (one process per GPU).

A single pair's DP is one wavefront and does not shard; a batch of pairs
does, with no data-path exchange: every rank aligns its own share and the
results meet once at the end.  Shares are balanced with the greedy
longest-processing-time rule on the cell count La*Lb (the DP's work).
"""
from __future__ import annotations

import heapq
from typing import Callable, List, Sequence, Tuple


def partition_pairs(cells: Sequence[int], world_size: int) -> List[List[int]]:
    """Split pair indices over ranks, largest first onto the least-loaded rank.

    Deterministic (ties go to the lower rank), so every rank computes the
    same partition without communicating.  Each rank's list is ascending.
    """
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(cells)), key=lambda k: (-int(cells[k]), k))
    heap = [(0, r) for r in range(world_size)]
    shares: List[List[int]] = [[] for _ in range(world_size)]
    for k in order:
        load, r = heapq.heappop(heap)
        shares[r].append(k)
        heapq.heappush(heap, (load + int(cells[k]), r))
    return [sorted(s) for s in shares]


def align_share(pairs: Sequence[Tuple], rank: int, world_size: int,
                align: Callable) -> List[Tuple[int, object]]:
    """Align this rank's share; returns [(pair index, align(A, B))]."""
    cells = [a.shape[0] * b.shape[0] for a, b in pairs]
    mine = partition_pairs(cells, world_size)[rank]
    return [(k, align(*pairs[k])) for k in mine]


def gather_results(local: List[Tuple[int, object]], n_pairs: int, group=None) -> List[object]:
    """Collect every rank's (index, result) list; returns results in pair order.

    The only collective of the batch path, once, after all alignments.
    """
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts: List[List[Tuple[int, object]]] = [None] * world  # type: ignore[list-item]
    dist.all_gather_object(parts, local, group=group)
    out: List[object] = [None] * n_pairs
    seen = 0
    for part in parts:
        for k, res in part:
            if out[k] is not None:
                raise RuntimeError(f"pair {k} aligned twice")
            out[k] = res
            seen += 1
    if seen != n_pairs:
        raise RuntimeError(f"{n_pairs - seen} pairs were not aligned")
    return out
