"""Host-side sharding of independent apply work across ranks (one process per
GPU). An ensemble of Hamiltonians (disorder realisations, chains of several
lengths) has no coupling between its members, so its instances are split
across ranks with no collective on the data path: each rank builds and
applies only the members it owns. A single Hamiltonian is run as replicas.

Only scalar bookkeeping (timings) crosses ranks, through torch.distributed
with whatever backend the process group was created with.
"""
from __future__ import annotations

import heapq
from typing import Sequence


def partition(costs: Sequence[float], world_size: int) -> list[list[int]]:
    """Split instance indices over world_size ranks, balancing the summed cost
    (states x right-hand sides): longest-processing-time-first greedy, ties
    broken by index, so every rank computes the same answer without
    communicating. Each rank's list is in ascending index order."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    for c in costs:
        if not c >= 0:
            raise ValueError("instance costs must be non-negative")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world_size)]
    heapq.heapify(heap)
    parts: list[list[int]] = [[] for _ in range(world_size)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(p) for p in parts]


def owned(costs: Sequence[float], rank: int, world_size: int) -> list[int]:
    """Instance indices that rank owns under partition()."""
    if not 0 <= rank < world_size:
        raise ValueError("rank out of range")
    return partition(costs, world_size)[rank]


def imbalance(costs: Sequence[float], parts: Sequence[Sequence[int]]) -> float:
    """max rank load / mean rank load (1.0 = perfect balance)."""
    loads = [sum(costs[i] for i in p) for p in parts]
    mean = sum(loads) / max(1, len(loads))
    return max(loads) / mean if mean > 0 else 1.0


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar (e.g. a timed region's length) over the
    process group; the value itself when torch.distributed is not initialised."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of a per-rank scalar (e.g. states processed) over the process group."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.SUM)
    return float(t.item())
