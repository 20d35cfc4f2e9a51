"""Host-side sharding of apply work across ranks (one process per GPU).

Ensembles: the members of an ensemble of Hamiltonians (disorder
realisations, chains of several lengths) are not coupled, so its instances
are split across ranks with no collective on the data path: each rank
builds and applies only the members it owns.

One Hamiltonian: the output index range is cut into contiguous slices at
boundaries of the leading ("top") digits; rank g owns the target rows of
slice g (pull form, Sec. II: every row is written by its owner only). A
hop along a top site reads x from another slice (source = target +
offset, Sec. IV.B Eq. sourceoffset), so before each apply every rank
receives, point to point, the parts of the other slices that its rows'
sources reach (its halo) and then applies the operator to its own rows
with that extended x. Lanczos adds a sum over ranks of two scalars per step.

Only the halo exchange and scalar reductions cross ranks, through
torch.distributed with whatever backend the process group was created with.
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass, field
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


# ---------------------------------------------------------------------------
# One Hamiltonian over several ranks: slices of the output index range
# ---------------------------------------------------------------------------

# digit moves q (target digit = source digit + q) of each named local
# operator: the fixed-shift diagonals of Sec. IV.A, App. B and App. C
_MOVES = {"I": (0,), "Sz": (0,), "Sz2": (0,), "N": (0,), "Sp": (1,), "Sm": (-1,), "Sx": (1, -1),
          "Sy": (1, -1), "Sp2": (2,), "Sm2": (-2,), "a": (-1,), "adag": (1,)}
_OP_NAMES = {0: "I", 1: "Sz", 2: "Sx", 3: "Sy", 4: "Sp", 5: "Sm", 6: "Sz2", 7: "Sp2", 8: "Sm2", 9: "N",
             10: "a", 11: "adag"}


def source_offsets(sites, terms) -> list[int]:
    """Every source offset -(q_i M_i + q_j M_j) a term list can produce
    (Sec. IV.B Eq. sourceoffset), with 0 for the diagonal."""
    dims = [int(d) for _, d in sites]
    mult = [1] * len(dims)
    for k in range(len(dims) - 2, -1, -1):
        mult[k] = mult[k + 1] * dims[k + 1]
    offs = {0}
    for (i, oi, j, oj, _c) in terms:
        qi = _MOVES[_OP_NAMES.get(oi, oi)]
        qj = (0,) if j < 0 else _MOVES[_OP_NAMES.get(oj, oj)]
        for a in qi:
            for b in qj:
                offs.add(-(a * mult[i] + (b * mult[j] if j >= 0 else 0)))
    return sorted(offs)


@dataclass
class SlicePlan:
    """Rank `rank`'s share of one Hamiltonian over `world` ranks.

    bounds[g] .. bounds[g + 1]: the target rows of rank g (cut at multiples
    of `unit`, the number of states per combination of the top digits);
    [halo_lo, halo_hi): the x elements rank `rank` needs (its rows plus every
    source they reach); recv[r] / send[r]: global index ranges received from
    / sent to rank r before each apply."""
    D: int
    world: int
    rank: int
    unit: int
    bounds: list
    halo_lo: int
    halo_hi: int
    recv: dict = field(default_factory=dict)
    send: dict = field(default_factory=dict)

    @property
    def lo(self):
        return self.bounds[self.rank]

    @property
    def hi(self):
        return self.bounds[self.rank + 1]


def slice_plan(sites, terms, world: int, rank: int) -> SlicePlan:
    """Cut the index range into `world` slices at top-digit boundaries (the
    fewest leading sites whose digit combinations number at least `world`,
    shared out as evenly as whole combinations allow) and work out the
    halo exchange of every rank; every rank derives the same plan alone."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need world >= 1 and 0 <= rank < world")
    dims = [int(d) for _, d in sites]
    D = 1
    for d in dims:
        D *= d
    K, T = 0, 1
    while T < world and K < len(dims):
        T *= dims[K]
        K += 1
    if T < world:
        raise ValueError(f"{world} ranks need at least {world} states")
    unit = D // T
    bounds = [(g * T // world) * unit for g in range(world + 1)]
    offs = source_offsets(sites, terms)
    dmin, dmax = min(offs), max(offs)

    def halo(g):
        return max(0, bounds[g] + dmin), min(D, bounds[g + 1] + dmax)

    hl, hh = halo(rank)
    plan = SlicePlan(D, world, rank, unit, bounds, hl, hh)
    for r in range(world):
        if r == rank:
            continue
        a, b = max(hl, bounds[r]), min(hh, bounds[r + 1])
        if b > a:
            plan.recv[r] = (a, b)
        rl, rh = halo(r)
        a, b = max(rl, bounds[rank]), min(rh, bounds[rank + 1])
        if b > a:
            plan.send[r] = (a, b)
    return plan


def exchange_halo(plan: SlicePlan, x_local, nvec: int = 1):
    """x over [halo_lo, halo_hi) (state-major, nvec per state) from this
    rank's slice x_local (its rows [lo, hi)): the other ranks' parts arrive
    by point-to-point send/recv (the torch tensors' device decides the
    transport). Every rank must call it once per apply, in the same order."""
    import torch
    import torch.distributed as td
    ext = x_local.new_zeros((plan.halo_hi - plan.halo_lo) * nvec)
    ext[(plan.lo - plan.halo_lo) * nvec:(plan.hi - plan.halo_lo) * nvec] = x_local
    ops = []
    for r in sorted(plan.send):
        a, b = plan.send[r]
        ops.append(td.P2POp(td.isend, x_local[(a - plan.lo) * nvec:(b - plan.lo) * nvec].contiguous(), r))
    bufs = {}
    for r in sorted(plan.recv):
        a, b = plan.recv[r]
        bufs[r] = x_local.new_empty((b - a) * nvec)
        ops.append(td.P2POp(td.irecv, bufs[r], r))
    if ops:
        for req in td.batch_isend_irecv(ops):
            req.wait()
    for r, buf in bufs.items():
        a, b = plan.recv[r]
        ext[(a - plan.halo_lo) * nvec:(b - plan.halo_lo) * nvec] = buf
    return ext


def sharded_dot(a, b) -> float:
    """<a, b> over all ranks' slices: the local sum, then a sum over ranks."""
    import torch
    return sum_over_ranks(float(torch.dot(a.double().reshape(-1), b.double().reshape(-1))), device=a.device)


def sharded_lanczos(apply_local, plan: SlicePlan, v0_local, steps: int):
    """Lanczos on a vector sharded by `plan` (plain recurrence, no
    reorthogonalisation): apply_local(x_ext) returns this rank's rows of
    H x from the exchanged x; alpha and beta are sums over ranks of local dot
    products (two scalars per step). Returns (alpha, beta, E0)."""
    import numpy as np
    import torch
    v = v0_local / sharded_dot(v0_local, v0_local) ** 0.5
    v_prev = torch.zeros_like(v)
    alpha, beta = [], []
    b = 0.0
    for k in range(steps):
        w = apply_local(exchange_halo(plan, v))
        a = sharded_dot(v, w)
        w = w - a * v - b * v_prev
        b = sharded_dot(w, w) ** 0.5
        alpha.append(a)
        if k == steps - 1 or b < 1e-14:
            break
        beta.append(b)
        v_prev, v = v, w / b
    m = len(alpha)
    T = np.diag(alpha) + np.diag(beta[:m - 1], 1) + np.diag(beta[:m - 1], -1)
    return alpha, beta[:m - 1], float(np.linalg.eigvalsh(T)[0])
