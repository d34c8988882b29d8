"""Sharding of independent SG systems over ranks (one process per GPU).

The systems of a batch share nothing, so a multi-GPU run splits the list of
systems and each rank solves its part with one batched launch; there is no
collective on the data path. The split is longest-processing-time greedy on a
per-system cost, deterministic, so every rank computes the same assignment
without communicating. Only timing uses a collective (the max over ranks).
"""
from __future__ import annotations

import math
from typing import List, Sequence


def system_cost(ne: int, M: int, p: int) -> float:
    """Relative work of one solve: the SG product dominates, and it costs
    (P + couplings) multiply-adds per nonzero; nonzeros ~ 9 (ne-1)^2."""
    n = (ne - 1) ** 2
    P = math.comb(M + p, p)
    couplings = 2 * M * math.comb(M + p - 1, M) if p > 0 else 0
    return 9.0 * n * (P + couplings)


def assign(costs: Sequence[float], world: int) -> List[List[int]]:
    """Indices of the systems each rank solves: largest first, each to the
    least-loaded rank (ties: lowest rank); each rank's list in index order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world), key=lambda r: (load[r], r))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def my_systems(costs: Sequence[float], rank: int, world: int) -> List[int]:
    return assign(costs, world)[rank]


def max_over_ranks(value: float, device=None) -> float:
    """Max of a float over all ranks of the default process group (identity
    without one); a device tensor for NCCL, a host tensor for gloo."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
