"""Placement of independent instances on several GPUs (one process per GPU).

A batch of bounded-plasma instances has no exchange between instances, so N GPUs run
disjoint subsets with no collective on the data path; only the timing is combined
(maximum over ranks) and the particle-steps are summed.  A single large instance is
not split (that would need the domain decomposition with a per-step exchange); N GPUs
then run N independent replicas.
"""
from __future__ import annotations

import heapq
from typing import List, Sequence


def shard_instances(particle_counts: Sequence[int], world: int) -> List[List[int]]:
    """Partition instance indices over `world` ranks, balancing particle counts:
    largest instances first, each to the currently lightest rank (ties: lower rank).
    Deterministic; every instance lands on exactly one rank; each list is sorted."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(particle_counts)), key=lambda i: (-particle_counts[i], i))
    heap = [(0, r) for r in range(world)]
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + int(particle_counts[i]), r))
    return [sorted(x) for x in out]


def combine_timing(ms: float, particle_steps: float, device="cpu"):
    """Job-wide (max ms over ranks, summed particle-steps) with torch.distributed if it
    is initialised, else the local values."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, particle_steps
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    p = torch.tensor([particle_steps], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())
