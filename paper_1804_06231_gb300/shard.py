"""Host-side sharding of independent boxes over ranks (one process per GPU).

Boxes are independent periodic problems, so a multi-GPU run needs no data
exchange: every rank computes the same deterministic assignment from the same
cost list and processes its own boxes; only the step's totals are reduced
(sum of interactions, max of the step times).  The cost of a box is
proportional to its pair work; for the workloads here (constant expected
neighbour count per particle) that is its particle count times the
candidates per interaction, which grows with the cell edge over H.
"""
from __future__ import annotations

import heapq


def box_cost(n: int, nc: int, L: float = 1.0, h_max: float | None = None) -> float:
    """Relative cost of one box: particles x (edge / H_max)^3 when H_max is
    known (the sorted windows cover about edge^2 H of each cell pair, the pairs
    in range about H^3), else particles."""
    if h_max is None or h_max <= 0:
        return float(n)
    edge = L / nc
    return float(n) * max(1.0, edge / h_max) ** 3


def assign_boxes(costs, world_size: int) -> list[list[int]]:
    """Longest-processing-time-first assignment of boxes to ranks.

    Boxes are taken in decreasing cost (ties: lower index first) and each goes
    to the least-loaded rank (ties: lower rank).  Deterministic, so every rank
    derives the same plan without communication.  The largest load is at most
    4/3 of the optimum (Graham's bound for this rule).  Returns, per rank, the
    box indices in increasing order."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    costs = [float(c) for c in costs]
    if any(c < 0 for c in costs):
        raise ValueError("costs must be non-negative")
    order = sorted(range(len(costs)), key=lambda b: (-costs[b], b))
    heap = [(0.0, r) for r in range(world_size)]
    plan = [[] for _ in range(world_size)]
    for b in order:
        load, r = heapq.heappop(heap)
        plan[r].append(b)
        heapq.heappush(heap, (load + costs[b], r))
    return [sorted(p) for p in plan]


def rank_loads(costs, plan) -> list[float]:
    return [sum(float(costs[b]) for b in p) for p in plan]


def local_boxes(costs, rank: int, world_size: int) -> list[int]:
    """The boxes `rank` processes."""
    if not 0 <= rank < world_size:
        raise ValueError("rank out of range")
    return assign_boxes(costs, world_size)[rank]


def step_totals(units: float, ms: float, device=None) -> tuple[float, float]:
    """(sum of `units`, max of `ms`) over the ranks of the default process
    group; the identity without one.  `device` is where the reduction tensors
    live (a CUDA device for NCCL, None = CPU for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(units), float(ms)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())
