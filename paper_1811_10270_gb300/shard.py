"""Host-side logic for running the operator on several ranks (one process per GPU).

The operator shards by target ownership: each rank owns whole drops and evaluates the layer
operators at their targets, which needs every drop's density (an all-gather of coefficient
vectors per application) and, for GMRES, all-reduced dot products. This module holds the
partition and the cross-rank reductions; it performs none of the method's arithmetic.
"""
from __future__ import annotations


def partition_drops(costs, world: int):
    """Greedy balanced partition of drops (cost = targets x sources of a drop's work) over
    `world` ranks: returns a list of drop-index lists, each sorted ascending."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(p) for p in parts]


def drop_cost(p: int) -> int:
    """Work of one drop's targets against one unit of sources: (p+1)(2p+2) targets x
    (2p+2)(4p+4) nodes of its own degree-(2p+1) grid (self rows) -- the balance weight."""
    return (p + 1) * (2 * p + 2) * (2 * p + 2) * (4 * p + 4)


def reduce_timing(ms: float, units: float, dist=None):
    """Max of the per-rank times and sum of the per-rank work units over the job (the
    throughput contract: whole-job units / slowest rank's time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms, units
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(u)
    return float(t.item()), float(u.item())
