"""Host-side logic for running the Lagrangian step on several GPUs (one process per GPU).

Particles are independent given the fluid field, so the work shards by particle index: rank r of
W takes a contiguous range of generation indices.  The only exchange is the per-cell source field
once per coupling interval; it is summed over ranks in rank order, so every rank gets the same
bits whatever the arrival order.  Timings are reduced with the maximum over ranks.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """(first, count) of rank's contiguous share of n particles; shares differ by at most one."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def reduce_sources_rank_order(src: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of every rank's per-cell sources [3, ncell] (float64), added in rank order 0, 1, ..."""
    world = dist.get_world_size(group)
    parts = [torch.empty_like(src) for _ in range(world)]
    dist.all_gather(parts, src.contiguous(), group=group)
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return out


def max_over_ranks(x: float, device=None, group=None) -> float:
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
