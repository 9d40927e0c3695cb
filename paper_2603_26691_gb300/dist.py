"""Host-side logic for running the Lagrangian step on several GPUs (one process per GPU).

Particles are independent given the fluid field, so the work shards by particle index: rank r of
W takes a contiguous range of generation indices.  The only exchange is the per-cell source field
once per coupling interval.  Each rank keeps its sources as exact fixed-point integers (value =
integer x 2^-E, E chosen per rank from its own bounds), so the sum over ranks is taken on those
integers: every rank's integers are shifted to the finest scale (the largest E) and added with an
integer all-reduce, which is exact and independent of the order of the ranks; the total is rounded
to FP64 once.  Timings are reduced with the maximum over ranks.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

_MASK = 0xFFFFFFFF


def shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """(first, count) of rank's contiguous share of n particles; shares differ by at most one."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def _limbs(words: torch.Tensor, shift: int, nlimbs: int) -> torch.Tensor:
    """Normalised fixed-point words [..., 4] (digits in [0, 2^32) below a signed top word) times
    2^shift, as nlimbs int64 limbs of weight 2^(32 j) (each limb below 2^33 in magnitude)."""
    q, r = divmod(shift, 32)
    out = torch.zeros(words.shape[:-1] + (nlimbs,), dtype=torch.int64, device=words.device)
    for j in range(words.shape[-1]):
        v = words[..., j] << r  # exact: digits < 2^32 and a top word < 2^31 in magnitude, r < 32
        out[..., q + j] += v & _MASK
        out[..., q + j + 1] += v >> 32
    return out


def _to_f64(limbs: torch.Tensor, E: int) -> torch.Tensor:
    """The value sum_j limbs[..., j] 2^(32 j - E) rounded to FP64: carries propagated first, then the
    limbs added from the most significant down (each term exact)."""
    limbs = limbs.clone()
    K = limbs.shape[-1]
    for j in range(K - 1):
        carry = limbs[..., j] >> 32
        limbs[..., j] &= _MASK
        limbs[..., j + 1] += carry
    out = torch.zeros(limbs.shape[:-1], dtype=torch.float64, device=limbs.device)
    for j in range(K - 1, -1, -1):
        out += limbs[..., j].to(torch.float64) * (2.0 ** (32 * j - E))
    return out


def reduce_sources_exact(words: torch.Tensor, E: int, group=None) -> torch.Tensor:
    """Sum over ranks of fixed-point sources (each rank's (words, E) from Sim.sources_fixed), exact in
    integers and the same bits on every rank whatever the order; returns FP64 [3, ncell]."""
    e = torch.tensor([int(E)], dtype=torch.int64, device=words.device)
    world = dist.get_world_size(group)
    es = [torch.empty_like(e) for _ in range(world)]
    dist.all_gather(es, e, group=group)
    es = [int(x.item()) for x in es]
    e_max, e_min = max(es), min(es)
    nlimbs = 6 + (e_max - e_min + 31) // 32
    limbs = _limbs(words.to(torch.int64), e_max - int(E), nlimbs)
    dist.all_reduce(limbs, op=dist.ReduceOp.SUM, group=group)
    return _to_f64(limbs, e_max)


def reduce_sources_rank_order(src: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of every rank's FP64 per-cell fields [3, ncell], added in rank order 0, 1, ... (the same bits
    on every rank, rounded per addition; the sources themselves go through reduce_sources_exact)."""
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
