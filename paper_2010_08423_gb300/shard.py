"""Sharding one query's sieve points across ranks (one process per GPU).

The per-vertex sums are XOR-linear in the sieve points (Eq. 2: a sum over
L of per-point evaluations), so rank r of W can evaluate a contiguous range
of points and the ranks' partial witnesses combine by XOR. NCCL has no XOR
reduction, so the exchange is an all-gather of the n x 8-byte partials
followed by a local XOR.
"""
from __future__ import annotations

import numpy as np


def point_range(k: int, rank: int, world: int, align: int = 128) -> tuple:
    """Contiguous [first, first + count) share of the 2^k points for `rank`;
    shares are multiples of `align` points where 2^k allows it."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    total = 1 << k
    unit = align if total >= align * world else 1
    units = total // unit
    base, extra = divmod(units, world)
    first = (rank * base + min(rank, extra)) * unit
    count = (base + (1 if rank < extra else 0)) * unit
    return first, count


def xor_combine(parts) -> np.ndarray:
    """XOR of equally shaped uint64 arrays."""
    out = None
    for p in parts:
        p = np.asarray(p, dtype=np.uint64)
        out = p.copy() if out is None else out ^ p
    return out


def allgather_xor(partial, group=None):
    """All-gather the ranks' int64/uint64 partial witnesses (torch tensors,
    same shape) and XOR them locally; returns the combined tensor."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    t = partial.contiguous().view(torch.int64)
    bufs = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(bufs, t, group=group)
    out = bufs[0].clone()
    for b in bufs[1:]:
        out ^= b
    return out
