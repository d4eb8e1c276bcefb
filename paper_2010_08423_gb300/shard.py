"""Sharding one query's sieve points across ranks (one process per GPU).

The per-vertex sums are XOR-linear in the sieve points (Eq. 2: a sum over
L of per-point evaluations), so rank r of W evaluates a contiguous range of
points with ``rr_reach_range_device`` on its own copy of the graph, and the
ranks' partial witnesses combine by XOR. NCCL has no XOR reduction, so the
exchange is an all-gather of the n x 8-byte partials followed by a local XOR.
"""
from __future__ import annotations

import numpy as np

# rr_reach_range_device takes ranges that start on multiples of this
RANGE_ALIGN = 128


def point_range(k: int, rank: int, world: int, align: int = RANGE_ALIGN) -> tuple:
    """Contiguous [first, first + count) share of the 2^k points for `rank`.
    Shares start on multiples of `align`; when 2^k holds fewer than `world`
    such units the last ranks get empty shares, and for k <= 3 (summed in
    closed form) rank 0 takes every point."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    total = 1 << k
    if k <= 3:
        return (0, total) if rank == 0 else (total, 0)
    units = (total + align - 1) // align
    base, extra = divmod(units, world)
    first = min(total, (rank * base + min(rank, extra)) * align)
    end = min(total, first + (base + (1 if rank < extra else 0)) * align)
    return first, end - first


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
    dev = t.device
    if t.is_cuda and dist.get_backend(group) == "gloo":
        t = t.cpu()  # gloo gathers host tensors
    bufs = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(bufs, t, group=group)
    out = bufs[0].clone()
    for b in bufs[1:]:
        out ^= b
    return out.to(dev)


def reach_sharded(graph_handle, n: int, source: int, k: int, seed: int, d_partial,
                  motif=None, stream=None, group=None):
    """One query split over the ranks of `group`: this rank computes the
    witness part of its point range into d_partial (n int64, device) with the
    library, then the parts are all-gathered and XOR-combined. Returns the full
    witness (n int64, on d_partial's device) on every rank."""
    import torch.distributed as dist
    from . import capi
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    first, count = point_range(k, rank, world)
    capi.rr_reach_range_device(graph_handle, source, k, seed, first, count, d_partial,
                               None if stream is None else stream.cuda_stream, motif)
    if stream is not None:
        stream.synchronize()
    return allgather_xor(d_partial, group)
