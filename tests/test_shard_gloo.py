"""Multi-rank sharding of sieve points (host logic), world size 2 over gloo on
the CPU: each rank evaluates its share of the points with the oracle and the
all-gather + XOR combine must give the full sums."""
import os
import socket

import numpy as np
import pytest

from paper_2010_08423_gb300 import shard
from paper_2010_08423_gb300 import workloads as W


def test_point_ranges_partition_the_points():
    for k in (2, 3, 4, 5, 7, 8, 9, 12, 20):
        for world in (1, 2, 3, 4, 8):
            seen = []
            for r in range(world):
                f, c = shard.point_range(k, r, world)
                # the library's range entry takes starts on multiples of 128
                # (k <= 3: the whole range or nothing)
                assert c == 0 or (f % shard.RANGE_ALIGN == 0 if k > 3 else (f, c) == (0, 1 << k))
                seen.extend(range(f, f + c))
            assert seen == list(range(1 << k)), (k, world)
    f, c = shard.point_range(10, 1, 2)
    assert f % 128 == 0 and c % 128 == 0
    # fewer 128-point units than ranks: the last ranks get empty shares
    assert [shard.point_range(8, r, 4) for r in range(4)] == [(0, 128), (128, 128), (256, 0), (256, 0)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = W.uniform(300, 3000, 12, 0, 4, 61)
        k = 6
        first, count = shard.point_range(k, rank, world, align=16)
        part = oracle.sieve(g, 3, k, 17, masks=np.arange(first, first + count, dtype=np.uint32),
                            threads=1)
        full = shard.allgather_xor(torch.from_numpy(part.view(np.int64).copy()))
        q.put((rank, full.numpy().view(np.uint64).copy()))
    finally:
        dist.destroy_process_group()


def test_allgather_xor_two_ranks_gloo():
    import multiprocessing as mp
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = W.uniform(300, 3000, 12, 0, 4, 61)
    ref = oracle.sieve(g, 3, 6, 17)
    assert np.count_nonzero(ref) > 0
    assert np.array_equal(res[0], ref) and np.array_equal(res[1], ref)
