"""Point ranges of one query (rr_reach_range_device) and the sharded query
built on them: the witness part of a range equals the oracle's sum over the
same sieve points bit for bit, ranges that partition the points XOR to the
full witness (both engines, plain and motif, layer 3 per point and in
pair-label space), bad ranges are refused, and two processes sharing the GPU,
each evaluating its share through the library and exchanging parts over gloo,
reproduce the oracle's full witness (Eq. 2: the sum over L is independent per
point)."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2010_08423_gb300 import capi, shard
from paper_2010_08423_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    capi.load()
    oracle.build()


def _graph(ncolors=0, seed=0x5EED0000 + 301):
    # t ~ U[1,40] on n=3000, m=40000: windows hold several rows, so walks of
    # 12 vertices survive and every layer kind has rows
    return W.uniform(3000, 40_000, 40, 1, 6, seed, ncolors=ncolors)


@pytest.mark.parametrize("flags", [0, capi.FLAG_DENSE_STATE, capi.FLAG_PAIR_ON,
                                   capi.FLAG_PAIR_ON | capi.FLAG_HEAD_TABLE_ON])
def test_ranges_xor_to_full_witness_and_match_oracle(flags):
    g = _graph(ncolors=3)
    motif = [int(g["color"][5]), 0, 1, 2, 1, 0, 2, 1, 0]
    with capi.Graph(g, flags) as G:
        for k, mo in ((4, None), (6, None), (9, None), (9, motif), (12, None)):
            full = G.reach(5, k, 77, motif=mo)[1]
            for world in (1, 2, 3, 8):
                parts = [G.reach_range(5, k, 77, *shard.point_range(k, r, world), motif=mo)
                         for r in range(world)]
                assert np.array_equal(shard.xor_combine(parts), full), (k, world, flags)
            # one range against the oracle's sum over the same points
            first, count = (128, 128) if k >= 8 else (0, 1 << k)
            part = G.reach_range(5, k, 77, first, count, motif=mo)
            ref = oracle.sieve(g, 5, k, 77, motif=mo,
                               masks=np.arange(first, first + count, dtype=np.uint32))
            assert np.array_equal(part, ref), (k, flags)
        assert np.count_nonzero(full) > 0
        # ranges shorter than a chunk and not ending on a lane group
        ref = oracle.sieve(g, 5, 10, 3, masks=np.arange(256, 256 + 37, dtype=np.uint32))
        assert np.array_equal(G.reach_range(5, 10, 3, 256, 37), ref)
        # empty range
        assert not G.reach_range(5, 10, 3, 1024, 0).any()


def test_small_k_and_bad_ranges():
    g = _graph()
    with capi.Graph(g) as G:
        for k in (2, 3):
            full = G.reach(5, k, 9)[1]
            assert np.array_equal(G.reach_range(5, k, 9, 0, 1 << k), full)
            assert not G.reach_range(5, k, 9, 0, 0).any()
        for k, first, count in ((3, 0, 4), (8, 64, 64), (8, 128, 256), (10, 1024, 1)):
            with pytest.raises(capi.RRError) as ei:
                G.reach_range(5, k, 9, first, count)
            assert ei.value.status == capi.RR_EINVAL, (k, first, count)
        # the graph still answers after the refusals
        assert np.array_equal(G.reach(5, 5, 9)[1], oracle.sieve(g, 5, 5, 9))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, k, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        g = _graph(ncolors=3)
        with capi.Graph(g) as G:
            d_part = torch.empty(g["n"], dtype=torch.int64, device="cuda")
            st = torch.cuda.Stream()
            full = shard.reach_sharded(G.handle, g["n"], 5, k, 123, d_part, stream=st)
            q.put((rank, full.cpu().numpy().view(np.uint64).copy(),
                   d_part.cpu().numpy().view(np.uint64).copy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("k", [7, 11])
def test_sharded_query_two_processes_gloo(k):
    """Two ranks (processes) on one GPU: each runs its share of the points in
    its own CUDA context (kernels of the two never wait on each other), then
    the parts are all-gathered over gloo and XOR-combined."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, k, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r, full, part = q.get(timeout=300)
        res[r] = (full, part)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = _graph(ncolors=3)
    ref = oracle.sieve(g, 5, k, 123)
    assert np.count_nonzero(ref) > 0
    assert np.array_equal(res[0][0], ref) and np.array_equal(res[1][0], ref)
    # each rank's own part is the oracle's sum over its share
    for r in range(2):
        f, c = shard.point_range(k, r, 2)
        want = oracle.sieve(g, 5, k, 123, masks=np.arange(f, f + c, dtype=np.uint32))
        assert np.array_equal(res[r][1], want)
