"""at-most-k with the smaller queries taken from the k query's own layers: for
one seed the k'-vertex query's per-point layers agree with the k-vertex
query's on the first 2^k' points, so rows k' >= 5 come from the k query (k' =
5 from its pair rows in closed form when layer 3 runs in pair-label space). Every row must equal the single query's
witness and the lanes-only form's (load flag bit 6; bit 7 forces the branches
on these small graphs), bit for bit: k = 6..12,
one and several point chunks, layer 3 per point or in pair-label space, cut
hub segments, branch k-1 from the pair tail's sums; a few rows against the
oracle."""
import numpy as np
import pytest

import oracle
from paper_2010_08423_gb300 import capi
from paper_2010_08423_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    capi.load()
    oracle.build()
    torch.cuda.set_device(0)


def _atmost(G, n, s, k, seed):
    import torch
    d_w = torch.full((k - 1, n), -1, dtype=torch.int64, device="cuda")
    d_bm = torch.zeros((n + 7) // 8, dtype=torch.uint8, device="cuda")
    capi.rr_reach_atmost_device(G.handle, s, k, seed, d_w, d_bm)
    torch.cuda.synchronize()
    bm = np.unpackbits(d_bm.cpu().numpy(), bitorder="little")[:n].astype(bool)
    return d_w.cpu().numpy().view(np.uint64), bm


@pytest.mark.parametrize("pair_flag", [0, capi.FLAG_PAIR_OFF, capi.FLAG_PAIR_ON])
def test_rows_equal_single_queries_and_lanes(pair_flag):
    g = W.uniform(2000, 25_000, 25, 0, 5, 81)
    n = g["n"]
    with capi.Graph(g, pair_flag | capi.FLAG_ATMOST_BRANCHES) as G, \
            capi.Graph(g, pair_flag | capi.FLAG_ATMOST_LANES) as H:
        for s, k, seed in ((3, 6, 11), (7, 8, 12), (1, 10, 13), (4, 12, 14)):
            w, bm = _atmost(G, n, s, k, seed)
            w_l, bm_l = _atmost(H, n, s, k, seed)
            union = np.zeros(n, dtype=bool)
            for kk in range(2, k + 1):
                _, ref = G.reach(s, kk, seed)
                assert np.array_equal(w[kk - 2], ref), (pair_flag, k, kk)
                assert np.array_equal(w_l[kk - 2], ref), (pair_flag, k, kk)
                union |= ref != 0
            assert np.array_equal(bm, union) and np.array_equal(bm_l, union), k
            assert union.sum() > 10


def test_several_chunks_and_hubs_against_oracle():
    """k = 11 with 256-point chunks: the k query's chunks 0..3 each feed the
    branches whose points they hold; a hub whose head segments are cut."""
    from test_gpu_parity import _hub_graph
    g = _hub_graph()
    n = g["n"]
    with capi.Graph(g, capi.FLAG_ATMOST_BRANCHES) as G:
        capi.rr_set_tuning(G.handle, 11, 4, 256)
        w, _ = _atmost(G, n, 9, 11, 77)
        for kk in (5, 6, 8, 9, 10, 11):
            assert np.array_equal(w[kk - 2], oracle.sieve(g, 9, kk, 77)), kk
        assert sum(int(np.count_nonzero(w[kk - 2]) > 0) for kk in range(5, 12)) >= 4
        for kk in range(2, 12):
            assert np.array_equal(w[kk - 2], G.reach(9, kk, 77)[1]), kk


@pytest.mark.parametrize("k", [8, 11])
def test_bounded_reach_with_branches(k):
    """Bounded RestlessReach (minimum arrival over k' <= k and the shortest
    length) with the branches' per-edge sums and arrivals, against the lanes
    form and the oracle."""
    import torch
    g = W.uniform(1500, 20_000, 30, 0, 5, 60 + k)
    n = g["n"]
    R_ref, L_ref = oracle.atmost_arrival(g, 4, k, 13)
    for flags in (capi.FLAG_ATMOST_BRANCHES, capi.FLAG_ATMOST_LANES):
        with capi.Graph(g, flags) as G:
            d_r = torch.zeros(n, dtype=torch.int32, device="cuda")
            d_l = torch.full((n,), 99, dtype=torch.uint8, device="cuda")
            d_b = torch.zeros((n + 7) // 8, dtype=torch.uint8, device="cuda")
            for rep in range(2):  # the lanes' and branches' buffers reused
                capi.rr_reach_bounded_device(G.handle, 4, k, 13, d_r, d_l, d_b)
                torch.cuda.synchronize()
                assert np.array_equal(d_r.cpu().numpy().view(np.uint32), R_ref), flags
                assert np.array_equal(d_l.cpu().numpy(), L_ref), flags
                D = np.unpackbits(d_b.cpu().numpy(), bitorder="little")[:n].astype(bool)
                assert np.array_equal(D, R_ref != oracle.NO_ARRIVAL)
    assert (L_ref >= 5).sum() > 3


@pytest.mark.parametrize("k,ppl,chunk", [(7, 2, 256), (7, 4, 256), (8, 4, 256), (9, 2, 512),
                                         (10, 4, 512), (11, 4, 1024), (12, 2, 256)])
def test_branch_from_pair_sums(k, ppl, chunk):
    """With the pair tail the k query's layer k-3 stores pair sums, and branch
    k-1 is the (k-1)-vertex query's last layer over their single-label slots:
    it must equal the pair tail off and the single queries, on a hub whose
    cut segments the sums' fix-up completes, with 64- and 128-point groups and
    one or several chunks below 2^(k-1). With 128-point groups and k = 7 a
    group straddles 2^6, so there the pair tail stays off. Once with each
    launch enqueued (kernel timing on, which counts the label-space layer) and
    once from the captured graph."""
    from test_gpu_parity import _hub_graph
    g = _hub_graph()
    n = g["n"]
    seed = 31 + k
    with capi.Graph(g, capi.FLAG_ATMOST_BRANCHES) as G, \
            capi.Graph(g, capi.FLAG_ATMOST_BRANCHES | capi.FLAG_PAIR_TAIL_OFF) as H:
        for X in (G, H):
            capi.rr_set_tuning(X.handle, k, ppl, chunk)
        capi.rr_timing_enable(True)
        try:
            capi.rr_timing_read(reset=True)
            w_t, bm_t = _atmost(G, n, 9, k, seed)
            tail_launches = capi.rr_timing_read(reset=True)["label_tail_layer"][1]
            w_off, bm_off = _atmost(H, n, 9, k, seed)
            assert capi.rr_timing_read(reset=True)["label_tail_layer"][1] == 0
        finally:
            capi.rr_timing_enable(False)
        straddles = (1 << (k - 1)) % (32 * ppl) != 0
        assert (tail_launches == 0) == straddles, tail_launches
        w, bm = _atmost(G, n, 9, k, seed)
        assert np.array_equal(w, w_t) and np.array_equal(bm, bm_t)
        assert np.array_equal(w, w_off) and np.array_equal(bm, bm_off)
        for kk in range(2, k + 1):
            assert np.array_equal(w[kk - 2], G.reach(9, kk, seed)[1]), kk
        assert np.array_equal(w[k - 3], oracle.sieve(g, 9, k - 1, seed))
        assert np.count_nonzero(w[k - 3]) > 0
