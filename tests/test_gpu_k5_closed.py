"""k = 5 in closed form: layer 3 in pair-label space, then per deep-tail row
y_{e,4} times the sum over the splits of the five labels into one for z_w, a
pair for z_v and z_s (their 2x2 permanent) and a pair for the window's pair
sums (only the bijections of labels survive the sum over all 32 points).
Load flag bit 9 turns it on (per point is the default). Against the oracle
and the per-point form, bit for bit:
witness and per-edge sums, plain and motif queries, a hub whose in-rows are
cut into segments, a part of the points (per point), and at-most-k's branch
k' = 5 taken from the k query's own pair rows (the pair-label layer 3 on) or
from its per-point layer 3."""
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


def _graphs():
    from test_gpu_parity import _hub_graph
    return [("uniform", W.uniform(2000, 30_011, 40, 0, 6, 11, ncolors=3), (0, 5, 17)),
            ("dense windows", W.uniform(1500, 20_000, 30, 0, 5, 12, ncolors=3), (3, 8)),
            ("hub", _hub_graph(), (0, 9, 40))]


@pytest.mark.parametrize("idx", [0, 1, 2])
def test_witness_and_edges_match_oracle_and_per_point(idx):
    name, g, sources = _graphs()[idx]
    nonzero = 0
    with capi.Graph(g, capi.FLAG_K5_CLOSED) as G, capi.Graph(g) as H:
        for s in sources:
            for seed in (3, 77):
                ref = oracle.sieve(g, s, 5, seed)
                _, w = G.reach(s, 5, seed)
                _, w_pp = H.reach(s, 5, seed)
                assert np.array_equal(w, ref), (name, s, seed)
                assert np.array_equal(w_pp, ref), (name, s, seed)
                nonzero += int(np.count_nonzero(ref) > 0)
            S, E, R, _ = G.arrival(s, 5, 5)
            S_pp, E_pp, R_pp, _ = H.arrival(s, 5, 5)
            S_ref, E_ref = oracle.sieve(g, s, 5, 5, edges=True)
            assert np.array_equal(S, S_ref) and np.array_equal(E, E_ref), (name, s)
            assert np.array_equal(E_pp, E_ref) and np.array_equal(R, R_pp), (name, s)
            assert np.array_equal(R, oracle.arrival_times(g, E_ref)), (name, s)
    assert nonzero >= len(sources)


def test_motif_queries_and_ranges():
    name, g, _ = _graphs()[0]
    with capi.Graph(g, capi.FLAG_K5_CLOSED) as G:
        for s, seed in ((5, 2), (17, 9)):
            motif = [int(g["color"][s]), 0, 1, 2, 1]
            ref = oracle.sieve(g, s, 5, seed, motif=motif)
            _, w = G.reach(s, 5, seed, motif=motif)
            assert np.array_equal(w, ref), s
            S, E, _, _ = G.arrival(s, 5, seed, motif=motif)
            S_ref, E_ref = oracle.sieve(g, s, 5, seed, motif=motif, edges=True)
            assert np.array_equal(S, S_ref) and np.array_equal(E, E_ref), s
        # all 32 points in closed form, a part per point
        ref = oracle.sieve(g, 5, 5, 8)
        assert np.array_equal(G.reach_range(5, 5, 8, 0, 32), ref)
        for c in (7, 20):
            assert np.array_equal(G.reach_range(5, 5, 8, 0, c), oracle.sieve(g, 5, 5, 8, masks=range(c))), c


@pytest.mark.parametrize("pair_flag", [0, capi.FLAG_PAIR_ON])
def test_atmost_branch_five(pair_flag):
    """k = 7 and 10 with the branches forced: branch k' = 5 from the k query's
    pair rows (pair_count(k) values a row, labels 0..4 their first 15) when
    the pair-label layer 3 is on, else from its per-point layer 3; bounded
    reachability reads the branch's per-edge sums."""
    import torch
    name, g, _ = _graphs()[1]
    n = g["n"]
    with capi.Graph(g, pair_flag | capi.FLAG_ATMOST_BRANCHES) as G:
        for k in (7, 10):
            d_w = torch.full((k - 1, n), -1, dtype=torch.int64, device="cuda")
            d_bm = torch.zeros((n + 7) // 8, dtype=torch.uint8, device="cuda")
            capi.rr_reach_atmost_device(G.handle, 3, k, 21, d_w, d_bm)
            torch.cuda.synchronize()
            w = d_w.cpu().numpy().view(np.uint64)
            ref5 = oracle.sieve(g, 3, 5, 21)
            assert np.array_equal(w[3], ref5), (pair_flag, k)
            assert np.count_nonzero(ref5) > 0
            for kk in range(2, k + 1):
                assert np.array_equal(w[kk - 2], G.reach(3, kk, 21)[1]), (pair_flag, k, kk)
        R_ref, L_ref = oracle.atmost_arrival(g, 3, 7, 13)
        d_r = torch.zeros(n, dtype=torch.int32, device="cuda")
        d_l = torch.full((n,), 99, dtype=torch.uint8, device="cuda")
        capi.rr_reach_bounded_device(G.handle, 3, 7, 13, d_r, d_l)
        torch.cuda.synchronize()
        assert np.array_equal(d_r.cpu().numpy().view(np.uint32), R_ref)
        assert np.array_equal(d_l.cpu().numpy(), L_ref)
