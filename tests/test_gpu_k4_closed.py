"""k = 4 in closed form: layer 2 in label space, then per tail row y_{e,3}
times the 4 x 4 permanent of z_s, z_v, z_w and the window's label-space sums
(only the bijections of labels survive the sum over all 16 points). Against
the oracle and the per-point form (load flag bit 8), bit for bit: witness and
per-edge sums, plain and motif queries, a hub whose in-rows are cut into
segments (the label-space prefix's carry fix-up) and whose rows fill whole
warps with one head, many heads per warp, the at-most-k lanes, a part of the
points (per point) and path extraction."""
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
    with capi.Graph(g) as G, capi.Graph(g, capi.FLAG_K4_PER_POINT) as H:
        for s in sources:
            for seed in (3, 77):
                ref = oracle.sieve(g, s, 4, seed)
                _, w = G.reach(s, 4, seed)
                _, w_pp = H.reach(s, 4, seed)
                assert np.array_equal(w, ref), (name, s, seed)
                assert np.array_equal(w_pp, ref), (name, s, seed)
                nonzero += int(np.count_nonzero(ref) > 0)
            S, E, R, _ = G.arrival(s, 4, 5)
            S_pp, E_pp, R_pp, _ = H.arrival(s, 4, 5)
            S_ref, E_ref = oracle.sieve(g, s, 4, 5, edges=True)
            assert np.array_equal(S, S_ref) and np.array_equal(E, E_ref), (name, s)
            assert np.array_equal(E_pp, E_ref) and np.array_equal(R, R_pp), (name, s)
            assert np.array_equal(R, oracle.arrival_times(g, E_ref)), (name, s)
    assert nonzero >= len(sources)


def test_motif_queries():
    name, g, _ = _graphs()[0]
    with capi.Graph(g) as G:
        for s, seed in ((5, 2), (17, 9)):
            motif = [int(g["color"][s]), 0, 1, 2]
            ref = oracle.sieve(g, s, 4, seed, motif=motif)
            _, w = G.reach(s, 4, seed, motif=motif)
            assert np.array_equal(w, ref), s
            S, E, _, _ = G.arrival(s, 4, seed, motif=motif)
            S_ref, E_ref = oracle.sieve(g, s, 4, seed, motif=motif, edges=True)
            assert np.array_equal(S, S_ref) and np.array_equal(E, E_ref), s


def test_atmost_range_and_extraction():
    import torch
    name, g, _ = _graphs()[1]
    n = g["n"]
    with capi.Graph(g) as G, capi.Graph(g, capi.FLAG_K4_PER_POINT) as H:
        # at-most-k: the k' = 4 lane takes the closed form
        for k in (4, 7):
            d_w = torch.full((k - 1, n), -1, dtype=torch.int64, device="cuda")
            d_bm = torch.zeros((n + 7) // 8, dtype=torch.uint8, device="cuda")
            capi.rr_reach_atmost_device(G.handle, 3, k, 21, d_w, d_bm)
            torch.cuda.synchronize()
            w = d_w.cpu().numpy().view(np.uint64)
            assert np.array_equal(w[2], oracle.sieve(g, 3, 4, 21)), k
        # a part of the 16 points runs per point, all of them in closed form
        ref = oracle.sieve(g, 3, 4, 8)
        assert np.array_equal(G.reach_range(3, 4, 8, 0, 16), ref)
        for c in (5, 11):
            assert np.array_equal(G.reach_range(3, 4, 8, 0, c), oracle.sieve(g, 3, 4, 8, masks=range(c))), c
        # extraction deletes vertices (their z rows zero) and re-runs the query
        reach = ref != 0
        targets = np.flatnonzero(reach)[:3]
        assert len(targets) > 0
        for t in targets:
            p = G.extract_path(3, 4, 8, int(t))
            assert p == H.extract_path(3, 4, 8, int(t)), t


def test_persistent_batch():
    """The batch's k = 4 queries finish in its prologue (label-space layer 2 for
    every query with k >= 4, then the closed form); with load flag bit 8 they
    run per point in the persistent kernel. Mixed k = 3..6, plain and motif,
    on the hub graph and a uniform one, against single queries and the oracle."""
    import torch
    for idx in (0, 2):
        name, g, _ = _graphs()[idx]
        n = g["n"]
        ncol = int(g["color"].max()) + 1
        qs = W.query_set(g, 24, 3, 6, 0x5EED0044 + idx, colored_every_other=True, ncolors=ncol)
        assert sum(q["k"] == 4 for q in qs) >= 3
        for flags in (0, capi.FLAG_K4_PER_POINT):
            with capi.Graph(g, flags) as G:
                d_w = torch.zeros((len(qs), n), dtype=torch.int64, device="cuda")
                capi.rr_reach_batch_device(G.handle, qs, d_w)
                torch.cuda.synchronize()
                w = d_w.cpu().numpy().view(np.uint64)
                for i, q in enumerate(qs):
                    _, ref = G.reach(q["source"], q["k"], q["seed"], motif=q["motif"])
                    assert np.array_equal(w[i], ref), (name, flags, i, q["k"])
                    if q["k"] == 4:
                        assert np.array_equal(ref, oracle.sieve(g, q["source"], 4, q["seed"],
                                                                motif=q["motif"])), (name, i)
