"""GPU parity of layer 3 in pair-label space.

Layer 3 stores per deep row the k(k+1)/2 values of a symmetric label-pair
matrix (no sieve points) and layer 4 evaluates, per point, each window's
quadratic form sum_{i,j in L} dQ_ij times x_u x_s. The field products are the
same, so witnesses, per-edge sums and arrival times must equal the oracle bit
for bit with the form forced on (from k = 6), forced off, and by default.
"""
import numpy as np
import pytest

import oracle
from paper_2010_08423_gb300 import capi
from paper_2010_08423_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MODES = [0, capi.FLAG_PAIR_ON, capi.FLAG_PAIR_OFF]
MIN_K = {0: 9, capi.FLAG_PAIR_ON: 6, capi.FLAG_PAIR_OFF: 21}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    capi.load()
    oracle.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("flags", MODES)
def test_witness_all_k_plain_and_motif(flags):
    g = W.uniform(1500, 24_000, 30, 0, 6, 606, ncolors=3)
    with capi.Graph(g, flags) as G:
        assert G.info()["pair_layer3_min_k"] == MIN_K[flags]
        for s, k, seed in ((0, 5, 1), (3, 6, 2), (9, 7, 3), (4, 8, 4), (2, 10, 5)):
            _, w = G.reach(s, k, seed)
            assert np.array_equal(w, oracle.sieve(g, s, k, seed)), (s, k)
            motif = [int(g["color"][s])] + [(j * 7 + k) % 3 for j in range(k - 1)]
            _, w = G.reach(s, k, seed, motif=motif)
            assert np.array_equal(w, oracle.sieve(g, s, k, seed, motif=motif)), (s, k, motif)


@pytest.mark.parametrize("flags", MODES)
def test_larger_k_on_a_small_dense_graph(flags):
    g = W.uniform(200, 4_000, 12, 0, 5, 616)
    with capi.Graph(g, flags) as G:
        for s, k in ((1, 11), (2, 12), (3, 13)):
            _, w = G.reach(s, k, 70 + k)
            assert np.array_equal(w, oracle.sieve(g, s, k, 70 + k)), (s, k)


@pytest.mark.parametrize("flags", MODES)
def test_per_edge_sums_and_arrivals(flags):
    g = W.uniform(1200, 16_000, 25, 0, 5, 707)
    with capi.Graph(g, flags) as G:
        for s, k in ((1, 6), (5, 9)):
            S, E, R, _ = G.arrival(s, k, 40 + k)
            S_ref, E_ref = oracle.sieve(g, s, k, 40 + k, edges=True)
            assert np.array_equal(S, S_ref) and np.array_equal(E, E_ref)
            assert np.array_equal(R, oracle.arrival_times(g, E_ref))


@pytest.mark.parametrize("flags", MODES)
def test_cut_hub_segments_and_both_point_widths(flags):
    from test_gpu_parity import _hub_graph
    g = _hub_graph(seed=11)
    with capi.Graph(g, flags) as G:
        for s, k in ((3, 6), (0, 7), (5, 8)):
            want = oracle.sieve(g, s, k, 90 + k)
            for ppl, chunk in ((2, 64), (4, 128)):
                capi.rr_set_tuning(G.handle, k, ppl, chunk)
                _, w = G.reach(s, k, 90 + k)
                assert np.array_equal(w, want), (s, k, ppl, chunk)


def test_both_pair_row_builders_on_a_sparse_graph():
    """A graph whose deep-row ranges are all short builds the pair rows in one
    launch (fused); the others (hub and uniform graphs above) in two."""
    g = W.uniform(3000, 12_000, 60, 0, 8, 626)
    with capi.Graph(g, capi.FLAG_PAIR_ON) as G:
        assert G.info()["deep_max_range_rows"] <= 4
        for s, k in ((0, 6), (1, 8), (2, 10)):
            _, w = G.reach(s, k, 50 + k)
            assert np.array_equal(w, oracle.sieve(g, s, k, 50 + k)), (s, k)
    from test_gpu_parity import _hub_graph
    with capi.Graph(_hub_graph(seed=11)) as G:
        assert G.info()["deep_max_range_rows"] > 4


@pytest.mark.parametrize("table", [capi.FLAG_HEAD_TABLE_ON, capi.FLAG_HEAD_TABLE_OFF])
def test_head_factor_table_on_and_off(table):
    from test_gpu_parity import _hub_graph
    for g, cases in ((W.uniform(1500, 24_000, 30, 0, 6, 636, ncolors=3), ((0, 7), (5, 10))),
                     (_hub_graph(seed=13), ((3, 6), (0, 9)))):
        with capi.Graph(g, capi.FLAG_PAIR_ON | table) as G:
            assert G.info()["head_table"] == (1 if table == capi.FLAG_HEAD_TABLE_ON else 0)
            for s, k in cases:
                _, w = G.reach(s, k, 30 + k)
                assert np.array_equal(w, oracle.sieve(g, s, k, 30 + k)), (s, k)
                motif = [int(g["color"][s])] + [(j + k) % 3 for j in range(k - 1)]
                _, w = G.reach(s, k, 30 + k, motif=motif)
                assert np.array_equal(w, oracle.sieve(g, s, k, 30 + k, motif=motif)), (s, k)


@pytest.mark.parametrize("table", [capi.FLAG_HEAD_TABLE_ON, capi.FLAG_HEAD_TABLE_OFF])
def test_deleted_vertices_extraction_and_separators(table):
    """The pair form with z rows of deleted vertices (extraction steps) and
    separators: paths equal the oracle's extraction, witnesses its sieve."""
    import torch
    g = W.uniform(600, 6_000, 15, 0, 4, 85, ncolors=3)
    n, s = g["n"], 3
    with capi.Graph(g, capi.FLAG_PAIR_ON | table) as G:
        for k in (6, 7):
            _, _, _, _, arrive = oracle.dfs_paths(g, s, k, with_edges=True)
            targets = [int(v) for v in np.nonzero(arrive != oracle.NO_ARRIVAL)[0][:3]]
            assert targets
            for target in targets:
                assert G.extract_path(s, k, 7, target) == tuple(oracle.extract_path(g, s, k, 7, target))
        rng = np.random.default_rng(87)
        seps = np.zeros(n, np.uint8)
        seps[rng.choice(n, size=60, replace=False)] = 1
        seps[s] = 0
        d_w = torch.zeros(n, dtype=torch.int64, device="cuda")
        d_s = torch.from_numpy(seps).cuda()
        for k in (6, 8):
            capi.rr_reach_sources_device(G.handle, [s], k, 23, d_w, None, d_s)
            torch.cuda.synchronize()
            ref = oracle.sieve(g, 0, k, 23, sources=[s], deleted=seps)
            assert np.array_equal(d_w.cpu().numpy().view(np.uint64), ref), k


def test_atmost_lanes_in_the_pair_form():
    import torch
    g = W.uniform(1500, 20_000, 20, 0, 5, 66)
    n, k = g["n"], 8
    with capi.Graph(g, capi.FLAG_PAIR_ON) as G:
        d_w = torch.zeros((k - 1, n), dtype=torch.int64, device="cuda")
        d_bm = torch.zeros((n + 7) // 8, dtype=torch.uint8, device="cuda")
        capi.rr_reach_atmost_device(G.handle, 3, k, 99, d_w, d_bm)
        torch.cuda.synchronize()
        w = d_w.cpu().numpy().view(np.uint64)
        for kk in range(2, k + 1):
            assert np.array_equal(w[kk - 2], oracle.sieve(g, 3, kk, 99)), kk


def test_pair_on_and_off_together_are_rejected():
    g = W.tiny_random(5, n=6, m=10, tau=3, dmax=2)
    for fl in (capi.FLAG_PAIR_ON | capi.FLAG_PAIR_OFF, capi.FLAG_HEAD_TABLE_ON | capi.FLAG_HEAD_TABLE_OFF):
        with pytest.raises(capi.RRError) as ei:
            capi.Graph(g, fl)
        assert ei.value.status == capi.RR_EINVAL
