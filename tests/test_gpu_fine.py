"""GPU parity of the fine-grained outputs (Algorithm 1's per-time polynomials).

rr_reach_arrival_device returns, besides the witness, the per-edge sums E
(every input edge's last-layer value summed over all sieve points), the
minimum arrival time R and the set D = {u : R_u defined}. All are exact
GF(2^64) / integer results: compared with the oracle element by element.
"""
import numpy as np
import pytest

import oracle
from paper_2010_08423_gb300 import capi
from paper_2010_08423_gb300 import workloads as W
from conftest import read_arrivals, read_fixture

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    capi.load()
    oracle.build()
    torch.cuda.set_device(0)


def _check(G, g, s, k, seed, motif=None):
    S, E, R, bm = G.arrival(s, k, seed, motif=motif)
    S_ref, E_ref = oracle.sieve(g, s, k, seed, motif=motif, edges=True)
    R_ref = oracle.arrival_times(g, E_ref)
    assert np.array_equal(S, S_ref), (s, k)
    assert np.array_equal(E, E_ref), (s, k)
    assert np.array_equal(R, R_ref), (s, k)
    D = np.unpackbits(bm, bitorder="little")[:g["n"]].astype(bool)
    assert np.array_equal(D, R_ref != oracle.NO_ARRIVAL)
    return R_ref


@pytest.mark.parametrize("flags", [0, capi.FLAG_DENSE_STATE])
def test_random_tiny_graphs_both_engines(flags):
    rng = np.random.default_rng(71)
    hits = 0
    for gi in range(30):
        g = W.tiny_random(1700 + gi, n=int(rng.integers(3, 9)), m=int(rng.integers(1, 25)),
                          tau=int(rng.integers(1, 7)), dmax=int(rng.integers(0, 4)), ncolors=2)
        with capi.Graph(g, flags) as G:
            for k in (2, 3, 4, 5):
                s = int(rng.integers(0, g["n"]))
                seed = int(rng.integers(0, 2**63))
                R = _check(G, g, s, k, seed)
                hits += int((R != oracle.NO_ARRIVAL).any())
                motif = [int(g["color"][s])] + [int(x) for x in rng.integers(0, 2, k - 1)]
                _check(G, g, s, k, seed, motif=motif)
    assert hits >= 30


def test_fine_grained_figure():
    g, s, _, _ = read_fixture("fig_fine_grained.txt")
    want = read_arrivals("fig_fine_grained.txt")
    with capi.Graph(g) as G:
        for k, per_v in want.items():
            _, _, R, _ = G.arrival(s, k, 3)
            got = {int(v): int(R[v]) for v in np.nonzero(R != capi.NO_ARRIVAL)[0]}
            assert got == per_v, k


@pytest.mark.parametrize("flags", [0, capi.FLAG_DENSE_STATE])
def test_ragged_uniform_graph_several_k(flags):
    g = W.uniform(2000, 30_011, 40, 0, 6, 11, ncolors=3)
    with capi.Graph(g, flags) as G:
        for s, k, seed in ((0, 5, 1), (17, 6, 2), (5, 7, 3)):
            R = _check(G, g, s, k, seed)
            assert (R != oracle.NO_ARRIVAL).sum() > 20
        _check(G, g, 5, 5, 9, motif=[int(g["color"][5]), 0, 1, 2, 1])


def test_multi_chunk_k10():
    g = W.uniform(800, 9_000, 12, 0, 4, 80)
    with capi.Graph(g) as G:
        R = _check(G, g, 1, 10, 1010)
        assert (R != oracle.NO_ARRIVAL).sum() > 10


def test_cut_hub_segments():
    from test_gpu_parity import _hub_graph
    g = _hub_graph()
    with capi.Graph(g) as G:
        for s, k in ((3, 3), (5, 4), (7, 5), (0, 6)):
            _check(G, g, s, k, 70 + k)


def test_without_edge_buffer_and_on_an_edgeless_graph():
    import torch
    g = W.uniform(500, 6_000, 15, 0, 4, 12)
    n = g["n"]
    with capi.Graph(g) as G:
        _, _, R_full, _ = G.arrival(2, 6, 4)
        d_w = torch.zeros(n, dtype=torch.int64, device="cuda")
        d_r = torch.zeros(n, dtype=torch.int32, device="cuda")
        capi.rr_reach_arrival_device(G.handle, 2, 6, 4, d_w, d_r)
        torch.cuda.synchronize()
        assert np.array_equal(d_r.cpu().numpy().view(np.uint32), R_full)
        with pytest.raises(capi.RRError) as ei:
            capi.rr_reach_arrival_device(G.handle, 2, 6, 4, d_w, None)
        assert ei.value.status == capi.RR_EINVAL
    empty = {"n": 4, "src": np.zeros(0, np.uint32), "dst": np.zeros(0, np.uint32),
             "t": np.zeros(0, np.uint32), "delta": np.ones(4, np.uint32)}
    with capi.Graph(empty) as G:
        S, E, R, bm = G.arrival(0, 3, 1)
        assert not S.any() and E.size == 0 and (R == capi.NO_ARRIVAL).all() and not bm.any()


@pytest.mark.parametrize("k", [2, 5, 8])
def test_bounded_reach_min_arrival_and_shortest_length(k):
    import torch
    g = W.uniform(1500, 20_000, 30, 0, 5, 60 + k)
    n = g["n"]
    R_ref, L_ref = oracle.atmost_arrival(g, 4, k, 13)
    with capi.Graph(g) as G:
        d_r = torch.zeros(n, dtype=torch.int32, device="cuda")
        d_l = torch.full((n,), 99, dtype=torch.uint8, device="cuda")
        d_b = torch.zeros((n + 7) // 8, dtype=torch.uint8, device="cuda")
        for rep in range(2):  # lanes reused on the second call
            capi.rr_reach_bounded_device(G.handle, 4, k, 13, d_r, d_l, d_b)
            torch.cuda.synchronize()
            R = d_r.cpu().numpy().view(np.uint32)
            assert np.array_equal(R, R_ref)
            assert np.array_equal(d_l.cpu().numpy(), L_ref)
            D = np.unpackbits(d_b.cpu().numpy(), bitorder="little")[:n].astype(bool)
            assert np.array_equal(D, R_ref != oracle.NO_ARRIVAL)
        assert (L_ref > 0).sum() > 3
