"""GPU parity of queries from a set of sources and with separators.

rr_reach_sources_device must equal the oracle's multi-source sieve bit for
bit (one source: the reduced-state engine, with separators as deleted z rows;
several: the per-point engine with a source mask), and the XOR of the
single-source witnesses (every layer is linear in layer 1).
"""
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


def _run(G, n, sources, k, seed, separators=None, motif=None):
    import torch
    d_w = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    d_b = torch.full(((n + 7) // 8,), 255, dtype=torch.uint8, device="cuda")
    d_s = None
    if separators is not None:
        d_s = torch.from_numpy(np.asarray(separators, dtype=np.uint8)).cuda()
    capi.rr_reach_sources_device(G.handle, sources, k, seed, d_w, d_b, d_s, motif=motif)
    torch.cuda.synchronize()
    w = d_w.cpu().numpy().view(np.uint64)
    bm = np.unpackbits(d_b.cpu().numpy(), bitorder="little")[:n].astype(bool)
    assert np.array_equal(bm, w != 0)
    return w


@pytest.mark.parametrize("flags", [0, capi.FLAG_DENSE_STATE])
def test_random_sets_of_sources(flags):
    rng = np.random.default_rng(91)
    hits = 0
    for gi in range(30):
        g = W.tiny_random(9100 + gi, n=int(rng.integers(4, 10)), m=int(rng.integers(4, 28)),
                          tau=int(rng.integers(1, 6)), dmax=int(rng.integers(0, 4)), ncolors=2)
        n = g["n"]
        with capi.Graph(g, flags) as G:
            for k in (2, 3, 4, 5):
                srcs = [int(x) for x in rng.choice(n, size=int(rng.integers(1, 4)), replace=False)]
                seed = int(rng.integers(0, 2**62))
                w = _run(G, n, srcs, k, seed)
                assert np.array_equal(w, oracle.sieve(g, 0, k, seed, sources=srcs)), (gi, k, srcs)
                hits += int(w.any())
                motif = [int(x) for x in rng.integers(0, 2, k)]
                w = _run(G, n, srcs, k, seed, motif=motif)
                assert np.array_equal(w, oracle.sieve(g, 0, k, seed, sources=srcs, motif=motif))
    assert hits >= 30


def test_sources_xor_of_single_sources_on_a_larger_graph():
    g = W.uniform(1500, 20_000, 25, 0, 5, 93)
    n = g["n"]
    srcs = [3, 77, 400, 901, 1200]
    with capi.Graph(g) as G:
        for k in (4, 7):
            w = _run(G, n, srcs, k, 17)
            assert np.array_equal(w, oracle.sieve(g, 0, k, 17, sources=srcs))
            x = np.zeros(n, np.uint64)
            for s in srcs:
                _, ws = G.reach(s, k, 17)
                x ^= ws
            assert np.array_equal(w, x) and w.any()


@pytest.mark.parametrize("flags", [0, capi.FLAG_DENSE_STATE])
def test_separators(flags):
    rng = np.random.default_rng(97)
    g = W.uniform(800, 9_000, 15, 0, 4, 97, ncolors=3)
    n = g["n"]
    seps = np.zeros(n, np.uint8)
    seps[rng.choice(n, size=80, replace=False)] = 1
    seps[[2, 9]] = 0
    with capi.Graph(g, flags) as G:
        for srcs, k in (([2], 5), ([2], 8), ([2, 9], 6)):
            w = _run(G, n, srcs, k, 23, separators=seps)
            ref = oracle.sieve(g, 0, k, 23, sources=srcs, deleted=seps)
            assert np.array_equal(w, ref), (srcs, k)
            assert not w[seps.astype(bool)].any()
            w_open = _run(G, n, srcs, k, 23)
            assert (w_open != 0).sum() > (w != 0).sum()
        motif = [int(g["color"][2]), 0, 1, 2, 0]
        w = _run(G, n, [2], 5, 29, separators=seps, motif=motif)
        assert np.array_equal(w, oracle.sieve(g, 2, 5, 29, motif=motif, deleted=seps))


def test_argument_errors():
    import torch
    g = W.tiny_random(3, n=6, m=10, tau=3, dmax=2)
    d_w = torch.zeros(6, dtype=torch.int64, device="cuda")
    with capi.Graph(g) as G:
        for srcs in ([], [6]):
            with pytest.raises(capi.RRError) as ei:
                capi.rr_reach_sources_device(G.handle, srcs, 3, 1, d_w)
            assert ei.value.status == capi.RR_EINVAL
