"""GPU path extraction (rr_extract_path) against the oracle's extraction.

Both follow the same steps and tie-breaks (Sec. "Extracting an optimal
solution using k queries"), so the returned paths must be identical; each is
also checked against the path definition and for optimality.
"""
import numpy as np
import pytest

import oracle
from paper_2010_08423_gb300 import capi
from paper_2010_08423_gb300 import workloads as W
from conftest import read_fixture, read_paths
from test_oracle_extract import valid_restless_path

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    capi.load()
    oracle.build()
    torch.cuda.set_device(0)


def test_extraction_figure():
    g, s, _, _ = read_fixture("fig_extraction.txt")
    want = read_paths("fig_extraction.txt")
    with capi.Graph(g) as G:
        for k, (verts, times) in want.items():
            res = G.extract_path(s, k, 11, verts[-1])
            assert res is not None and res[0] == verts and res[2] == times


@pytest.mark.parametrize("flags", [0, capi.FLAG_DENSE_STATE])
def test_random_graphs_equal_the_oracle(flags):
    rng = np.random.default_rng(83)
    found = 0
    for gi in range(25):
        g = W.tiny_random(8300 + gi, n=int(rng.integers(4, 9)), m=int(rng.integers(6, 26)),
                          tau=int(rng.integers(2, 7)), dmax=int(rng.integers(1, 4)), ncolors=2)
        s = int(rng.integers(0, g["n"]))
        k = int(rng.integers(2, min(6, g["n"]) + 1))
        seed = int(rng.integers(0, 2**62))
        motif = [int(g["color"][s])] + [int(x) for x in rng.integers(0, 2, k - 1)]
        with capi.Graph(g, flags) as G:
            for target in range(g["n"]):
                if target == s:
                    continue
                for mo in (None, motif):
                    got = G.extract_path(s, k, seed, target, motif=mo)
                    ref = oracle.extract_path(g, s, k, seed, target, motif=mo)
                    assert got == (None if ref is None else tuple(ref)), (gi, target, mo)
                    if got is not None:
                        valid_restless_path(g, s, target, k, got, motif=mo)
                        found += 1
    assert found >= 20


def test_medium_graph_paths_are_optimal():
    g = W.uniform(600, 6_000, 15, 0, 4, 85, ncolors=3)
    s = 3
    with capi.Graph(g) as G:
        for k in (5, 6):
            _, _, _, _, arrive = oracle.dfs_paths(g, s, k, with_edges=True)
            targets = [int(v) for v in np.nonzero(arrive != oracle.NO_ARRIVAL)[0][:4]]
            assert targets
            for target in targets:
                got = G.extract_path(s, k, 7, target)
                assert got == tuple(oracle.extract_path(g, s, k, 7, target))
                valid_restless_path(g, s, target, k, got)
                assert got[2][-1] == arrive[target]


def test_argument_errors():
    g = W.tiny_random(5, n=5, m=8, tau=3, dmax=2)
    with capi.Graph(g) as G:
        for target in (0, 5):
            with pytest.raises(capi.RRError) as ei:
                G.extract_path(0, 3, 1, target)
            assert ei.value.status == capi.RR_EINVAL
