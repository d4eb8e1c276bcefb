"""Pins for the oracle's path extraction (no GPU).

Sec. "Extracting an optimal solution using k queries": k-1 fine-grained
queries, each on the graph without the vertices already chosen, recover one
restless path whose last time is the target's minimum arrival time.

* The worked example in the text (extraction figure): v1 v4 v5 v6 at 2, 3, 5.
* On random graphs the result is checked by a plain validator of the path
  definition (consecutive edges, restless waits, distinct vertices, the motif's
  colours) and its last time against the earliest arrival found by DFS; no
  path is returned exactly when DFS finds none.
"""
import random

import numpy as np

import oracle
from paper_2010_08423_gb300 import workloads as W
from conftest import read_fixture, read_paths


def valid_restless_path(g, s, target, k, res, motif=None):
    path, edges, times = res
    src, dst, t, delta = g["src"], g["dst"], g["t"], g["delta"]
    assert len(path) == k and len(edges) == k - 1 and len(times) == k - 1
    assert path[0] == s and path[-1] == target and len(set(path)) == k
    for j, e in enumerate(edges):
        assert src[e] == path[j] and dst[e] == path[j + 1] and t[e] == times[j]
    for j in range(1, k - 1):
        assert 0 <= times[j] - times[j - 1] <= delta[path[j]]
    if motif is not None:
        assert sorted(int(g["color"][v]) for v in path) == sorted(motif)


def test_extraction_figure_path():
    g, s, _, _ = read_fixture("fig_extraction.txt")
    want = read_paths("fig_extraction.txt")
    for k, (verts, times) in want.items():
        for seed in (1, 2, 3):
            res = oracle.extract_path(g, s, k, seed, verts[-1])
            assert res is not None
            assert res[0] == verts and res[2] == times, (k, seed, res)
            valid_restless_path(g, s, verts[-1], k, res)


def test_random_graphs_valid_and_optimal():
    rng = random.Random(61)
    found = missing = 0
    for gi in range(50):
        g = W.tiny_random(6100 + gi, n=rng.randint(4, 8), m=rng.randint(6, 24),
                          tau=rng.randint(2, 6), dmax=rng.randint(1, 3))
        s = rng.randrange(g["n"])
        k = rng.randint(2, min(5, g["n"]))
        _, _, _, _, arrive = oracle.dfs_paths(g, s, k, with_edges=True)
        for target in range(g["n"]):
            if target == s:
                continue
            res = oracle.extract_path(g, s, k, rng.getrandbits(63), target)
            if arrive[target] == oracle.NO_ARRIVAL:
                assert res is None
                missing += 1
            else:
                assert res is not None
                valid_restless_path(g, s, target, k, res)
                assert res[2][-1] == arrive[target]
                found += 1
    assert found >= 30 and missing >= 30


def test_random_graphs_motif():
    rng = random.Random(67)
    found = 0
    for gi in range(60):
        g = W.tiny_random(6700 + gi, n=rng.randint(4, 8), m=rng.randint(8, 24),
                          tau=rng.randint(2, 6), dmax=rng.randint(1, 3), ncolors=2)
        s = rng.randrange(g["n"])
        k = rng.randint(2, min(5, g["n"]))
        motif = [int(g["color"][s])] + [rng.randrange(2) for _ in range(k - 1)]
        _, _, _, _, arrive = oracle.dfs_paths(g, s, k, motif=motif, with_edges=True)
        for target in range(g["n"]):
            if target == s:
                continue
            res = oracle.extract_path(g, s, k, 5 + gi, target, motif=motif)
            if arrive[target] == oracle.NO_ARRIVAL:
                assert res is None
            else:
                assert res is not None
                valid_restless_path(g, s, target, k, res, motif=motif)
                assert res[2][-1] == arrive[target]
                found += 1
    assert found >= 15


def test_deleted_vertices_equal_paths_that_avoid_them():
    # z_u = 0 for deleted u (the sieve) against a DFS that never visits them:
    # the determinant sums split by last edge must agree bit for bit
    rng = random.Random(71)
    hits = 0
    for gi in range(40):
        g = W.tiny_random(7100 + gi, n=rng.randint(4, 8), m=rng.randint(6, 22),
                          tau=rng.randint(2, 5), dmax=rng.randint(0, 3), ncolors=2)
        s = rng.randrange(g["n"])
        k = rng.randint(2, min(5, g["n"]))
        deleted = np.zeros(g["n"], np.uint8)
        for v in rng.sample([v for v in range(g["n"]) if v != s], rng.randint(1, 2)):
            deleted[v] = 1
        seed = rng.getrandbits(63)
        motif = None if gi % 2 else [int(g["color"][s])] + [rng.randrange(2) for _ in range(k - 1)]
        _, E = oracle.sieve(g, s, k, seed, motif=motif, edges=True, deleted=deleted)
        _, _, _, edet, _ = oracle.dfs_paths(g, s, k, seed, motif=motif, with_det=True,
                                            with_edges=True, deleted=deleted)
        assert np.array_equal(E, edet), gi
        _, E_all = oracle.sieve(g, s, k, seed, motif=motif, edges=True)
        hits += int(not np.array_equal(E, E_all))
    assert hits >= 5
