"""Pins for the multi-source and separator forms of the oracle (no GPU).

Sec. "Discussion": RestlessReach from a set of sources. Starting walks at
every edge leaving a source makes the sieve sum the XOR over the sources of
their single-source sums (every layer is linear in layer 1); the determinant
identity, by DFS from each source, pins it without any sieve. Separators
(case study: vertices no path may use) are deleted vertices; the reachable
set then equals DFS on the graph without them.
"""
import random

import numpy as np

import oracle
from paper_2010_08423_gb300 import workloads as W


def _graphs(count, seed, ncolors=0):
    rng = random.Random(seed)
    for gi in range(count):
        g = W.tiny_random(seed * 100 + gi, n=rng.randint(4, 9), m=rng.randint(4, 26),
                          tau=rng.randint(1, 6), dmax=rng.randint(0, 3), ncolors=ncolors)
        k = rng.randint(2, min(5, g["n"]))
        srcs = rng.sample(range(g["n"]), rng.randint(1, min(3, g["n"] - 1)))
        yield g, srcs, k, rng.getrandbits(63), rng


def test_sources_equal_determinant_sums_from_each_source():
    hits = 0
    for g, srcs, k, seed, _ in _graphs(60, 31):
        S, E = oracle.sieve(g, 0, k, seed, sources=srcs, edges=True)
        want_S = np.zeros(g["n"], np.uint64)
        want_E = np.zeros(len(g["src"]), np.uint64)
        for s in srcs:
            _, sdet, _, edet, _ = oracle.dfs_paths(g, s, k, seed, with_det=True, with_edges=True)
            want_S ^= sdet
            want_E ^= edet
        assert np.array_equal(S, want_S) and np.array_equal(E, want_E), (srcs, k)
        hits += int(S.any())
    assert hits >= 20


def test_sources_motif_equal_determinant_sums():
    hits = 0
    for g, srcs, k, seed, rng in _graphs(60, 37, ncolors=2):
        motif = [rng.randrange(2) for _ in range(k)]
        S = oracle.sieve(g, 0, k, seed, sources=srcs, motif=motif)
        want = np.zeros(g["n"], np.uint64)
        for s in srcs:
            _, sdet, _ = oracle.dfs_paths(g, s, k, seed, motif=motif, with_det=True)
            want ^= sdet
        assert np.array_equal(S, want)
        hits += int(S.any())
    assert hits >= 5


def test_one_source_in_the_set_is_the_single_source_query():
    g = W.uniform(50, 400, 10, 0, 3, 3)
    for k in (2, 4, 6):
        assert np.array_equal(oracle.sieve(g, 0, k, 5, sources=[7]), oracle.sieve(g, 7, k, 5))


def test_separators_block_every_path():
    rng = random.Random(43)
    checked = 0
    for g, srcs, k, seed, _ in _graphs(60, 43):
        s = srcs[0]
        others = [v for v in range(g["n"]) if v != s]
        seps = rng.sample(others, min(2, len(others)))
        deleted = np.zeros(g["n"], np.uint8)
        deleted[seps] = 1
        S = oracle.sieve(g, s, k, seed, deleted=deleted)
        reach, _, _ = oracle.dfs_paths(g, s, k, deleted=deleted)
        assert np.array_equal(S != 0, reach.astype(bool))
        assert not (S[seps] != 0).any()
        checked += int(reach.any())
    assert checked >= 10
