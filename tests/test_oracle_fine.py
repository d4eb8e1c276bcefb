"""Pins for the oracle's fine-grained outputs (no GPU).

Algorithm 1 keeps one polynomial per (vertex u, arrival time i): the walks of
k vertices ending at u with a last edge at time i. In the edge-layer form that
is the XOR of the per-edge sums E[e] over the edges e into u with t_e = i, and
R_u is the smallest i whose polynomial is non-zero.

* The determinant identity split by last edge: E[e] equals the XOR over the
  restless k-vertex paths whose last edge is e of prod_l y_{e_l,l} * det(Z_P),
  from exhaustive DFS with no sieve. A wrong layer, a dropped term or a
  per-vertex (not per-edge) accumulation fails it.
* R from the sums equals the earliest last-edge time of a DFS path ending at u
  (a path's polynomial is non-zero with probability >= 1 - (3k-1)/2^64).
* The worked figure's arrival times, one of them stated in the paper's text.
"""
import random

import numpy as np
import pytest

import oracle
from paper_2010_08423_gb300 import workloads as W
from conftest import read_arrivals, read_fixture


def _random_graphs(count, seed, ncolors=0):
    rng = random.Random(seed)
    for gi in range(count):
        g = W.tiny_random(seed * 100 + gi, n=rng.randint(3, 8), m=rng.randint(2, 22),
                          tau=rng.randint(1, 6), dmax=rng.randint(0, 3), ncolors=ncolors)
        s = rng.randrange(g["n"])
        k = rng.randint(2, min(6, g["n"]))
        yield g, s, k, rng.getrandbits(64), rng


def test_edge_sums_equal_determinant_split_by_last_edge():
    hits = 0
    for g, s, k, seed, _ in _random_graphs(60, 41):
        S, E = oracle.sieve(g, s, k, seed, edges=True)
        _, sdet, npaths, edet, _ = oracle.dfs_paths(g, s, k, seed, with_det=True, with_edges=True)
        assert np.array_equal(E, edet), (s, k)
        assert np.array_equal(S, sdet)
        hits += np.count_nonzero(E) > 0
    assert hits >= 20


def test_edge_sums_colored_equal_determinant_split():
    hits = 0
    for g, s, k, seed, rng in _random_graphs(100, 43, ncolors=2):
        motif = [int(g["color"][s])] + [rng.randrange(2) for _ in range(k - 1)]
        _, E = oracle.sieve(g, s, k, seed, motif=motif, edges=True)
        _, _, _, edet, _ = oracle.dfs_paths(g, s, k, seed, motif=motif, with_det=True,
                                            with_edges=True)
        assert np.array_equal(E, edet), (s, k, motif)
        hits += np.count_nonzero(E) > 0
    assert hits >= 10


def test_edge_sums_xor_to_the_witness():
    g = W.uniform(60, 500, 12, 0, 3, 7)
    for k in (2, 3, 5):
        S, E = oracle.sieve(g, 1, k, 99 + k, edges=True)
        per_head = np.zeros(g["n"], dtype=np.uint64)
        np.bitwise_xor.at(per_head, g["dst"].astype(np.int64), E)
        assert np.array_equal(per_head, S)


def test_arrival_times_equal_dfs_earliest_arrival():
    nonempty = 0
    for g, s, k, seed, _ in _random_graphs(60, 47):
        _, E = oracle.sieve(g, s, k, seed, edges=True)
        R = oracle.arrival_times(g, E)
        reach, _, _, _, arrive = oracle.dfs_paths(g, s, k, with_edges=True)
        assert np.array_equal(R, arrive), (s, k)
        assert np.array_equal(R != oracle.NO_ARRIVAL, reach.astype(bool))
        nonempty += int((R != oracle.NO_ARRIVAL).any())
    assert nonempty >= 20


def test_arrival_on_a_uniform_graph_with_many_times():
    g = W.uniform(80, 900, 12, 0, 5, 8)
    for k in (3, 4):
        _, E = oracle.sieve(g, 2, k, 5, edges=True)
        R = oracle.arrival_times(g, E)
        _, _, _, _, arrive = oracle.dfs_paths(g, 2, k, with_edges=True)
        assert np.array_equal(R, arrive)
        assert (R != oracle.NO_ARRIVAL).sum() > 10


def test_fine_grained_figure_arrivals():
    g, s, _, _ = read_fixture("fig_fine_grained.txt")
    want = read_arrivals("fig_fine_grained.txt")
    assert want[4] == {4: 5}
    for k, per_v in want.items():
        for seed in (1, 2):
            _, E = oracle.sieve(g, s, k, seed, edges=True)
            R = oracle.arrival_times(g, E)
            got = {int(v): int(R[v]) for v in np.nonzero(R != oracle.NO_ARRIVAL)[0]}
            assert got == per_v, (k, seed)


def test_arrival_times_definition_on_hand_made_sums():
    # grouping by (head, time) and the minimum, on values set by hand:
    # edges into v=1 at t=4 cancel, so R[1] is the next time with a non-zero sum
    g = {"n": 3, "src": np.array([0, 2, 0, 0], np.uint32), "dst": np.array([1, 1, 1, 2], np.uint32),
         "t": np.array([4, 4, 7, 3], np.uint32), "delta": np.zeros(3, np.uint32)}
    E = np.array([5, 5, 9, 0], dtype=np.uint64)
    R = oracle.arrival_times(g, E)
    assert R.tolist() == [oracle.NO_ARRIVAL, 7, oracle.NO_ARRIVAL]


def test_bounded_restless_reach_equals_dfs_over_lengths():
    # R = min over k' <= k of the DFS earliest arrival with k' vertices; L = the
    # smallest k' that reaches v (shortest restless path, in vertices)
    checked = 0
    for g, s, k, seed, _ in _random_graphs(50, 53):
        R, L = oracle.atmost_arrival(g, s, k, seed)
        want_R = np.full(g["n"], oracle.NO_ARRIVAL, dtype=np.uint32)
        want_L = np.zeros(g["n"], dtype=np.uint8)
        for kk in range(2, k + 1):
            _, _, _, _, arrive = oracle.dfs_paths(g, s, kk, with_edges=True)
            want_L[(want_L == 0) & (arrive != oracle.NO_ARRIVAL)] = kk
            want_R = np.minimum(want_R, arrive)
        assert np.array_equal(R, want_R) and np.array_equal(L, want_L), (s, k)
        checked += int((L > 0).any())
    assert checked >= 20
