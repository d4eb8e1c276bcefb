"""Pins for the oracle's sieve (no GPU).

* The paper's worked figures: the exact-k reachable sets read off by hand.
* The determinant identity: for every vertex v the sieve sum equals
  XOR over restless k-vertex paths P from s to v of prod_l y_{e_l,l} * det(Z_P),
  computed by exhaustive DFS + Gaussian elimination, with no sieve at all.
  A dropped term, a wrong window end, a wrong delta owner, a wrong y index
  or a transposed operand changes some sum and fails it.
* The k=2 closed form, one-sided error against brute force, and invariants.
"""
import random

import numpy as np
import pytest

import oracle
from paper_2010_08423_gb300 import workloads as W
from conftest import read_fixture

FIXTURES = ["fig_restless_paths.txt", "fig_fine_grained.txt", "fig_extraction.txt",
            "fig_random_walk.txt"]


def _reach(S):
    return sorted(int(v) for v in np.nonzero(S)[0])


@pytest.mark.parametrize("name", FIXTURES)
def test_figure_reach_sets(name):
    g, s, expect, _ = read_fixture(name)
    for k, want in expect.items():
        for seed in (1, 2, 3):
            S = oracle.sieve(g, s, k, seed)
            assert _reach(S) == want, (name, k, seed)
        reach, _, _ = oracle.dfs_paths(g, s, k)
        assert sorted(np.nonzero(reach)[0].tolist()) == want, (name, k)


def test_random_walk_figure_cancels_exactly():
    g, s, _, _ = read_fixture("fig_random_walk.txt")
    for seed in range(1, 20):
        S = oracle.sieve(g, s, 6, seed)
        assert int(S[4]) == 0  # the walk v1 v2 v3 v4 v2 v5 vanishes
        S5 = oracle.sieve(g, s, 5, seed)
        assert int(S5[1]) == 0  # v1 v2 v3 v4 v2 revisits v2


def test_figure_motif_panel():
    g, s, _, motif = read_fixture("fig_restless_paths.txt")
    for seed in (11, 12):
        S = oracle.sieve(g, s, 6, seed, motif=motif)
        assert _reach(S) == [5]
        reach, _, _ = oracle.dfs_paths(g, s, 6, motif=motif)
        assert np.nonzero(reach)[0].tolist() == [5]


def test_determinant_identity_plain_random_tiny():
    rng = random.Random(7)
    checked = 0
    for gi in range(250):
        g = W.tiny_random(1000 + gi, n=rng.randint(3, 8), m=rng.randint(3, 20),
                          tau=rng.randint(1, 6), dmax=rng.randint(0, 3))
        s = rng.randrange(g["n"])
        for k in range(2, min(g["n"], 5) + 1):
            seed = rng.getrandbits(64)
            S = oracle.sieve(g, s, k, seed)
            _, sdet, npaths = oracle.dfs_paths(g, s, k, seed, with_det=True)
            assert np.array_equal(S, sdet), (gi, k)
            checked += npaths > 0
    assert checked > 100


def test_determinant_identity_colored_random_tiny():
    rng = random.Random(8)
    checked = 0
    for gi in range(200):
        ncol = rng.randint(1, 3)
        g = W.tiny_random(5000 + gi, n=rng.randint(3, 8), m=rng.randint(3, 20),
                          tau=rng.randint(1, 6), dmax=rng.randint(0, 3), ncolors=ncol)
        s = rng.randrange(g["n"])
        for k in range(2, min(g["n"], 5) + 1):
            motif = [int(g["color"][s])] + [rng.randrange(ncol + 1) for _ in range(k - 1)]
            seed = rng.getrandbits(64)
            S = oracle.sieve(g, s, k, seed, motif=motif)
            _, sdet, npaths = oracle.dfs_paths(g, s, k, seed, motif=motif, with_det=True)
            assert np.array_equal(S, sdet), (gi, k, motif)
            checked += npaths > 0
    assert checked > 50


def test_k2_closed_form():
    # k = 2: S[v] = (z_{s,1} z_{v,2} + z_{s,2} z_{v,1}) * sum_{e: s->v} y_{e,1}
    g = W.tiny_random(77, n=6, m=20, tau=4, dmax=2)
    s = 0
    seed = 0xDEADBEEF
    S = oracle.sieve(g, s, 2, seed)
    z = oracle.ztable(g["n"], 2, seed)
    for v in range(g["n"]):
        ysum = 0
        for e in range(len(g["src"])):
            if g["src"][e] == s and g["dst"][e] == v:
                ysum ^= oracle.y_value(seed, e, 1)
        det = oracle.gf_mul(int(z[s, 0]), int(z[v, 1])) ^ oracle.gf_mul(int(z[s, 1]), int(z[v, 0]))
        assert int(S[v]) == oracle.gf_mul(det, ysum)


def test_per_mask_sums_and_empty_mask():
    g = W.tiny_random(78, n=7, m=18)
    S, pm = oracle.sieve(g, 0, 4, 99, per_mask=True)
    acc = np.zeros_like(S)
    for row in pm:
        acc ^= row
    assert np.array_equal(acc, S)
    assert not pm[0].any()  # L = {} gives x = 0 everywhere
    sub = oracle.sieve(g, 0, 4, 99, masks=[3, 5, 9])
    assert np.array_equal(sub, pm[3] ^ pm[5] ^ pm[9])


def test_small_uniform_one_sided_and_invariants():
    # The n=1,000 / m=10,000 uniform workload has few long restless paths
    # (none of 5 vertices from s=0), so several sources and k are checked.
    g = W.small_uniform()
    total = 0
    indeg = np.bincount(g["dst"], minlength=g["n"])
    for s in range(6):
        for k in (3, 4, 5):
            S = oracle.sieve(g, s, k, 0x5EED0001 ^ (s * 16 + k))
            reach, _, npaths = oracle.dfs_paths(g, s, k)
            total += npaths
            nz = S != 0
            # one-sided: every non-zero sum is witnessed by a path
            assert not np.any(nz & (reach == 0))
            # false negatives have probability <= (2k-1)/2^64 per vertex
            assert np.array_equal(nz, reach.astype(bool)), (s, k)
            assert S[s] == 0
            assert not np.any(S[indeg == 0])
    assert total > 10


def test_separator_colour_and_plain_vs_single_colour():
    g = W.tiny_random(90, n=8, m=20, tau=5, dmax=2, ncolors=2)
    s = 0
    k = 4
    # single colour: decisions equal the plain query
    g1 = dict(g, color=np.zeros(g["n"], dtype=np.uint8))
    Sp = oracle.sieve(g1, s, k, 5)
    Sm = oracle.sieve(g1, s, k, 5, motif=[0] * k)
    assert np.array_equal(Sp != 0, Sm != 0)
    # separators: vertices of a colour not in M never lie on a reported path
    motif = [int(g["color"][s])] * k
    Sc = oracle.sieve(g, s, k, 6, motif=motif)
    reach, _, _ = oracle.dfs_paths(g, s, k, motif=motif)
    assert np.array_equal(Sc != 0, reach.astype(bool))
    other = 1 - int(g["color"][s])
    assert not np.any((Sc != 0) & (g["color"] == other))


def test_rejects_bad_input():
    g = W.tiny_random(91)
    with pytest.raises(ValueError):
        oracle.sieve(g, 0, 1, 1)
    with pytest.raises(ValueError):
        oracle.sieve(g, g["n"], 3, 1)
    bad = dict(g, dst=g["src"].copy())
    with pytest.raises(ValueError):
        oracle.sieve(bad, 0, 3, 1)
