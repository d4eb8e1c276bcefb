"""The algebra behind the pair-label layer 3, checked on the CPU with the
oracle's field multiply (no GPU, no CUDA code involved).

Layer 3 of a head keeps, instead of one value per sieve point L, the k(k+1)/2
values of the symmetric label-pair matrix Q = XOR over the head's rows e of
z_{u_e} (x) g_e (value (i, j), i >= j, at i(i+1)/2 + j: Q_ii on the diagonal,
Q_ij ^ Q_ji off it), because
    XOR_e x_{u_e}^L g_e^L = sum_{i,j in L} Q_ij   for every L,
with x^L = sum_{i in L} z_i and g^L = sum_{i in L} g_i. The kernels evaluate
the right-hand side per lane from a base over the labels above the lane's
lowest LOGP bits plus per-low-label corrections; both the identity and that
split evaluation are checked here for every point.
"""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module", autouse=True)
def _lib():
    oracle.build()


def _lin(vals, L):
    acc = 0
    for i, v in enumerate(vals):
        if (L >> i) & 1:
            acc ^= v
    return acc


def _pairs(zs, gs, k):
    Q = [[0] * k for _ in range(k)]
    for z, g in zip(zs, gs):
        for i in range(k):
            for j in range(k):
                Q[i][j] ^= oracle.gf_mul(z[i], g[j])
    P = [0] * (k * (k + 1) // 2)
    for i in range(k):
        for j in range(i + 1):
            P[i * (i + 1) // 2 + j] = Q[i][i] if i == j else Q[i][j] ^ Q[j][i]
    return P


def _form(P, L, k):
    acc = 0
    for i in range(k):
        for j in range(i + 1):
            if (L >> i) & 1 and (L >> j) & 1:
                acc ^= P[i * (i + 1) // 2 + j]
    return acc


def _split(P, pbits, k, logp):
    """The per-lane evaluation: labels >= logp from pbits, then the points
    pbits + i, i < 2^logp."""
    base, t0 = 0, P[0]
    t1 = P[2] if logp == 2 else 0
    s01 = P[1] if logp == 2 else 0
    for i in range(logp, k):
        r = i * (i + 1) // 2
        row = P[r + i]
        for j in range(logp, i):
            if (pbits >> j) & 1:
                row ^= P[r + j]
        if (pbits >> i) & 1:
            base ^= row
            t0 ^= P[r]
            if logp == 2:
                t1 ^= P[r + 1]
    out = [base, base ^ t0]
    if logp == 2:
        out += [base ^ t1, base ^ t0 ^ t1 ^ s01]
    return out


@pytest.mark.parametrize("k,rows", [(6, 1), (9, 3), (11, 5)])
def test_pair_form_equals_the_sum_of_products(k, rows):
    rng = np.random.default_rng(1000 + k)
    zs = [[int(x) << 1 | 1 for x in rng.integers(0, 2**63, k, dtype=np.int64)] for _ in range(rows)]
    gs = [[int(x) for x in rng.integers(0, 2**63, k, dtype=np.int64)] for _ in range(rows)]
    P = _pairs(zs, gs, k)
    for L in range(1 << k):
        direct = 0
        for z, g in zip(zs, gs):
            direct ^= oracle.gf_mul(_lin(z, L), _lin(g, L))
        assert _form(P, L, k) == direct, L
    for logp in (1, 2):
        for pbits in range(0, 1 << k, 1 << logp):
            got = _split(P, pbits, k, logp)
            assert got == [_form(P, pbits + i, k) for i in range(1 << logp)], (logp, pbits)


def test_a_wrong_symmetrisation_is_caught():
    k = 6
    rng = np.random.default_rng(7)
    z = [int(x) | 1 for x in rng.integers(1, 2**62, k)]
    g = [int(x) for x in rng.integers(1, 2**62, k)]
    P = _pairs([z], [g], k)
    bad = list(P)
    bad[4] = bad[4] ^ oracle.gf_mul(z[2], g[1])  # drop one order of (2, 1)
    L = (1 << 1) | (1 << 2)
    direct = oracle.gf_mul(_lin(z, L), _lin(g, L))
    assert _form(P, L, k) == direct and _form(bad, L, k) != direct
