"""The algebra behind the pair-label layer 3 and the k = 4 and k = 5 closed
forms, checked on the CPU with the oracle's field multiply (no GPU, no CUDA
code involved).

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


# ---------------------------------------------------------------------------
# Closed forms for k = 4 and k = 5 (no sieve points): summed over every L in
# [k], a product of k linear forms in L's labels keeps only the choices of one
# label per form that use every label once (each other choice is counted an
# even number of times), i.e. a permanent.
# ---------------------------------------------------------------------------
def _rand(rng, n):
    return [int(x) for x in rng.integers(1, 2**63, n, dtype=np.int64)]


def _mul(*vals):
    acc = vals[0]
    for v in vals[1:]:
        acc = oracle.gf_mul(acc, v)
    return acc


def _perm(rows):
    """Permanent over GF(2^64) by its definition (every bijection)."""
    from itertools import permutations
    n = len(rows)
    acc = 0
    for sigma in permutations(range(n)):
        acc ^= _mul(*[rows[r][sigma[r]] for r in range(n)])
    return acc


def _k4_quads(zs, b, c, d, slip=False):
    """The k = 4 last layer as the quad of lanes computes it: lane j holds
    column j; Q_{j,j^x} from its own c_j d_{j^x} and lane j^x's, then the minor
    without column j along z_v, then z_{s,j} times it, XORed over the quad.
    slip: Q_{j^2,j^3} taken from lane j^1 instead of j^2 (a wrong partner)."""
    Q = [[oracle.gf_mul(c[j], d[j ^ x]) ^ oracle.gf_mul(c[j ^ x], d[j]) if x else 0 for x in range(4)]
         for j in range(4)]  # Q[j][x] = Q_{j, j^x} as lane j holds it
    perm = 0
    for j in range(4):
        t = (oracle.gf_mul(b[j ^ 1], Q[(j ^ 1) if slip else (j ^ 2)][1]) ^ oracle.gf_mul(b[j ^ 2], Q[j ^ 1][2]) ^
             oracle.gf_mul(b[j ^ 3], Q[j ^ 1][3]))
        perm ^= oracle.gf_mul(zs[j], t)
    return perm


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_k4_closed_form_is_a_permanent(seed):
    rng = np.random.default_rng(40 + seed)
    zs, zv, zw, d = (_rand(rng, 4) for _ in range(4))
    direct = 0
    for L in range(16):
        direct ^= _mul(_lin(zs, L), _lin(zv, L), _lin(zw, L), _lin(d, L))
    assert direct == _perm([zs, zv, zw, d])
    assert _k4_quads(zs, zv, zw, d) == direct
    # a plausible slip in the lane arithmetic: a 2x2 permanent taken from the
    # wrong partner lane
    assert _k4_quads(zs, zv, zw, d, slip=True) != direct


def _k5_lanes(zw, zv, zs, S):
    """The k = 5 last layer as the eight lanes compute it: lane c < 5 forms
    P over {c, c+1} and {c, c+2} (labels mod 5), takes the four others from
    their owners, and adds w_c X_c over the three splits of the other labels."""
    own = [{1: oracle.gf_mul(zv[c], zs[(c + 1) % 5]) ^ oracle.gf_mul(zv[(c + 1) % 5], zs[c]),
            2: oracle.gf_mul(zv[c], zs[(c + 2) % 5]) ^ oracle.gf_mul(zv[(c + 2) % 5], zs[c])}
           for c in range(5)]

    def P(x, y):
        d = (y - x) % 5
        return own[x][d] if d <= 2 else own[y][5 - d]

    total = 0
    for c in range(5):
        o = [t for t in range(5) if t != c]
        X = 0
        for (a, b), (e, f) in (((o[0], o[1]), (o[2], o[3])), ((o[0], o[2]), (o[1], o[3])),
                               ((o[0], o[3]), (o[1], o[2]))):
            X ^= oracle.gf_mul(S[a][b], P(e, f)) ^ oracle.gf_mul(S[e][f], P(a, b))
        total ^= oracle.gf_mul(zw[c], X)
    return total


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_k5_closed_form_over_pair_sums(seed):
    """sum_L x_w^L x_v^L x_s^L sum_{i,j in L} Q_ij for an arbitrary (not
    symmetric) Q equals the split formula over S_ij = Q_ij + Q_ji and the 2x2
    permanents of z_v, z_s, and the sum over every bijection of the labels
    onto (w, v, s, the pair) by definition."""
    from itertools import permutations
    rng = np.random.default_rng(50 + seed)
    zw, zv, zs = (_rand(rng, 5) for _ in range(3))
    Q = [_rand(rng, 5) for _ in range(5)]
    direct = 0
    for L in range(32):
        q = 0
        for i in range(5):
            for j in range(5):
                if (L >> i) & 1 and (L >> j) & 1:
                    q ^= Q[i][j]
        direct ^= _mul(_lin(zw, L), _lin(zv, L), _lin(zs, L), q)
    brute = 0
    for a, b, c, i, j in permutations(range(5)):
        brute ^= _mul(zw[a], zv[b], zs[c], Q[i][j])
    assert direct == brute
    S = [[Q[i][j] ^ Q[j][i] if i != j else 0 for j in range(5)] for i in range(5)]
    assert _k5_lanes(zw, zv, zs, S) == direct
    # the diagonal of Q never survives the sum over L ...
    Qd = [[Q[i][j] ^ (int(rng.integers(1, 2**62)) if i == j else 0) for j in range(5)] for i in range(5)]
    direct_d = 0
    for L in range(32):
        q = 0
        for i in range(5):
            for j in range(5):
                if (L >> i) & 1 and (L >> j) & 1:
                    q ^= Qd[i][j]
        direct_d ^= _mul(_lin(zw, L), _lin(zv, L), _lin(zs, L), q)
    assert direct_d == direct
    # ... and one order of each pair alone (not symmetrised) is wrong
    S_half = [[Q[i][j] if i > j else Q[j][i] if i != j else 0 for j in range(5)] for i in range(5)]
    assert _k5_lanes(zw, zv, zs, S_half) != direct
