"""Pins for the oracle's GF(2^64) arithmetic and splitmix64 (no GPU).

None of these re-types the oracle's formulas: they check closed forms on the
basis, the ring axioms, Fermat's little theorem (which holds for every
non-zero element only if the modulus is irreducible, i.e. the ring is the field
GF(2^64)), an independent irreducibility proof of the modulus by polynomial
gcd, and published splitmix64 output values.
"""
import itertools
import random

import pytest

import oracle

P_LOW = 0x1B  # x^64 = x^4 + x^3 + x + 1
MOD_FULL = (1 << 64) | P_LOW
M64 = (1 << 64) - 1


def test_basis_products_below_degree_64():
    # x^i * x^j = x^(i+j) when i + j < 64: a single set bit.
    for i in range(64):
        for j in range(64 - i):
            assert oracle.gf_mul(1 << i, 1 << j) == 1 << (i + j)


def test_x64_reduces_to_modulus_tail():
    assert oracle.gf_mul(1 << 63, 2) == P_LOW
    assert oracle.gf_mul(1 << 32, 1 << 32) == P_LOW
    # x^127 = x^63 * x^64 = x^63 (x^4+x^3+x+1) = x^67 + x^66 + x^64 + x^63
    #       = x^3 P + x^2 P + P + x^63 where P = x^4+x^3+x+1 (from x^64 = P)
    x127 = oracle.gf_mul(1 << 63, 1 << 63) ^ 0  # x^126
    x127 = oracle.gf_mul(x127, 2)
    Pp = P_LOW
    expect = ((Pp << 3) ^ (Pp << 2) ^ Pp ^ (1 << 63)) & M64
    assert x127 == expect


def test_identity_and_zero():
    rng = random.Random(1)
    for _ in range(200):
        a = rng.getrandbits(64)
        assert oracle.gf_mul(a, 1) == a
        assert oracle.gf_mul(1, a) == a
        assert oracle.gf_mul(a, 0) == 0


def test_ring_axioms_random():
    rng = random.Random(2)
    for _ in range(2000):
        a, b, c = (rng.getrandbits(64) for _ in range(3))
        ab = oracle.gf_mul(a, b)
        assert ab == oracle.gf_mul(b, a)
        assert oracle.gf_mul(ab, c) == oracle.gf_mul(a, oracle.gf_mul(b, c))
        assert oracle.gf_mul(a, b ^ c) == ab ^ oracle.gf_mul(a, c)


def test_fermat_every_nonzero_has_order_dividing_2_64_minus_1():
    rng = random.Random(3)
    for _ in range(100):
        a = rng.getrandbits(64) or 1
        assert oracle.gf_pow(a, M64) == 1
        inv = oracle.gf_inv(a)
        assert oracle.gf_mul(a, inv) == 1
    # x^(2^64) = x: the Frobenius fixes every element of GF(2^64).
    x = 2
    for _ in range(64):
        x = oracle.gf_mul(x, x)
    assert x == 2
    # ... but x^(2^32) != x, so x is not in the subfield GF(2^32).
    x = 2
    for _ in range(32):
        x = oracle.gf_mul(x, x)
    assert x != 2


def _pmod(a, m):
    dm = m.bit_length() - 1
    while a and a.bit_length() - 1 >= dm:
        a ^= m << (a.bit_length() - 1 - dm)
    return a


def _pmulmod(a, b, m):
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a = _pmod(a << 1, m)
    return _pmod(r, m)


def _pgcd(a, b):
    while b:
        a, b = b, _pmod(a, b)
    return a


def test_modulus_is_irreducible_rabin():
    """Rabin's test for degree 64 (only prime divisor of 64 is 2), done with
    plain GF(2)[x] arithmetic on Python ints, independent of the oracle:
    x^(2^64) = x mod p and gcd(x^(2^32) - x, p) = 1."""
    x = 2
    for _ in range(64):
        x = _pmulmod(x, x, MOD_FULL)
    assert x == 2
    x = 2
    for _ in range(32):
        x = _pmulmod(x, x, MOD_FULL)
    assert _pgcd(MOD_FULL, x ^ 2) == 1


def _perm(mat):
    k = len(mat)
    tot = 0
    for sigma in itertools.permutations(range(k)):
        prod = 1
        for i in range(k):
            prod = oracle.gf_mul(prod, mat[i][sigma[i]])
        tot ^= prod
    return tot


def test_det_equals_permanent_in_char_2():
    rng = random.Random(4)
    for k in range(1, 6):
        for _ in range(20):
            mat = [[rng.getrandbits(64) for _ in range(k)] for _ in range(k)]
            assert oracle.gf_det(mat) == _perm(mat)


def test_det_special_cases():
    rng = random.Random(5)
    a, b, c, d = (rng.getrandbits(64) for _ in range(4))
    # 2x2: ad - bc = ad + bc in characteristic 2
    assert oracle.gf_det([[a, b], [c, d]]) == oracle.gf_mul(a, d) ^ oracle.gf_mul(b, c)
    # equal rows -> 0
    assert oracle.gf_det([[a, b, c], [a, b, c], [d, a, b]]) == 0
    # zero first column forces a pivot search -> still exact
    assert oracle.gf_det([[0, a], [b, c]]) == oracle.gf_mul(a, b)


# splitmix64 reference outputs (Steele, Lea & Flood 2014; the public
# splitmix64.c reference generator, state advanced by 0x9E3779B97F4A7C15
# before each output).
SM_SEED0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
            0xF88BB8A8724C81EC]
SM_SEED1234567 = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                  4593380528125082431, 16408922859458223821]


def test_splitmix64_published_outputs():
    assert [oracle.sm_draw(0, i) for i in range(4)] == SM_SEED0
    assert [oracle.sm_draw(1234567, i) for i in range(5)] == SM_SEED1234567


def test_family_keys_distinct():
    keys = {oracle.family_key(7, tag) for tag in (1, 2, 3, 4)}
    assert len(keys) == 4
