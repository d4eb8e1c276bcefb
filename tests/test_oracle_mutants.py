"""The pins catch plausible mistakes in the oracle (no GPU).

Each case plants one mistake in a temporary copy of oracle/oracle.c (the
committed oracle is never modified), builds it, and checks that at least one
of the pins -- the field's closed forms, the paper's figures, the
determinant identity and its split by last edge -- fails on it, while the
unmodified copy passes them all.
"""
import ctypes
import os
import random
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_2010_08423_gb300 import workloads as W
from conftest import read_fixture

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "oracle.c")

MUTANTS = {
    "window end exclusive": ("return d >= 0 && d <= (int64_t)delta_u;",
                             "return d >= 0 && d < (int64_t)delta_u;"),
    "delta of the head": ("uint64_t w = orc_window_sum(IN, u, t[e], delta[u], prev);",
                          "uint64_t w = orc_window_sum(IN, u, t[e], delta[dst[e]], prev);"),
    "window start one late": ("orc_first_at_or_after(IN, u, (int64_t)te - (int64_t)delta_u)",
                              "orc_first_at_or_after(IN, u, (int64_t)te - (int64_t)delta_u + 1)"),
    "window start search skips equal times": ("if ((int64_t)IN->time[mid] < tmin)",
                                              "if ((int64_t)IN->time[mid] <= tmin)"),
    "time order reversed": ("int64_t d = (int64_t)te - (int64_t)tf;",
                            "int64_t d = (int64_t)tf - (int64_t)te;"),
    "y dropped at layers >= 2": ("cur[e] = w ? orc_gf_mul(orc_gf_mul(orc_y(seed, e, l), x[dst[e]]), w) : 0;",
                                 "cur[e] = w ? orc_gf_mul(x[dst[e]], w) : 0;"),
    "x_s dropped at layer 1": ("prev[e] = orc_gf_mul(orc_gf_mul(orc_y(seed, e, 1), x[s]), x[dst[e]]);",
                               "prev[e] = orc_gf_mul(orc_y(seed, e, 1), x[dst[e]]);"),
    "source not enforced": ("if (src[e] == s)\n            prev[e]",
                            "if (src[e] == src[e])\n            prev[e]"),
    "label bit shifted": ("if ((mask >> (j - 1)) & 1U)\n                acc ^= z[u * k + (j - 1)];",
                          "if ((mask >> j) & 1U)\n                acc ^= z[u * k + (j - 1)];"),
    "wrong reduction constant": ("#define ORC_POLY_LOW 0x1BULL", "#define ORC_POLY_LOW 0x1DULL"),
    "edge sums overwritten per point": ("            eout[e] ^= prev[e];", "            eout[e] = prev[e];"),
}


def _build(text, tmp, name):
    src = os.path.join(tmp, name + ".c")
    lib = os.path.join(tmp, name + ".so")
    with open(src, "w") as fh:
        fh.write(text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", lib, src],
                   check=True)
    return lib


def _pins_fail(libpath) -> list:
    """Runs the pins against the library at libpath; returns the failing ones."""
    saved = oracle._lib
    oracle._lib = None
    real_build = oracle.build
    oracle.build = lambda force=False: libpath
    failures = []
    try:
        oracle._load()
        # field closed forms
        if oracle.gf_mul(1 << 63, 2) != 0x1B or oracle.gf_mul(1 << 10, 1 << 20) != 1 << 30:
            failures.append("field")
        # figures
        for name in ("fig_restless_paths.txt", "fig_fine_grained.txt", "fig_extraction.txt",
                     "fig_random_walk.txt"):
            g, s, expect, _ = read_fixture(name)
            for k, want in expect.items():
                S = oracle.sieve(g, s, k, 3)
                if sorted(np.nonzero(S)[0].tolist()) != want:
                    failures.append("figure " + name)
                    break
        # determinant identity
        rng = random.Random(17)
        for gi in range(40):
            g = W.tiny_random(3000 + gi, n=rng.randint(3, 7), m=rng.randint(4, 16),
                              tau=rng.randint(1, 5), dmax=rng.randint(0, 3))
            s = rng.randrange(g["n"])
            k = rng.randint(2, min(5, g["n"]))
            seed = rng.getrandbits(64)
            S = oracle.sieve(g, s, k, seed)
            _, sdet, _ = oracle.dfs_paths(g, s, k, seed, with_det=True)
            if not np.array_equal(S, sdet):
                failures.append("determinant identity")
                break
        # the same identity split by last edge (fine-grained outputs)
        rng = random.Random(19)
        for gi in range(30):
            g = W.tiny_random(3100 + gi, n=rng.randint(3, 7), m=rng.randint(4, 16),
                              tau=rng.randint(1, 5), dmax=rng.randint(0, 3))
            s = rng.randrange(g["n"])
            k = rng.randint(2, min(5, g["n"]))
            seed = rng.getrandbits(64)
            _, E = oracle.sieve(g, s, k, seed, edges=True)
            _, _, _, edet, _ = oracle.dfs_paths(g, s, k, seed, with_det=True, with_edges=True)
            if not np.array_equal(E, edet):
                failures.append("edge determinant identity")
                break
    finally:
        oracle._lib = saved
        oracle.build = real_build
    return failures


@pytest.fixture(scope="module")
def tmpdir_mod():
    d = tempfile.mkdtemp(prefix="orc_mut_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


def test_unmodified_copy_passes_all_pins(tmpdir_mod):
    text = open(SRC).read()
    assert _pins_fail(_build(text, tmpdir_mod, "orig")) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmpdir_mod, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, name
    lib = _build(text.replace(old, new), tmpdir_mod, "m" + str(abs(hash(name)) % 10**8))
    assert _pins_fail(lib), f"mutant '{name}' passed every pin"
