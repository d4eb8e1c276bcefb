"""Seeded synthetic temporal graphs and query sets.

This module only draws inputs (edges, timestamps, waiting times, colours,
sources, seeds); it holds none of the sieve's arithmetic, and is the one
module that both the CUDA path's tests/benchmarks and the CPU oracle's tests
take their inputs from.

The paper's real-world datasets (socio-patterns, KONECT, Copenhagen study,
public transport) are not available; these generators stand in for them with
the shapes of the paper's synthetic workloads (Sec. "Experimental setup":
power-law and uniform temporal graphs, uniform timestamps, per-vertex waiting
times):

  uniform(n, m, tau, dmin, dmax)  u, v uniform, self-loops resampled,
                                  t ~ U[1, tau], delta(v) ~ U{dmin..dmax}
  chung_lu(n, m, gamma, ...)      endpoints drawn independently with
                                  probability proportional to
                                  w_i = (i+1)^(-1/(gamma-1)), self-loops resampled
  burst_times(m, tau, ...)        B ~ Poisson(rate) burst centres ~ U[1, tau],
                                  each edge picks a burst and adds U{0..width-1},
                                  clamped to tau
"""
from __future__ import annotations

import numpy as np

GRAPH_SEED_BASE = 0x5EED0000


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _resample_self_loops(rng, src, dst, draw):
    bad = np.nonzero(src == dst)[0]
    while bad.size:
        dst[bad] = draw(bad.size)
        bad = bad[src[bad] == dst[bad]]
    return dst


def uniform(n: int, m: int, tau: int, dmin: int, dmax: int, seed: int,
            ncolors: int = 0) -> dict:
    """Uniform random directed temporal multigraph (no self-loops)."""
    rng = _rng(seed)
    src = rng.integers(0, n, size=m, dtype=np.uint32)
    dst = rng.integers(0, n, size=m, dtype=np.uint32)
    dst = _resample_self_loops(rng, src, dst,
                               lambda c: rng.integers(0, n, size=c, dtype=np.uint32))
    t = rng.integers(1, tau + 1, size=m, dtype=np.uint32)
    delta = rng.integers(dmin, dmax + 1, size=n, dtype=np.uint32)
    g = {"n": n, "src": src, "dst": dst, "t": t, "delta": delta}
    if ncolors:
        g["color"] = rng.integers(0, ncolors, size=n, dtype=np.uint8)
    return g


def _weighted_vertices(rng, cdf, count):
    return np.searchsorted(cdf, rng.random(count), side="right").astype(np.uint32)


def burst_times(rng, m: int, tau: int, rate: float, width: int) -> np.ndarray:
    nb = max(1, int(rng.poisson(rate)))
    centres = rng.integers(1, tau + 1, size=nb)
    pick = rng.integers(0, nb, size=m)
    t = centres[pick] + rng.integers(0, width, size=m)
    return np.minimum(t, tau).astype(np.uint32)


def chung_lu(n: int, m: int, gamma: float, tau: int, dmin: int, dmax: int,
             seed: int, ncolors: int = 0, bursts: tuple | None = None) -> dict:
    """Chung-Lu power-law temporal multigraph with degree exponent ``gamma``."""
    rng = _rng(seed)
    w = np.power(np.arange(1, n + 1, dtype=np.float64), -1.0 / (gamma - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    cdf[-1] = 1.0
    src = _weighted_vertices(rng, cdf, m)
    dst = _weighted_vertices(rng, cdf, m)
    dst = _resample_self_loops(rng, src, dst,
                               lambda c: _weighted_vertices(rng, cdf, c))
    if bursts is None:
        t = rng.integers(1, tau + 1, size=m, dtype=np.uint32)
    else:
        t = burst_times(rng, m, tau, *bursts)
    delta = rng.integers(dmin, dmax + 1, size=n, dtype=np.uint32)
    g = {"n": n, "src": src, "dst": dst, "t": t, "delta": delta}
    if ncolors:
        g["color"] = rng.integers(0, ncolors, size=n, dtype=np.uint8)
    return g


# -- the five workload shapes (graph seed = GRAPH_SEED_BASE + index) -------

def small_uniform(seed_index: int = 1) -> dict:
    """n=1,000, m=10,000, t ~ U[1,100], delta ~ U{1..5}; queried at s=0, k=5."""
    return uniform(1000, 10_000, 100, 1, 5, GRAPH_SEED_BASE + seed_index)


def scale_uniform(seed_index: int = 2, ncolors: int = 0) -> dict:
    """n=100,000, m=1,000,000, t ~ U[1,1000], delta ~ U{1..20}; s=0, k=8."""
    return uniform(100_000, 1_000_000, 1000, 1, 20, GRAPH_SEED_BASE + seed_index,
                   ncolors=ncolors)


def motif_powerlaw(seed_index: int = 3) -> dict:
    """Chung-Lu exponent 2.5, n=1e6, m=1e7, bursty t in [1,10000] (Poisson(50)
    bursts of width 20), delta ~ U{5..50}, 8 colours."""
    return chung_lu(1_000_000, 10_000_000, 2.5, 10_000, 5, 50,
                    GRAPH_SEED_BASE + seed_index, ncolors=8, bursts=(50, 20))


def served_powerlaw(seed_index: int = 5, scale: int = 1) -> dict:
    """Chung-Lu exponent 2.3, n=1e7, m=1e8, t ~ U[1,1e5], delta ~ U{10..200};
    scale > 1 divides n and m by it (same generator, seed and time ranges)."""
    return chung_lu(10_000_000 // scale, 100_000_000 // scale, 2.3, 100_000, 10, 200,
                    GRAPH_SEED_BASE + seed_index)


def first_source(g: dict) -> int:
    """Smallest vertex id with out-degree >= 1."""
    return int(np.min(g["src"]))


def motif_for(g: dict, source: int, k: int, seed: int, ncolors: int = 8) -> np.ndarray:
    """Motif multiset of k colours: the source's colour plus k-1 uniform colours."""
    rng = _rng(seed)
    rest = rng.integers(0, ncolors, size=k - 1, dtype=np.uint8)
    return np.concatenate([np.array([g["color"][source]], dtype=np.uint8), rest])


def query_set(g: dict, count: int, kmin: int, kmax: int, graph_seed: int,
              colored_every_other: bool = True, ncolors: int = 8) -> list:
    """Queries q = 0..count-1: s ~ U, k ~ U{kmin..kmax}, seed = graph_seed ^ (q+1);
    odd q carry a motif (source colour + k-1 uniform colours) when the graph has
    colours and ``colored_every_other``."""
    rng = _rng(graph_seed ^ 0xA5A5)
    out = []
    for q in range(count):
        s = int(rng.integers(0, g["n"]))
        k = int(rng.integers(kmin, kmax + 1))
        seed = (graph_seed ^ (q + 1)) & ((1 << 64) - 1)
        motif = None
        if colored_every_other and (q % 2 == 1) and "color" in g:
            motif = motif_for(g, s, k, seed, ncolors)
        out.append({"source": s, "k": k, "seed": seed, "motif": motif})
    return out


def tiny_random(seed: int, n: int = 7, m: int = 18, tau: int = 6, dmax: int = 3,
                ncolors: int = 0) -> dict:
    """Tiny random temporal multigraph for brute-force checks."""
    rng = _rng(seed)
    src = rng.integers(0, n, size=m, dtype=np.uint32)
    dst = rng.integers(0, n, size=m, dtype=np.uint32)
    dst = _resample_self_loops(rng, src, dst,
                               lambda c: rng.integers(0, n, size=c, dtype=np.uint32))
    t = rng.integers(1, tau + 1, size=m, dtype=np.uint32)
    delta = rng.integers(0, dmax + 1, size=n, dtype=np.uint32)
    g = {"n": n, "src": src, "dst": dst, "t": t, "delta": delta}
    if ncolors:
        g["color"] = rng.integers(0, ncolors, size=n, dtype=np.uint8)
    return g


def load_edge_fixture(path: str) -> dict:
    """Reads a small text fixture: 'n N', 'delta d0 d1 ...', 'edge u v t' lines,
    optional 'color c0 c1 ...'; vertices are 0-based in the file."""
    n = None
    delta = None
    color = None
    src, dst, t = [], [], []
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            f = line.split()
            if f[0] == "n":
                n = int(f[1])
            elif f[0] == "delta":
                delta = [int(x) for x in f[1:]]
            elif f[0] == "color":
                color = [int(x) for x in f[1:]]
            elif f[0] == "edge":
                src.append(int(f[1]))
                dst.append(int(f[2]))
                t.append(int(f[3]))
    g = {"n": n, "src": np.array(src, dtype=np.uint32),
         "dst": np.array(dst, dtype=np.uint32), "t": np.array(t, dtype=np.uint32),
         "delta": np.array(delta, dtype=np.uint32)}
    if color is not None:
        g["color"] = np.array(color, dtype=np.uint8)
    return g
