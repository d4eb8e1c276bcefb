import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


GOLDEN = os.path.join(ROOT, "tests", "golden")


def read_arrivals(name):
    """The 'arrival k v t' lines of a fixture: {k: {v: t}}."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            f = line.split("#", 1)[0].split()
            if f and f[0] == "arrival":
                out.setdefault(int(f[1]), {})[int(f[2])] = int(f[3])
    return out


def read_paths(name):
    """The 'path k v..' and 'path_times k t..' lines: {k: (vertices, times)}."""
    verts, times = {}, {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            f = line.split("#", 1)[0].split()
            if f and f[0] == "path":
                verts[int(f[1])] = [int(x) for x in f[2:]]
            elif f and f[0] == "path_times":
                times[int(f[1])] = [int(x) for x in f[2:]]
    return {k: (verts[k], times.get(k)) for k in verts}


def read_fixture(name):
    """Graph plus the 'source', 'expect k v...' and 'motif' lines of a fixture."""
    from paper_2010_08423_gb300.workloads import load_edge_fixture
    path = os.path.join(GOLDEN, name)
    g = load_edge_fixture(path)
    source, expect, motif = None, {}, None
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            f = line.split()
            if f[0] == "source":
                source = int(f[1])
            elif f[0] == "expect":
                expect[int(f[1])] = sorted(int(x) for x in f[2:])
            elif f[0] == "motif":
                motif = [int(x) for x in f[1:]]
    return g, source, expect, motif


def walk_start_sources(g, k):
    """Vertices with an out-edge that starts some restless walk of k-1 edges
    (edge f may follow edge e when f leaves e's head v with t_e <= t_f <=
    t_e + delta(v)): the only sources from which a k-vertex path can exist.
    Plain boolean reachability over edges; candidates, to be confirmed by DFS."""
    import numpy as np
    src = np.asarray(g["src"], dtype=np.int64)
    dst = np.asarray(g["dst"], dtype=np.int64)
    t = np.asarray(g["t"], dtype=np.int64)
    d = np.asarray(g["delta"], dtype=np.int64)
    m = src.shape[0]
    order = np.lexsort((np.arange(m), t, src))  # out-edges by (tail, time)
    key = src[order] * (1 << 32) + t[order]
    lo = np.searchsorted(key, dst * (1 << 32) + t, side="left")
    hi = np.searchsorted(key, dst * (1 << 32) + t + d[dst], side="right")
    ok = np.ones(m, dtype=bool)  # e starts a walk of 1 edge
    for _ in range(k - 2):
        pre = np.concatenate([[0], np.cumsum(ok[order].astype(np.int64))])
        ok = (pre[hi] - pre[lo]) > 0
    return np.unique(src[ok])
