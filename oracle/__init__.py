"""CPU oracle for the constrained multilinear sieve (arXiv 2010.08423).

TEST INFRASTRUCTURE ONLY: the product path (the CUDA library and its Python
binding) never imports this package. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` use it.

The arithmetic lives in ``oracle.c`` (plain C, compiled here with gcc into
``oracle/_build/liborc.so``); this module only marshals numpy arrays through
ctypes. See ``oracle.c`` for the paper passages each routine follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-O2 -fopenmp) into oracle/_build/liborc.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
           "-Wextra", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u64, u32, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        vp = ctypes.c_void_p
        lib.orc_gf_mul.restype = u64
        lib.orc_gf_mul.argtypes = [u64, u64]
        lib.orc_gf_mul_many.restype = None
        lib.orc_gf_mul_many.argtypes = [vp, vp, vp, u64]
        lib.orc_gf_pow.restype = u64
        lib.orc_gf_pow.argtypes = [u64, u64]
        lib.orc_gf_inv.restype = u64
        lib.orc_gf_inv.argtypes = [u64]
        lib.orc_sm_mix.restype = u64
        lib.orc_sm_mix.argtypes = [u64]
        lib.orc_sm_draw.restype = u64
        lib.orc_sm_draw.argtypes = [u64, u64]
        lib.orc_family_key.restype = u64
        lib.orc_family_key.argtypes = [u64, u64]
        lib.orc_y.restype = u64
        lib.orc_y.argtypes = [u64, u64, u32]
        lib.orc_ztable.restype = i32
        lib.orc_ztable.argtypes = [u32, u32, u64, vp, vp, vp]
        lib.orc_sieve.restype = i32
        lib.orc_sieve.argtypes = [u32, u64, vp, vp, vp, vp, vp, vp, u32, u32, u64,
                                  vp, u32, vp, vp, vp, vp, vp, i32]
        lib.orc_gf_det.restype = u64
        lib.orc_gf_det.argtypes = [u32, vp]
        lib.orc_dfs_paths.restype = u64
        lib.orc_dfs_paths.argtypes = [u32, u64, vp, vp, vp, vp, vp, vp, u32, u32, u64,
                                      vp, vp, vp, vp, vp]
        lib.orc_max_threads.restype = i32
        lib.orc_max_threads.argtypes = []
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def _u8(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.uint8)


# -- field and PRNG --------------------------------------------------------

def gf_mul(a: int, b: int) -> int:
    return _load().orc_gf_mul(a, b)


def gf_mul_many(a, b) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    out = np.zeros_like(a)
    _load().orc_gf_mul_many(_ptr(a), _ptr(b), _ptr(out), a.shape[0])
    return out


def gf_pow(a: int, e: int) -> int:
    return _load().orc_gf_pow(a, e)


def gf_inv(a: int) -> int:
    return _load().orc_gf_inv(a)


def gf_det(mat) -> int:
    a = np.array(mat, dtype=np.uint64, copy=True)
    k = a.shape[0]
    return _load().orc_gf_det(k, _ptr(a))


def sm_mix(z: int) -> int:
    return _load().orc_sm_mix(z)


def sm_draw(key: int, i: int) -> int:
    return _load().orc_sm_draw(key, i)


def family_key(seed: int, tag: int) -> int:
    return _load().orc_family_key(seed, tag)


def y_value(seed: int, e: int, layer: int) -> int:
    return _load().orc_y(seed, e, layer)


def max_threads() -> int:
    return _load().orc_max_threads()


def ztable(n: int, k: int, seed: int, color=None, motif=None) -> np.ndarray:
    z = np.zeros((n, k), dtype=np.uint64)
    color, motif = _u8(color), _u8(motif)
    rc = _load().orc_ztable(n, k, seed, _ptr(color), _ptr(motif), _ptr(z))
    if rc:
        raise ValueError("orc_ztable: invalid arguments")
    return z


# -- sieve and brute force -------------------------------------------------

def sieve(graph, source: int, k: int, seed: int, motif=None, masks=None,
          per_mask: bool = False, threads: int = 0, edges: bool = False, deleted=None,
          sources=None):
    """Per-vertex sieve sums S (n uint64) over all 2^k points or ``masks``.

    ``graph`` is a mapping with n, src, dst, t, delta and optionally color.
    Returns S, or (S, per_mask_sums[nmasks, n]) when per_mask is True, or
    (S, E) when edges is True: E[e] (m uint64) is the sum over the points of
    the last layer's value of input edge e (Algorithm 1's fine-grained output
    before grouping by arrival time). ``deleted`` (n flags, optional) removes
    vertices from the graph (their z rows are zero). ``sources`` (a list of
    vertices, optional) starts walks at every one of them; ``source`` is then
    ignored.
    """
    n = int(graph["n"])
    src, dst, t, delta = (_u32(graph[x]) for x in ("src", "dst", "t", "delta"))
    m = src.shape[0]
    color = _u8(graph.get("color"))
    motif = _u8(motif)
    if masks is not None:
        masks = _u32(masks)
        nm = masks.shape[0]
    else:
        nm = 1 << k
    S = np.zeros(n, dtype=np.uint64)
    pm = np.zeros((nm, n), dtype=np.uint64) if per_mask else None
    E = np.zeros(m, dtype=np.uint64) if edges else None
    flags = None
    if sources is not None:
        flags = np.zeros(n, dtype=np.uint8)
        flags[np.asarray(list(sources), dtype=np.int64)] = 1
        source = 0
    rc = _load().orc_sieve(n, m, _ptr(src), _ptr(dst), _ptr(t), _ptr(delta),
                           _ptr(color), _ptr(motif), source, k, seed,
                           _ptr(masks), 0 if masks is None else nm, _ptr(S),
                           _ptr(pm), _ptr(E), _ptr(_u8(deleted)), _ptr(flags), int(threads))
    if rc == 1:
        raise ValueError("orc_sieve: invalid input")
    if rc:
        raise MemoryError("orc_sieve: allocation failed")
    if edges:
        return S, E
    return (S, pm) if per_mask else S


NO_ARRIVAL = 0xFFFFFFFF


def arrival_times(graph, E) -> np.ndarray:
    """R[v] (n uint32): the smallest time i such that the polynomial of the
    walks ending at v at time i -- the XOR of E[e] over the edges e into v with
    t_e = i -- is non-zero; NO_ARRIVAL if there is none (Algorithm 1's R)."""
    n = int(graph["n"])
    R = np.full(n, NO_ARRIVAL, dtype=np.uint32)
    for (v, ti), val in _group_sums(graph, E).items():
        if val and ti < R[v]:
            R[v] = ti
    return R


def atmost_arrival(graph, source: int, k: int, seed: int):
    """RestlessReach bounded by k (Algorithm 2 with its loop over k' stopped at
    k, R and D accumulated over the loop): R[v] (n uint32) = the minimum over
    k' = 2..k of Algorithm 1's minimum arrival time for k' vertices
    (NO_ARRIVAL if none), and L[v] (n uint8) = the smallest such k' with an
    arrival (0 if none) -- the vertex count of a shortest restless path."""
    n = int(graph["n"])
    R = np.full(n, NO_ARRIVAL, dtype=np.uint32)
    L = np.zeros(n, dtype=np.uint8)
    for kk in range(2, k + 1):
        _, E = sieve(graph, source, kk, seed, edges=True)
        Rk = arrival_times(graph, E)
        hit = Rk != NO_ARRIVAL
        L[(L == 0) & hit] = kk
        R = np.minimum(R, Rk)
    return R, L


def _group_sums(graph, E) -> dict:
    """{(v, t): XOR of E[e] over the edges e into v at time t}."""
    dst = np.asarray(graph["dst"], dtype=np.int64)
    t = np.asarray(graph["t"], dtype=np.int64)
    groups = {}
    for e in range(dst.shape[0]):
        key = (int(dst[e]), int(t[e]))
        groups[key] = groups.get(key, 0) ^ int(E[e])
    return groups


def extract_path(graph, source: int, k: int, seed: int, target: int, motif=None):
    """One optimal restless path of k vertices from source to target (Sec.
    "Extracting an optimal solution using k queries"): the last time of the path
    is the target's minimum arrival time R_target. Step l = k..2 queries the
    fine-grained oracle for l vertices on the graph without the vertices chosen
    so far (and, for motif queries, without their colours in M); the next vertex
    u is the tail of an edge (u, cur, t_cur) whose window t_cur - delta(u) <= i
    <= t_cur holds a time i with a non-zero (u, i) polynomial. Ties go to the
    earliest i, then the smallest edge index. The first edge is the smallest-
    index edge from the source at the chosen time.

    Returns (vertices[k], edges[k-1], times[k-1]) as lists, or None when the
    target has no arrival (or, with probability <= (3k-1)/2^64 per step, a
    polynomial vanished)."""
    n = int(graph["n"])
    src = np.asarray(graph["src"], dtype=np.int64)
    dst = np.asarray(graph["dst"], dtype=np.int64)
    t = np.asarray(graph["t"], dtype=np.int64)
    delta = np.asarray(graph["delta"], dtype=np.int64)
    color = graph.get("color")
    M = list(motif) if motif is not None else None
    deleted = np.zeros(n, dtype=np.uint8)
    _, E = sieve(graph, source, k, seed, motif=M, edges=True)
    R = arrival_times(graph, E)
    if R[target] == NO_ARRIVAL:
        return None
    path, times, edges = [int(target)], [int(R[target])], []
    deleted[target] = 1
    if M is not None:
        M.remove(int(color[target]))
    for ell in range(k - 1, 1, -1):
        _, E = sieve(graph, source, ell, seed, motif=M, edges=True, deleted=deleted)
        groups = _group_sums(graph, E)
        cur, tc = path[-1], times[-1]
        best = None
        for e in range(src.shape[0]):
            u = int(src[e])
            if dst[e] != cur or t[e] != tc or deleted[u]:
                continue
            for i in range(max(0, tc - int(delta[u])), tc + 1):
                if groups.get((u, i), 0):
                    if best is None or (i, e) < best:
                        best = (i, e)
                    break
        if best is None:
            return None
        i, e = best
        u = int(src[e])
        path.append(u)
        times.append(i)
        edges.append(e)
        deleted[u] = 1
        if M is not None:
            M.remove(int(color[u]))
    cur, tc = path[-1], times[-1]
    first = [e for e in range(src.shape[0]) if src[e] == source and dst[e] == cur and t[e] == tc]
    if not first:
        return None
    edges.append(min(first))
    path.append(int(source))
    path.reverse()
    edges.reverse()
    return path, [int(e) for e in edges], [int(t[e]) for e in edges]


def dfs_paths(graph, source: int, k: int, seed: int = 0, motif=None,
              with_det: bool = False, with_edges: bool = False, deleted=None):
    """Exhaustive temporal DFS over restless k-vertex paths from ``source``.

    Returns (reach[n] uint8, Sdet[n] uint64 or None, number_of_paths), and
    with_edges=True appends Edet[m] (the determinant sums split by the path's
    last edge) and arrive[n] uint32 (earliest last-edge time of a path ending at
    v, NO_ARRIVAL if none). ``deleted`` (n flags) bars vertices from every path.
    """
    n = int(graph["n"])
    src, dst, t, delta = (_u32(graph[x]) for x in ("src", "dst", "t", "delta"))
    m = src.shape[0]
    color = _u8(graph.get("color"))
    motif = _u8(motif)
    reach = np.zeros(n, dtype=np.uint8)
    sdet = np.zeros(n, dtype=np.uint64) if with_det else None
    edet = np.zeros(m, dtype=np.uint64) if with_edges else None
    arrive = np.zeros(n, dtype=np.uint32) if with_edges else None
    cnt = _load().orc_dfs_paths(n, m, _ptr(src), _ptr(dst), _ptr(t), _ptr(delta),
                                _ptr(color), _ptr(motif), source, k, seed,
                                _ptr(reach), _ptr(sdet), _ptr(edet), _ptr(arrive),
                                _ptr(_u8(deleted)))
    if cnt == (1 << 64) - 1:
        raise ValueError("orc_dfs_paths: invalid input")
    if with_edges:
        return reach, sdet, int(cnt), edet, arrive
    return reach, sdet, int(cnt)
