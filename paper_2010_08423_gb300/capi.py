"""Thin ctypes binding of include/restless_reach.h (argument marshalling only).

Every function has the C entry point's name and raises ``RRError`` on a
non-OK status. Host arrays are numpy arrays; device arrays are anything with a
``data_ptr()`` (torch tensors) or raw integer addresses. All computation runs
in the CUDA library; if the library is missing or cannot be loaded this module
raises at import-time use, it never falls back to another implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

RR_OK, RR_EINVAL, RR_ENOMEM, RR_EAGAIN, RR_ETIMEDOUT, RR_ECANCELED, RR_ECUDA, RR_ENOPATH = range(8)
STATUS_NAMES = {0: "RR_OK", 1: "RR_EINVAL", 2: "RR_ENOMEM", 3: "RR_EAGAIN",
                4: "RR_ETIMEDOUT", 5: "RR_ECANCELED", 6: "RR_ECUDA", 7: "RR_ENOPATH"}
FLAG_DENSE_STATE = 1
FLAG_PAIR_ON = 2
FLAG_PAIR_OFF = 4
FLAG_HEAD_TABLE_ON = 8
FLAG_HEAD_TABLE_OFF = 16
FLAG_PAIR_TAIL_OFF = 32
FLAG_ATMOST_LANES = 64
FLAG_ATMOST_BRANCHES = 128
FLAG_K4_PER_POINT = 256
FLAG_K5_CLOSED = 512


class RRError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class rr_query(ctypes.Structure):
    _fields_ = [("source", ctypes.c_uint32), ("k", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("motif", ctypes.c_void_p)]


class rr_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("m", ctypes.c_uint64),
                ("state_rows", ctypes.c_uint64), ("window_rows", ctypes.c_uint64),
                ("max_in_degree", ctypes.c_uint32), ("num_items", ctypes.c_uint32),
                ("device_bytes", ctypes.c_uint64), ("has_colors", ctypes.c_int),
                ("compact", ctypes.c_int), ("producer_window_rows", ctypes.c_uint64),
                ("state_compute_rows", ctypes.c_uint64), ("tail_rows", ctypes.c_uint64),
                ("deep_compute_rows", ctypes.c_uint64), ("deep_tail_rows", ctypes.c_uint64),
                ("deep_head_runs", ctypes.c_uint64), ("pair_layer3_min_k", ctypes.c_int),
                ("deep_max_range_rows", ctypes.c_uint32), ("deep_heads", ctypes.c_uint32),
                ("head_table", ctypes.c_int), ("pair_tail", ctypes.c_int)]


class rr_batch_tuning(ctypes.Structure):
    _fields_ = [("blocks_per_sm", ctypes.c_uint32), ("ranges", ctypes.c_uint32),
                ("max_chunk", ctypes.c_uint32)]


class rr_kernel_times(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 9), ("launches", ctypes.c_uint64 * 9)]


TIMING_KINDS = ["first_layer", "mid_layer", "last_layer", "ztable", "batch", "second_layer",
                "tail_layer", "third_layer", "label_tail_layer"]


EXPORTED = [
    "rr_graph_load", "rr_graph_free", "rr_graph_get_info", "rr_reach_sync",
    "rr_reach_device", "rr_reach_batch_device", "rr_server_create", "rr_server_destroy",
    "rr_query_submit", "rr_query_poll", "rr_query_cancel", "rr_query_times", "rr_server_stats",
    "rr_server_set_batching",
    "rr_autotune",
    "rr_set_tuning", "rr_debug_point_sums", "rr_debug_graph", "rr_debug_ztable",
    "rr_debug_gf_mul", "rr_debug_draw", "rr_last_error", "rr_kernel_launches",
    "rr_timing_enable", "rr_timing_read", "rr_reach_device_noalloc", "rr_reach_atmost_device",
    "rr_reach_arrival_device", "rr_extract_path", "rr_reach_sources_device", "rr_bench_gf_mul",
    "rr_debug_wait_probe", "rr_reach_bounded_device", "rr_reach_range_device",
    "rr_autotune_batch", "rr_set_batch_tuning", "rr_get_batch_tuning",
]

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads librestless_reach.so (building it first if asked and needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or (build_if_missing and not _build.up_to_date()):
        if not build_if_missing:
            raise RRError(RR_ECUDA, f"CUDA library not built: {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32
    pq = ctypes.POINTER(rr_query)
    sig = {
        "rr_graph_load": [u32, u64, vp, vp, vp, vp, vp, u32, ctypes.POINTER(vp)],
        "rr_graph_free": [vp],
        "rr_graph_get_info": [vp, ctypes.POINTER(rr_graph_info)],
        "rr_reach_sync": [vp, pq, vp, vp],
        "rr_reach_device": [vp, pq, vp, vp, vp],
        "rr_reach_device_noalloc": [vp, pq, vp, vp, vp],
        "rr_reach_range_device": [vp, pq, u32, u32, vp, vp],
        "rr_reach_batch_device": [vp, pq, u32, vp, vp, vp, vp],
        "rr_reach_atmost_device": [vp, u32, u32, u64, vp, vp, vp],
        "rr_reach_bounded_device": [vp, u32, u32, u64, vp, vp, vp, vp],
        "rr_reach_arrival_device": [vp, pq, vp, vp, vp, vp, vp],
        "rr_extract_path": [vp, pq, u32, vp, vp, vp],
        "rr_bench_gf_mul": [u32, u32, u32, vp, ctypes.POINTER(u64), vp],
        "rr_debug_wait_probe": [u64, i32, ctypes.POINTER(i32), ctypes.POINTER(u64)],
        "rr_reach_sources_device": [vp, vp, u32, u32, u64, vp, vp, vp, vp, vp],
        "rr_server_create": [vp, u64, u32, ctypes.POINTER(vp)],
        "rr_server_destroy": [vp],
        "rr_query_submit": [vp, pq, ctypes.POINTER(u64)],
        "rr_query_poll": [vp, u64, i32, vp, vp],
        "rr_query_cancel": [vp, u64],
        "rr_server_stats": [vp, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64)],
        "rr_server_set_batching": [vp, u32, u32],
        "rr_query_times": [vp, u64, ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double)],
        "rr_autotune": [vp, u32, ctypes.POINTER(u32), ctypes.POINTER(u32)],
        "rr_autotune_batch": [vp, pq, u32, ctypes.POINTER(rr_batch_tuning)],
        "rr_set_batch_tuning": [vp, ctypes.POINTER(rr_batch_tuning)],
        "rr_get_batch_tuning": [vp, ctypes.POINTER(rr_batch_tuning)],
        "rr_set_tuning": [vp, u32, u32, u32],
        "rr_debug_point_sums": [vp, pq, vp, u32, vp],
        "rr_debug_graph": [vp, vp, vp, vp, vp],
        "rr_debug_ztable": [vp, pq, vp],
        "rr_debug_gf_mul": [vp, vp, vp, u64],
        "rr_debug_draw": [u64, u64, u64, vp],
        "rr_timing_enable": [ctypes.c_int],
        "rr_timing_read": [ctypes.POINTER(rr_kernel_times), ctypes.c_int],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.rr_last_error.restype = ctypes.c_char_p
    lib.rr_last_error.argtypes = []
    lib.rr_kernel_launches.restype = ctypes.c_uint64
    lib.rr_kernel_launches.argtypes = []
    _lib = lib
    return lib


def _check(st):
    if st != RR_OK:
        raise RRError(st, (_lib.rr_last_error() or b"").decode())
    return st


def _host(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def _hp(a):
    return None if a is None else a.ctypes.data


def _dp(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def make_query(source: int, k: int, seed: int, motif=None):
    """Returns (rr_query, keepalive) -- keep the second item alive during the call."""
    m = None if motif is None else np.ascontiguousarray(motif, dtype=np.uint8)
    q = rr_query(int(source), int(k), int(seed) & ((1 << 64) - 1),
                 None if m is None else m.ctypes.data)
    return q, m


# -- entry points (same names as the C ABI) ----------------------------------

def rr_graph_load(n, src, dst, t, delta, color=None, flags: int = 0):
    lib = load()
    src, dst, t = _host(src, np.uint32), _host(dst, np.uint32), _host(t, np.uint32)
    delta, color = _host(delta, np.uint32), _host(color, np.uint8)
    out = ctypes.c_void_p()
    _check(lib.rr_graph_load(int(n), int(src.shape[0]), _hp(src), _hp(dst), _hp(t), _hp(delta),
                             _hp(color), int(flags), ctypes.byref(out)))
    return out.value


def rr_graph_free(g):
    _check(load().rr_graph_free(g))


def rr_graph_get_info(g) -> dict:
    info = rr_graph_info()
    _check(load().rr_graph_get_info(g, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in rr_graph_info._fields_}


def rr_reach_sync(g, n, source, k, seed, motif=None, out=None):
    """Returns (bitmap uint8[ceil(n/8)], witness uint64[n]); `out` = a
    preallocated (bitmap, witness) pair of C-contiguous host arrays (pinned
    memory, e.g. views of pinned torch tensors, makes the copies plain DMA)."""
    q, keep = make_query(source, k, seed, motif)
    if out is None:
        bm = np.zeros((n + 7) // 8, dtype=np.uint8)
        w = np.zeros(n, dtype=np.uint64)
    else:
        bm, w = out
        if (bm.dtype != np.uint8 or w.dtype != np.uint64 or bm.shape[0] < (n + 7) // 8
                or w.shape[0] < n or not bm.flags.c_contiguous or not w.flags.c_contiguous):
            raise ValueError("rr_reach_sync: out must be (uint8[ceil(n/8)], uint64[n]) C-contiguous")
    _check(load().rr_reach_sync(g, ctypes.byref(q), _hp(bm), _hp(w)))
    del keep
    return bm, w


def rr_reach_device(g, source, k, seed, d_witness, d_bitmap=None, stream=None, motif=None):
    q, keep = make_query(source, k, seed, motif)
    _check(load().rr_reach_device(g, ctypes.byref(q), _dp(d_bitmap), _dp(d_witness),
                                  _dp(stream)))
    del keep


def rr_reach_range_device(g, source, k, seed, first, count, d_witness, stream=None, motif=None):
    """The witness part of sieve points [first, first + count) (first a
    multiple of 128); parts of disjoint ranges XOR to the full witness."""
    q, keep = make_query(source, k, seed, motif)
    _check(load().rr_reach_range_device(g, ctypes.byref(q), int(first), int(count),
                                        _dp(d_witness), _dp(stream)))
    del keep


def rr_reach_device_noalloc(g, source, k, seed, d_witness, d_bitmap=None, stream=None,
                            motif=None):
    """rr_reach_device without any device allocation (static 256 MiB scratch)."""
    q, keep = make_query(source, k, seed, motif)
    _check(load().rr_reach_device_noalloc(g, ctypes.byref(q), _dp(d_bitmap), _dp(d_witness),
                                          _dp(stream)))
    del keep


def _query_array(queries):
    arr = (rr_query * len(queries))()
    keep = []
    for i, qd in enumerate(queries):
        q, m = make_query(qd["source"], qd["k"], qd["seed"], qd.get("motif"))
        arr[i] = q
        keep.append(m)
    return arr, keep


def rr_reach_batch_device(g, queries, d_witness, d_bitmaps=None, d_status=None, stream=None):
    """queries: list of dicts with source, k, seed and optional motif."""
    arr, keep = _query_array(queries)
    _check(load().rr_reach_batch_device(g, arr, len(queries), _dp(d_bitmaps), _dp(d_witness),
                                        _dp(d_status), _dp(stream)))
    del keep


NO_ARRIVAL = 0xFFFFFFFF


def rr_reach_arrival_device(g, source, k, seed, d_witness, d_arrival, d_edge_sums=None,
                            d_bitmap=None, stream=None, motif=None):
    """Fine-grained oracle: witness (n), minimum arrival time R (n uint32,
    NO_ARRIVAL if none), optional per-edge sums (m) and bitmap of R < NO_ARRIVAL."""
    q, keep = make_query(source, k, seed, motif)
    _check(load().rr_reach_arrival_device(g, ctypes.byref(q), _dp(d_witness), _dp(d_edge_sums),
                                          _dp(d_arrival), _dp(d_bitmap), _dp(stream)))
    del keep


def rr_reach_sources_device(g, sources, k, seed, d_witness, d_bitmap=None, d_separators=None,
                            stream=None, motif=None):
    """k-RestlessReach from a set of sources, avoiding optional separators."""
    srcs = np.ascontiguousarray(sources, dtype=np.uint32)
    mo = None if motif is None else np.ascontiguousarray(motif, dtype=np.uint8)
    _check(load().rr_reach_sources_device(g, srcs.ctypes.data, int(srcs.shape[0]), int(k),
                                          int(seed) & ((1 << 64) - 1),
                                          None if mo is None else mo.ctypes.data,
                                          _dp(d_separators), _dp(d_bitmap), _dp(d_witness),
                                          _dp(stream)))


def rr_debug_wait_probe(timeout_ns: int, abort_preset: bool = False):
    """(status, elapsed_ns) of the batch kernel's bounded wait on a counter that
    nothing increments."""
    st, ns = ctypes.c_int32(), ctypes.c_uint64()
    _check(load().rr_debug_wait_probe(int(timeout_ns), 1 if abort_preset else 0, ctypes.byref(st),
                                      ctypes.byref(ns)))
    return st.value, ns.value


def rr_bench_gf_mul(blocks, threads, iters, d_sink, stream=None) -> int:
    """Enqueues the multiply-rate microbenchmark; returns the multiplications."""
    n = ctypes.c_uint64()
    _check(load().rr_bench_gf_mul(int(blocks), int(threads), int(iters), _dp(d_sink),
                                  ctypes.byref(n), _dp(stream)))
    return n.value


def rr_extract_path(g, source, k, seed, target, motif=None):
    """One optimal restless path: (vertices[k], edges[k-1], times[k-1]) as lists,
    or None if the target has no path of k vertices (RR_ENOPATH)."""
    q, keep = make_query(source, k, seed, motif)
    verts = np.zeros(k, dtype=np.uint32)
    edges = np.zeros(max(1, k - 1), dtype=np.uint32)
    times = np.zeros(max(1, k - 1), dtype=np.uint32)
    st = load().rr_extract_path(g, ctypes.byref(q), int(target), verts.ctypes.data,
                                edges.ctypes.data, times.ctypes.data)
    del keep
    if st == RR_ENOPATH:
        return None
    _check(st)
    return verts.tolist(), edges[:k - 1].tolist(), times[:k - 1].tolist()


def rr_reach_bounded_device(g, source, k, seed, d_arrival, d_length=None, d_bitmap=None,
                            stream=None):
    """Bounded RestlessReach: minimum arrival over paths of at most k vertices
    (n uint32), shortest path length in vertices (n uint8) and D."""
    _check(load().rr_reach_bounded_device(g, int(source), int(k), int(seed) & ((1 << 64) - 1),
                                          _dp(d_arrival), _dp(d_length), _dp(d_bitmap),
                                          _dp(stream)))


def rr_reach_atmost_device(g, source, k, seed, d_witness, d_bitmap=None, stream=None):
    """At most k vertices: d_witness is (k-1) x n (row k'-2 = witness of k')."""
    _check(load().rr_reach_atmost_device(g, int(source), int(k), int(seed) & ((1 << 64) - 1),
                                         _dp(d_bitmap), _dp(d_witness), _dp(stream)))


def rr_server_create(g, budget: int = 0, max_slots: int = 0):
    out = ctypes.c_void_p()
    _check(load().rr_server_create(g, int(budget), int(max_slots), ctypes.byref(out)))
    return out.value


def rr_server_destroy(s):
    _check(load().rr_server_destroy(s))


def rr_query_submit(s, source, k, seed, motif=None) -> int:
    q, keep = make_query(source, k, seed, motif)
    t = ctypes.c_uint64()
    _check(load().rr_query_submit(s, ctypes.byref(q), ctypes.byref(t)))
    del keep
    return t.value


def rr_query_poll(s, ticket, n, timeout_ms=-1):
    """Returns (status, bitmap, witness); status RR_EAGAIN means not finished."""
    bm = np.zeros((n + 7) // 8, dtype=np.uint8)
    w = np.zeros(n, dtype=np.uint64)
    st = load().rr_query_poll(s, int(ticket), int(timeout_ms), _hp(bm), _hp(w))
    if st == RR_EAGAIN:
        return st, None, None
    _check(st)
    return st, bm, w


def rr_query_cancel(s, ticket):
    _check(load().rr_query_cancel(s, int(ticket)))


def rr_query_times(s, ticket):
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().rr_query_times(s, int(ticket), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def rr_server_stats(s):
    """(queries admitted singly, queries admitted in batches, batches)."""
    a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().rr_server_stats(s, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def rr_server_set_batching(s, min_batch, max_batch):
    _check(load().rr_server_set_batching(s, int(min_batch), int(max_batch)))


def rr_autotune(g, k):
    p, c = ctypes.c_uint32(), ctypes.c_uint32()
    _check(load().rr_autotune(g, int(k), ctypes.byref(p), ctypes.byref(c)))
    return p.value, c.value


def rr_autotune_batch(g, queries) -> dict:
    """Times the persistent batch's shapes on `queries` (dicts as for
    rr_reach_batch_device), keeps the fastest in the graph and returns it."""
    arr, keep = _query_array(queries)
    t = rr_batch_tuning()
    _check(load().rr_autotune_batch(g, arr, len(queries), ctypes.byref(t)))
    del keep
    return {f: getattr(t, f) for f, _ in rr_batch_tuning._fields_}


def rr_set_batch_tuning(g, blocks_per_sm=0, ranges=0, max_chunk=0):
    t = rr_batch_tuning(int(blocks_per_sm), int(ranges), int(max_chunk))
    _check(load().rr_set_batch_tuning(g, ctypes.byref(t)))


def rr_get_batch_tuning(g) -> dict:
    t = rr_batch_tuning()
    _check(load().rr_get_batch_tuning(g, ctypes.byref(t)))
    return {f: getattr(t, f) for f, _ in rr_batch_tuning._fields_}


def rr_set_tuning(g, k, ppl, chunk):
    _check(load().rr_set_tuning(g, int(k), int(ppl), int(chunk)))


def rr_debug_point_sums(g, n, source, k, seed, masks, motif=None):
    q, keep = make_query(source, k, seed, motif)
    masks = _host(masks, np.uint32)
    out = np.zeros((masks.shape[0], n), dtype=np.uint64)
    _check(load().rr_debug_point_sums(g, ctypes.byref(q), _hp(masks), masks.shape[0], _hp(out)))
    del keep
    return out


def rr_debug_graph(g, n, m):
    off = np.zeros(n + 1, dtype=np.uint32)
    eid = np.zeros(m, dtype=np.uint32)
    lo = np.zeros(m, dtype=np.uint32)
    hi = np.zeros(m, dtype=np.uint32)
    _check(load().rr_debug_graph(g, _hp(off), _hp(eid), _hp(lo), _hp(hi)))
    return off, eid, lo, hi


def rr_debug_ztable(g, n, source, k, seed, motif=None):
    q, keep = make_query(source, k, seed, motif)
    out = np.zeros((n, k), dtype=np.uint64)
    _check(load().rr_debug_ztable(g, ctypes.byref(q), _hp(out)))
    del keep
    return out


def rr_debug_gf_mul(a, b):
    a, b = _host(a, np.uint64), _host(b, np.uint64)
    out = np.zeros_like(a)
    _check(load().rr_debug_gf_mul(_hp(a), _hp(b), _hp(out), a.shape[0]))
    return out


def rr_debug_draw(key, first, count):
    out = np.zeros(count, dtype=np.uint64)
    _check(load().rr_debug_draw(int(key), int(first), int(count), _hp(out)))
    return out


def rr_timing_enable(enable: bool):
    _check(load().rr_timing_enable(1 if enable else 0))


def rr_timing_read(reset: bool = True) -> dict:
    """{kind: (total_ms, launches)} for kinds in TIMING_KINDS."""
    t = rr_kernel_times()
    _check(load().rr_timing_read(ctypes.byref(t), 1 if reset else 0))
    return {name: (t.ms[i], int(t.launches[i])) for i, name in enumerate(TIMING_KINDS)}


def rr_last_error() -> str:
    return (load().rr_last_error() or b"").decode()


def rr_kernel_launches() -> int:
    return int(load().rr_kernel_launches())


class Graph:
    """Convenience owner of an rr_graph handle (frees it on close)."""

    def __init__(self, g: dict, flags: int = 0):
        self.n = int(g["n"])
        self.m = int(len(g["src"]))
        self.handle = rr_graph_load(self.n, g["src"], g["dst"], g["t"], g["delta"],
                                    g.get("color"), flags)

    def info(self):
        return rr_graph_get_info(self.handle)

    def reach(self, source, k, seed, motif=None, out=None):
        return rr_reach_sync(self.handle, self.n, source, k, seed, motif, out)

    def extract_path(self, source, k, seed, target, motif=None):
        return rr_extract_path(self.handle, source, k, seed, target, motif)

    def reach_range(self, source, k, seed, first, count, motif=None):
        """Witness part of sieve points [first, first + count) on the current
        CUDA device, returned as a host uint64 array."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        d_w = torch.empty(self.n, dtype=torch.int64, device=dev)
        st = torch.cuda.current_stream(dev)
        rr_reach_range_device(self.handle, source, k, seed, first, count, d_w, st.cuda_stream, motif)
        st.synchronize()
        return d_w.cpu().numpy().view(np.uint64)

    def point_sums(self, source, k, seed, masks, motif=None):
        return rr_debug_point_sums(self.handle, self.n, source, k, seed, masks, motif)

    def arrival(self, source, k, seed, motif=None):
        """Fine-grained oracle on the current CUDA device: returns host arrays
        (witness[n] uint64, edge_sums[m] uint64, arrival[n] uint32, bitmap)."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        d_w = torch.empty(self.n, dtype=torch.int64, device=dev)
        d_e = torch.empty(max(1, self.m), dtype=torch.int64, device=dev)
        d_r = torch.empty(self.n, dtype=torch.int32, device=dev)
        d_b = torch.empty((self.n + 7) // 8, dtype=torch.uint8, device=dev)
        st = torch.cuda.current_stream(dev)
        rr_reach_arrival_device(self.handle, source, k, seed, d_w, d_r, d_e, d_b,
                                st.cuda_stream, motif)
        st.synchronize()
        return (d_w.cpu().numpy().view(np.uint64), d_e.cpu().numpy().view(np.uint64)[:self.m],
                d_r.cpu().numpy().view(np.uint32), d_b.cpu().numpy())

    def close(self):
        if self.handle:
            rr_graph_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
