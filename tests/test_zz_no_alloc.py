"""rr_reach_device_noalloc, the entry point for callers that cannot allocate
device memory while serving queries (their device memory belongs to another
allocator's pool, or an allocation's device-wide synchronisation would stall
a latency-critical loop). It must give exactly what the allocating entry
point gives, also on a second call in a row that reuses the shared static
scratch left by the first.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2010_08423_gb300 import capi
from paper_2010_08423_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_twice_in_a_row():
    import torch

    torch.cuda.set_device(0)
    capi.load()
    g = W.uniform(3000, 40_000, 40, 0, 6, 424242, ncolors=3)
    n = g["n"]
    queries = [  # different k, source and kind, so the second call cannot pass on leftovers
        {"source": 0, "k": 7, "seed": 11, "motif": None},
        {"source": 1, "k": 5, "seed": 12, "motif": [int(g["color"][1]), 0, 1, 2, 1]},
    ]
    with capi.Graph(g) as G:
        stream = torch.cuda.Stream()
        for q in queries:
            want_bm, want_w = G.reach(q["source"], q["k"], q["seed"], motif=q["motif"])
            assert np.count_nonzero(want_w) > 0, q
            d_w = torch.full((n,), -1, dtype=torch.int64, device="cuda")
            d_bm = torch.full(((n + 7) // 8,), 255, dtype=torch.uint8, device="cuda")
            capi.rr_reach_device_noalloc(G.handle, q["source"], q["k"], q["seed"], d_w, d_bm,
                                         stream.cuda_stream, motif=q["motif"])
            stream.synchronize()
            got_w = d_w.cpu().numpy().view(np.uint64)
            got_bm = d_bm.cpu().numpy()
            # GF(2^64) sums are exact: the tolerance is zero
            assert np.array_equal(got_w, want_w)
            assert np.array_equal(got_bm, want_bm)


def test_noalloc_several_point_chunks_through_the_shared_array():
    """A shape with 64-point chunks (rr_set_tuning) makes a k = 9 query run 8
    chunks, each reusing the same prefix buffers inside the static array; the
    result must still equal the allocating entry point's, twice in a row."""
    import torch

    torch.cuda.set_device(0)
    capi.load()
    g = W.uniform(3000, 40_000, 40, 0, 6, 424243, ncolors=3)
    n = g["n"]
    with capi.Graph(g) as G:
        capi.rr_set_tuning(G.handle, 9, 2, 64)
        stream = torch.cuda.Stream()
        for seed in (21, 22):
            _, want_w = G.reach(2, 9, seed)
            assert np.count_nonzero(want_w) > 0
            d_w = torch.full((n,), -1, dtype=torch.int64, device="cuda")
            capi.rr_reach_device_noalloc(G.handle, 2, 9, seed, d_w, None, stream.cuda_stream)
            stream.synchronize()
            assert np.array_equal(d_w.cpu().numpy().view(np.uint64), want_w)


def test_noalloc_rejects_state_beyond_the_static_scratch():
    """A small graph (tiny z-table) whose windows cover almost every row: the
    prefix state of the smallest point chunk (2 x rows x 64 points x 8 bytes)
    does not fit the 256 MiB array."""
    import torch

    capi.load()
    g = W.uniform(1000, 400_000, 20, 5, 10, 424244)
    with capi.Graph(g) as G:
        info = G.info()
        assert 2 * info["state_rows"] * 64 * 8 > 256 << 20
        d_w = torch.zeros(g["n"], dtype=torch.int64, device="cuda")
        with pytest.raises(capi.RRError) as ei:
            capi.rr_reach_device_noalloc(G.handle, 0, 5, 1, d_w)
        assert ei.value.status == capi.RR_ENOMEM
        msg = capi.rr_last_error()
        assert "smallest point chunk (64 points)" in msg and "static scratch" in msg


def test_noalloc_rejects_queries_beyond_the_static_scratch():
    capi.load()
    # n * k * 8 bytes of z-table alone exceed the 256 MiB scratch
    n = 2_000_000
    g = {"n": n, "src": np.array([0], np.uint32), "dst": np.array([1], np.uint32),
         "t": np.array([1], np.uint32), "delta": np.ones(n, np.uint32)}
    import torch
    with capi.Graph(g) as G:
        d_w = torch.zeros(n, dtype=torch.int64, device="cuda")
        with pytest.raises(capi.RRError) as ei:
            capi.rr_reach_device_noalloc(G.handle, 0, 20, 1, d_w)
        assert ei.value.status == capi.RR_ENOMEM
        assert "static scratch" in capi.rr_last_error()
