"""GPU tests of the batched persistent launch and the serving loop.

Both must reproduce, bit for bit, what one query alone gives (and the CPU
oracle): the batch packs queries of uneven k, sources and motifs into one
persistent kernel; the server runs queries that arrive while others are on the
GPU. GF(2^64) sums are exact, so the tolerance is zero.
"""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2010_08423_gb300 import capi
from paper_2010_08423_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mixed():
    capi.load()
    oracle.build()
    g = W.uniform(3000, 40_000, 40, 0, 6, 424242, ncolors=3)
    rng = np.random.default_rng(9)
    qs = []
    for i, k in enumerate([2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 5, 8, 4, 3, 9]):
        s = int(rng.integers(0, 8))
        motif = None
        if i % 2 == 1:
            motif = [int(g["color"][s])] + [int(x) for x in rng.integers(0, 3, k - 1)]
        qs.append({"source": s, "k": k, "seed": int(rng.integers(0, 2**62)), "motif": motif})
    return g, qs


def _torch():
    import torch
    torch.cuda.set_device(0)
    return torch


def test_every_batch_shape_and_the_autotuned_one_match_single_queries(mixed):
    """The persistent batch in each forced shape (kernel variant with 2, 4, 5 or 6
    blocks per SM, fine or coarse ranges, 128/512/1024-point chunks) and in the
    shape rr_autotune_batch picks gives the single queries' sums bit for bit."""
    torch = _torch()
    g, qs = mixed
    n = g["n"]
    with capi.Graph(g) as G:
        singles = np.stack([G.reach(q["source"], q["k"], q["seed"], motif=q["motif"])[1] for q in qs])
        stream = torch.cuda.Stream()
        d_w = torch.empty((len(qs), n), dtype=torch.int64, device="cuda")
        d_st = torch.empty((len(qs),), dtype=torch.int32, device="cuda")
        shapes = [(mb, rg, mc) for mb in (2, 4, 5, 6) for rg in (1, 2) for mc in (128, 512, 1024)]
        for mb, rg, mc in shapes:
            capi.rr_set_batch_tuning(G.handle, mb, rg, mc)
            assert capi.rr_get_batch_tuning(G.handle) == {"blocks_per_sm": mb, "ranges": rg,
                                                          "max_chunk": mc}
            d_w.fill_(-1)
            capi.rr_reach_batch_device(G.handle, qs, d_w, None, d_st, stream.cuda_stream)
            stream.synchronize()
            assert (d_st.cpu().numpy() == 0).all()
            assert np.array_equal(d_w.cpu().numpy().view(np.uint64), singles), (mb, rg, mc)
        best = capi.rr_autotune_batch(G.handle, qs)
        assert best["blocks_per_sm"] in (2, 4, 5, 6) and best["ranges"] in (1, 2)
        assert best["max_chunk"] in (256, 512, 1024)
        assert capi.rr_get_batch_tuning(G.handle) == best
        d_w.fill_(-1)
        capi.rr_reach_batch_device(G.handle, qs, d_w, None, d_st, stream.cuda_stream)
        stream.synchronize()
        assert np.array_equal(d_w.cpu().numpy().view(np.uint64), singles)
        for bad in ((3, 0, 0), (0, 3, 0), (0, 0, 64)):
            with pytest.raises(capi.RRError) as ei:
                capi.rr_set_batch_tuning(G.handle, *bad)
            assert ei.value.status == capi.RR_EINVAL


def test_batch_matches_single_queries_and_oracle(mixed):
    torch = _torch()
    g, qs = mixed
    n = g["n"]
    nb = (n + 7) // 8
    with capi.Graph(g) as G:
        singles = [G.reach(q["source"], q["k"], q["seed"], motif=q["motif"]) for q in qs]
        d_w = torch.full((len(qs), n), -1, dtype=torch.int64, device="cuda")
        d_bm = torch.full((len(qs), nb), 255, dtype=torch.uint8, device="cuda")
        d_st = torch.full((len(qs),), 7, dtype=torch.int32, device="cuda")
        stream = torch.cuda.Stream()
        capi.rr_reach_batch_device(G.handle, qs, d_w, d_bm, d_st, stream.cuda_stream)
        stream.synchronize()
        w = d_w.cpu().numpy().view(np.uint64)
        bm = d_bm.cpu().numpy()
        assert (d_st.cpu().numpy() == 0).all()
        nonzero = 0
        for i, q in enumerate(qs):
            assert np.array_equal(w[i], singles[i][1]), (i, q["k"])
            assert np.array_equal(bm[i], singles[i][0]), i
            nonzero += np.count_nonzero(w[i]) > 0
        assert nonzero >= 8
        for i in (1, 4, 7, 9):
            q = qs[i]
            assert np.array_equal(w[i], oracle.sieve(g, q["source"], q["k"], q["seed"],
                                                     motif=q["motif"]))
        # a second batch on the same graph reuses the batch buffers
        capi.rr_reach_batch_device(G.handle, qs[::-1], d_w, None, None, stream.cuda_stream)
        stream.synchronize()
        w2 = d_w.cpu().numpy().view(np.uint64)
        for i, q in enumerate(qs[::-1]):
            assert np.array_equal(w2[i], singles[len(qs) - 1 - i][1])


def test_batch_many_small_queries():
    torch = _torch()
    g = W.uniform(1500, 20_000, 25, 0, 5, 77, ncolors=2)
    rng = np.random.default_rng(3)
    qs = [{"source": int(rng.integers(0, 1500)), "k": int(rng.integers(4, 9)),
           "seed": i + 1, "motif": None} for i in range(96)]
    with capi.Graph(g) as G:
        d_w = torch.zeros((len(qs), g["n"]), dtype=torch.int64, device="cuda")
        capi.rr_reach_batch_device(G.handle, qs, d_w)
        torch.cuda.synchronize()
        w = d_w.cpu().numpy().view(np.uint64)
        for i in range(0, len(qs), 7):
            _, ref = G.reach(qs[i]["source"], qs[i]["k"], qs[i]["seed"])
            assert np.array_equal(w[i], ref), i


def test_server_result_alone_equals_result_in_mix(mixed):
    g, qs = mixed
    n = g["n"]
    with capi.Graph(g) as G:
        srv = capi.rr_server_create(G.handle, 0, 4)
        try:
            probe = qs[9]
            t = capi.rr_query_submit(srv, probe["source"], probe["k"], probe["seed"], probe["motif"])
            st, bm_alone, w_alone = capi.rr_query_poll(srv, t, n, -1)
            assert st == capi.RR_OK
            # the same query again, submitted while a stream of others arrives
            tickets = []
            for i, q in enumerate(qs * 2):
                tickets.append((i % len(qs), capi.rr_query_submit(srv, q["source"], q["k"],
                                                                   q["seed"], q["motif"])))
                if i == 5:
                    t_mix = capi.rr_query_submit(srv, probe["source"], probe["k"],
                                                 probe["seed"], probe["motif"])
            st, bm_mix, w_mix = capi.rr_query_poll(srv, t_mix, n, -1)
            assert st == capi.RR_OK
            assert np.array_equal(w_mix, w_alone) and np.array_equal(bm_mix, bm_alone)
            for qi, t in tickets:
                st, _, w = capi.rr_query_poll(srv, t, n, -1)
                assert st == capi.RR_OK
                _, ref = G.reach(qs[qi]["source"], qs[qi]["k"], qs[qi]["seed"], motif=qs[qi]["motif"])
                assert np.array_equal(w, ref), qi
                q_us, tot_us = capi.rr_query_times(srv, t)
                assert 0 <= q_us <= tot_us
        finally:
            capi.rr_server_destroy(srv)


def test_server_backlog_goes_through_batch_lanes(mixed):
    """With batching turned on, a burst of queued queries is admitted in batches
    (persistent kernel) and every result still equals the single-query result;
    a query cancelled in the middle of the burst ends cancelled, the others are
    unaffected."""
    g, qs = mixed
    n = g["n"]
    burst = (qs * 6)[:90]
    with capi.Graph(g) as G:
        srv = capi.rr_server_create(G.handle, 0, 2)
        try:
            capi.rr_server_set_batching(srv, 8, 64)
            ts = [capi.rr_query_submit(srv, q["source"], q["k"], q["seed"], q["motif"])
                  for q in burst]
            capi.rr_query_cancel(srv, ts[45])
            for i, (q, t) in enumerate(zip(burst, ts)):
                if i == 45:
                    with pytest.raises(capi.RRError) as ei:
                        capi.rr_query_poll(srv, t, n, -1)
                    assert ei.value.status == capi.RR_ECANCELED
                    continue
                st, bm, w = capi.rr_query_poll(srv, t, n, -1)
                assert st == capi.RR_OK
                bm_ref, w_ref = G.reach(q["source"], q["k"], q["seed"], motif=q["motif"])
                assert np.array_equal(w, w_ref) and np.array_equal(bm, bm_ref), i
            single, batched, batches = capi.rr_server_stats(srv)
            assert batched >= 8 and batches >= 1 and single + batched <= len(burst)
            # a lone query afterwards takes a slot again
            st, _, w = capi.rr_query_poll(srv, capi.rr_query_submit(srv, 3, 7, 77), n, -1)
            assert np.array_equal(w, G.reach(3, 7, 77)[1])
            assert capi.rr_server_stats(srv)[0] == single + 1
        finally:
            capi.rr_server_destroy(srv)


def test_server_batching_switch():
    g = W.uniform(2000, 20_000, 30, 0, 5, 8)
    n = g["n"]
    with capi.Graph(g) as G:
        srv = capi.rr_server_create(G.handle, 0, 2)
        try:
            for bad in ((1, 4), (9, 8), (8, 100_000)):
                with pytest.raises(capi.RRError) as ei:
                    capi.rr_server_set_batching(srv, *bad)
                assert ei.value.status == capi.RR_EINVAL
            # off by default: a burst takes the slots
            ts = [capi.rr_query_submit(srv, i % 50, 5 + i % 4, i) for i in range(40)]
            ws = [capi.rr_query_poll(srv, t, n, -1)[2] for t in ts]
            assert capi.rr_server_stats(srv) == (40, 0, 0)
            capi.rr_server_set_batching(srv, 8, 64)
            capi.rr_server_set_batching(srv, 0, 0)  # off again: every query takes a slot
            ts = [capi.rr_query_submit(srv, i % 50, 5 + i % 4, i) for i in range(40)]
            for w, t in zip(ws, ts):
                assert np.array_equal(capi.rr_query_poll(srv, t, n, -1)[2], w)
            assert capi.rr_server_stats(srv) == (80, 0, 0)
            capi.rr_server_set_batching(srv, 2, 256)  # on again, every backlog of 2
            ts = [capi.rr_query_submit(srv, i % 50, 5 + i % 4, i) for i in range(40)]
            for w, t in zip(ws, ts):
                assert np.array_equal(capi.rr_query_poll(srv, t, n, -1)[2], w)
            single, batched, batches = capi.rr_server_stats(srv)
            assert single + batched == 120 and batched >= 2 and batches >= 1
        finally:
            capi.rr_server_destroy(srv)


def test_server_cancel_and_admission():
    g = W.uniform(2000, 20_000, 30, 0, 5, 5)
    with capi.Graph(g) as G:
        srv = capi.rr_server_create(G.handle, 0, 1)
        try:
            ts = [capi.rr_query_submit(srv, 0, 12, i) for i in range(6)]
            capi.rr_query_cancel(srv, ts[-1])
            st, _, _ = capi.rr_query_poll(srv, ts[0], g["n"], -1)
            assert st == capi.RR_OK
            with pytest.raises(capi.RRError) as ei:
                capi.rr_query_poll(srv, ts[-1], g["n"], -1)
            assert ei.value.status == capi.RR_ECANCELED
            for t in ts[1:-1]:
                st, _, _ = capi.rr_query_poll(srv, t, g["n"], -1)
                assert st == capi.RR_OK
        finally:
            capi.rr_server_destroy(srv)
        # a budget too small for even one point chunk refuses the server
        with pytest.raises(capi.RRError) as ei:
            capi.rr_server_create(G.handle, 1 << 10, 1)
        assert ei.value.status == capi.RR_ENOMEM


def test_atmost_k_union_and_rows():
    """at-most-k (Algorithm 2 stopped at k): union of the exact-k' reach sets for
    k' = 2..k, each row equal to the single query's witness and the oracle's."""
    torch = _torch()
    g = W.uniform(1500, 20_000, 20, 0, 5, 66)
    n = g["n"]
    k = 6
    with capi.Graph(g) as G:
        d_w = torch.zeros((k - 1, n), dtype=torch.int64, device="cuda")
        d_bm = torch.zeros((n + 7) // 8, dtype=torch.uint8, device="cuda")
        capi.rr_reach_atmost_device(G.handle, 3, k, 99, d_w, d_bm)
        torch.cuda.synchronize()
        w = d_w.cpu().numpy().view(np.uint64)
        bm = d_bm.cpu().numpy()
        union = np.zeros(n, dtype=bool)
        for kk in range(2, k + 1):
            ref = oracle.sieve(g, 3, kk, 99)
            assert np.array_equal(w[kk - 2], ref), kk
            reach, _, _ = oracle.dfs_paths(g, 3, kk)
            assert np.array_equal(ref != 0, reach.astype(bool))
            union |= reach.astype(bool)
        got = np.array([(bm[v >> 3] >> (v & 7)) & 1 for v in range(n)], dtype=bool)
        assert union.any() and np.array_equal(got, union)


def test_atmost_lanes_reused_across_k():
    """Successive at-most calls with different k reuse the concurrent lanes
    (lane j runs k' = k - j), so each lane meets several query sizes; every row
    must equal the single query's witness."""
    torch = _torch()
    g = W.uniform(2500, 30_000, 25, 0, 6, 67, ncolors=2)
    n = g["n"]
    with capi.Graph(g) as G:
        st = torch.cuda.Stream()
        for k, s, seed in ((8, 2, 5), (3, 7, 6), (10, 1, 7), (5, 2, 8)):
            d_w = torch.full((k - 1, n), -1, dtype=torch.int64, device="cuda")
            d_bm = torch.zeros((n + 7) // 8, dtype=torch.uint8, device="cuda")
            capi.rr_reach_atmost_device(G.handle, s, k, seed, d_w, d_bm, st.cuda_stream)
            st.synchronize()
            w = d_w.cpu().numpy().view(np.uint64)
            union = np.zeros(n, dtype=bool)
            for kk in range(2, k + 1):
                _, ref = G.reach(s, kk, seed)
                assert np.array_equal(w[kk - 2], ref), (k, kk)
                union |= ref != 0
            bm = d_bm.cpu().numpy()
            got = np.unpackbits(bm, bitorder="little")[:n].astype(bool)
            assert np.array_equal(got, union), k
            assert union.sum() > 10


def test_large_batch_coarse_ranges_equal_single_queries():
    """A batch large enough to run on the coarse scheduling ranges (about 32
    entries a task) and the high-occupancy kernel variant: 64 mixed queries on
    the n = 1e5, m = 1e6 graph, every row equal to the single query's."""
    torch = _torch()
    g = W.scale_uniform(ncolors=8)
    qs = W.query_set(g, 64, 7, 11, 0x5EED0004, colored_every_other=True)
    n = g["n"]
    with capi.Graph(g) as G:
        d_w = torch.zeros((len(qs), n), dtype=torch.int64, device="cuda")
        capi.rr_reach_batch_device(G.handle, qs, d_w)
        torch.cuda.synchronize()
        w = d_w.cpu().numpy().view(np.uint64)
        for i, q in enumerate(qs):
            _, ref = G.reach(q["source"], q["k"], q["seed"], motif=q["motif"])
            assert np.array_equal(w[i], ref), (i, q["k"])


def test_calls_on_different_streams_are_ordered_on_the_graphs_scratch():
    """Calls that reuse the graph's scratch may be issued on different streams:
    each waits on the device for the previous one. Batches and single queries
    alternate over two streams without host synchronisation in between; every
    result must equal the single query's."""
    torch = _torch()
    g = W.uniform(3000, 40_000, 40, 0, 6, 31, ncolors=2)
    n = g["n"]
    qa = W.query_set(g, 24, 5, 10, 0x5EED0031, colored_every_other=True)
    qb = W.query_set(g, 24, 5, 10, 0x5EED0032, colored_every_other=True)
    with capi.Graph(g) as G:
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        wa = torch.zeros((len(qa), n), dtype=torch.int64, device="cuda")
        wb = torch.zeros((len(qb), n), dtype=torch.int64, device="cuda")
        w1 = torch.zeros(n, dtype=torch.int64, device="cuda")
        w2 = torch.zeros(n, dtype=torch.int64, device="cuda")
        capi.rr_reach_batch_device(G.handle, qa, wa, None, None, s1.cuda_stream)
        capi.rr_reach_device(G.handle, 3, 9, 77, w1, None, s2.cuda_stream)
        capi.rr_reach_batch_device(G.handle, qb, wb, None, None, s2.cuda_stream)
        capi.rr_reach_device(G.handle, 5, 8, 78, w2, None, s1.cuda_stream)
        torch.cuda.synchronize()
        for rows, qs in ((wa, qa), (wb, qb)):
            got = rows.cpu().numpy().view(np.uint64)
            for i, q in enumerate(qs):
                _, ref = G.reach(q["source"], q["k"], q["seed"], motif=q["motif"])
                assert np.array_equal(got[i], ref), i
        _, r1 = G.reach(3, 9, 77)
        _, r2 = G.reach(5, 8, 78)
        assert np.array_equal(w1.cpu().numpy().view(np.uint64), r1)
        assert np.array_equal(w2.cpu().numpy().view(np.uint64), r2)
