"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Every comparison is bit-exact (GF(2^64) arithmetic has no rounding): field
multiply, splitmix64 draws, graph windows, z-tables, per-vertex witness sums
and single-point sums, on the paper's figures, random tiny graphs, workloads
spanning many scheduling ranges with ragged tails, hubs, and (sampled) the
full-size n=100,000 / m=1,000,000 workload the benchmark times.
"""
import numpy as np
import pytest

import oracle
from paper_2010_08423_gb300 import capi
from paper_2010_08423_gb300 import workloads as W
from conftest import read_fixture

pytestmark = pytest.mark.gpu

FIXTURES = ["fig_restless_paths.txt", "fig_fine_grained.txt", "fig_extraction.txt",
            "fig_random_walk.txt"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    capi.load()
    oracle.build()


def _graph(g, flags=0):
    return capi.Graph(g, flags)


def test_device_gf_mul_matches_oracle():
    rng = np.random.default_rng(1)
    a = rng.integers(0, 2**63, size=2_000_000, dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=2_000_000, dtype=np.uint64)
    b = rng.integers(0, 2**63, size=2_000_000, dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=2_000_000, dtype=np.uint64)
    a[:1000] = np.uint64(2**64 - 1)
    b[500:1500] = np.uint64(2**64 - 1)
    a[2000:2100] = 0
    assert np.array_equal(capi.rr_debug_gf_mul(a, b), oracle.gf_mul_many(a, b))


def test_device_draws_match_oracle():
    for key in (0, 1234567, 0xDEADBEEFCAFEF00D):
        dev = capi.rr_debug_draw(key, 5, 1000)
        ref = np.array([oracle.sm_draw(key, 5 + i) for i in range(1000)], dtype=np.uint64)
        assert np.array_equal(dev, ref)


def test_graph_windows_follow_the_definition():
    g = W.tiny_random(3, n=50, m=600, tau=20, dmax=4)
    with _graph(g) as G:
        off, eid, lo, hi = capi.rr_debug_graph(G.handle, G.n, G.m)
    src, dst, t, delta = g["src"], g["dst"], g["t"], g["delta"]
    # rows sorted by (head, time, edge index)
    order = np.lexsort((np.arange(G.m), t, dst))
    assert np.array_equal(eid, order)
    assert np.array_equal(off, np.searchsorted(dst[order], np.arange(G.n + 1)))
    for r in range(G.m):
        e = eid[r]
        u = src[e]
        rows = np.arange(off[u], off[u + 1])
        f = eid[rows]
        inside = (t[f].astype(np.int64) <= t[e]) & (t[e] <= t[f].astype(np.int64) + delta[u])
        want = rows[inside]
        got = np.arange(lo[r], hi[r])
        assert np.array_equal(want, got), r


@pytest.mark.parametrize("colored", [False, True])
def test_ztable_matches_oracle(colored):
    g = W.tiny_random(4, n=300, m=100, ncolors=5)
    motif = [2, 2, 0, 4, 1, 2] if colored else None
    with _graph(g) as G:
        dev = capi.rr_debug_ztable(G.handle, G.n, 7, 6, 99, motif)
    ref = oracle.ztable(300, 6, 99, g["color"], motif)
    assert np.array_equal(dev, ref)


@pytest.mark.parametrize("name", FIXTURES)
def test_figures(name):
    g, s, expect, motif = read_fixture(name)
    with _graph(g) as G:
        for k, want in expect.items():
            for seed in (1, 2):
                bm, w = G.reach(s, k, seed)
                assert np.array_equal(w, oracle.sieve(g, s, k, seed)), (k, seed)
                got = [v for v in range(G.n) if (bm[v >> 3] >> (v & 7)) & 1]
                assert got == want
        if motif is not None:
            _, w = G.reach(s, 6, 5, motif=motif)
            assert np.array_equal(w, oracle.sieve(g, s, 6, 5, motif=motif))
            assert np.nonzero(w)[0].tolist() == [5]


def test_random_tiny_plain_and_colored():
    rng = np.random.default_rng(5)
    for gi in range(60):
        ncol = int(rng.integers(1, 4))
        g = W.tiny_random(900 + gi, n=int(rng.integers(3, 9)), m=int(rng.integers(1, 25)),
                          tau=int(rng.integers(1, 7)), dmax=int(rng.integers(0, 4)),
                          ncolors=ncol)
        with _graph(g) as G:
            for k in range(2, 7):
                s = int(rng.integers(0, g["n"]))
                seed = int(rng.integers(0, 2**63))
                _, w = G.reach(s, k, seed)
                assert np.array_equal(w, oracle.sieve(g, s, k, seed)), (gi, k)
                motif = [int(g["color"][s])] + [int(x) for x in rng.integers(0, ncol + 1, k - 1)]
                _, w = G.reach(s, k, seed, motif=motif)
                assert np.array_equal(w, oracle.sieve(g, s, k, seed, motif=motif)), (gi, k)


def _dense_uniform(n, m, tau, dmax, seed, ncolors=0):
    return W.uniform(n, m, tau, 0, dmax, seed, ncolors=ncolors)


@pytest.mark.parametrize("flags", [0, capi.FLAG_DENSE_STATE])
def test_many_ranges_ragged_full_witness(flags):
    # n=2,000 and m=30,011 (ragged), tight time range: long restless walks exist
    # and the windows span many scheduling ranges.
    g = _dense_uniform(2000, 30_011, 40, 6, 11, ncolors=3)
    with _graph(g, flags) as G:
        for s, k, seed in ((0, 5, 1), (17, 6, 2), (1999, 7, 3)):
            _, w = G.reach(s, k, seed)
            ref = oracle.sieve(g, s, k, seed)
            assert np.array_equal(w, ref), (s, k)
            assert np.count_nonzero(ref) > 0
        motif = [int(g["color"][5]), 0, 1, 2, 1]
        _, w = G.reach(5, 5, 9, motif=motif)
        assert np.array_equal(w, oracle.sieve(g, 5, 5, 9, motif=motif))


def test_hub_segments_and_bursts():
    # Chung-Lu graph: hub in-segments of hundreds of rows (own scheduling range),
    # bursty timestamps -> long windows.
    g = W.chung_lu(3000, 40_000, 2.2, 300, 2, 30, 21, ncolors=4, bursts=(8, 6))
    with _graph(g) as G:
        assert G.info()["max_in_degree"] > 200
        for s, k, seed in ((0, 4, 1), (3, 5, 2)):
            _, w = G.reach(s, k, seed)
            ref = oracle.sieve(g, s, k, seed)
            assert np.array_equal(w, ref)
            assert np.count_nonzero(ref) > 0


def test_small_uniform_workload_all_sources():
    g = W.small_uniform()
    with _graph(g) as G:
        for s in range(8):
            for k in (2, 3, 4, 5):
                seed = 0x5EED0001 ^ (s * 16 + k)
                _, w = G.reach(s, k, seed)
                assert np.array_equal(w, oracle.sieve(g, s, k, seed)), (s, k)


def test_tuning_shapes_do_not_change_results():
    g = _dense_uniform(1500, 20_000, 30, 5, 12)
    ref = oracle.sieve(g, 3, 8, 77)
    with _graph(g) as G:
        for ppl, chunk in ((2, 64), (2, 128), (4, 128), (4, 256), (2, 256)):
            capi.rr_set_tuning(G.handle, 8, ppl, chunk)
            _, w = G.reach(3, 8, 77)
            assert np.array_equal(w, ref), (ppl, chunk)


def test_point_sums_match_oracle():
    g = _dense_uniform(1200, 15_000, 25, 5, 13, ncolors=3)
    masks = [0, 1, 5, 31, 63, 64, 100, 127]
    with _graph(g) as G:
        dev = G.point_sums(2, 7, 55, masks)
        _, ref = oracle.sieve(g, 2, 7, 55, masks=masks, per_mask=True)
        assert np.array_equal(dev, ref)
        assert np.count_nonzero(ref) > 0
        motif = [int(g["color"][2]), 0, 1, 2, 0, 1, 2]
        dev = G.point_sums(2, 7, 56, masks, motif=motif)
        _, ref = oracle.sieve(g, 2, 7, 56, masks=masks, motif=motif, per_mask=True)
        assert np.array_equal(dev, ref)


def test_edge_cases():
    # no edges
    g0 = {"n": 5, "src": np.zeros(0, np.uint32), "dst": np.zeros(0, np.uint32),
          "t": np.zeros(0, np.uint32), "delta": np.ones(5, np.uint32)}
    with _graph(g0) as G:
        bm, w = G.reach(0, 3, 1)
        assert not w.any() and not bm.any()
    # extreme timestamps / waits: no overflow in t_e - delta or t_f + delta
    big = 2**32 - 1
    g1 = {"n": 4, "src": np.array([0, 1, 2, 1], np.uint32),
          "dst": np.array([1, 2, 3, 3], np.uint32),
          "t": np.array([big - 5, big, big, 0], np.uint32),
          "delta": np.array([0, big, big, 0], np.uint32)}
    with _graph(g1) as G:
        for k in (2, 3, 4):
            _, w = G.reach(0, k, 3)
            assert np.array_equal(w, oracle.sieve(g1, 0, k, 3))
    # parallel duplicate edges are distinct variables and do not cancel
    g2 = {"n": 3, "src": np.array([0, 0, 1, 1], np.uint32),
          "dst": np.array([1, 1, 2, 2], np.uint32), "t": np.array([1, 1, 2, 2], np.uint32),
          "delta": np.array([1, 1, 1], np.uint32)}
    with _graph(g2) as G:
        _, w = G.reach(0, 3, 4)
        ref = oracle.sieve(g2, 0, 3, 4)
        assert np.array_equal(w, ref) and ref[2] != 0
    # large k on a tiny graph (2^16 points, several chunks), and k = 20
    g3 = W.tiny_random(33, n=8, m=24, tau=4, dmax=3)
    with _graph(g3) as G:
        _, w = G.reach(0, 8, 5)
        assert np.array_equal(w, oracle.sieve(g3, 0, 8, 5))
        _, w16 = G.reach(0, 16, 6)
        assert not w16.any()  # 16 vertices cannot fit in an 8-vertex graph
    # invalid queries
    with _graph(g3) as G:
        for bad in ((0, 1), (0, 21), (8, 3)):
            with pytest.raises(capi.RRError) as ei:
                G.reach(bad[0], bad[1], 1)
            assert ei.value.status == capi.RR_EINVAL
        with pytest.raises(capi.RRError):
            G.reach(0, 3, 1, motif=[0, 0, 0])  # graph has no colours


def test_bench_workload_sampled_points_and_one_sided():
    """Full n=100,000 / m=1,000,000 workload at k=8 from s=0, the benchmark's
    launch shape: sampled single points against the oracle, and the whole
    witness against the determinant identity computed by exhaustive DFS (no
    restless path of 8 vertices leaves s=0, so every sum must be exactly zero;
    sources with paths are checked in test_gpu_scale_parity.py)."""
    g = W.scale_uniform()
    with _graph(g) as G:
        bm, w = G.reach(0, 8, 0x5EED0002 ^ 1)
        reach, sdet, npaths = oracle.dfs_paths(g, 0, 8, 0x5EED0002 ^ 1, with_det=True)
        assert np.array_equal(w, sdet)
        assert np.array_equal(w != 0, reach.astype(bool))
        masks = [1, 77, 200, 255]
        dev = G.point_sums(0, 8, 0x5EED0002 ^ 1, masks)
        _, ref = oracle.sieve(g, 0, 8, 0x5EED0002 ^ 1, masks=masks, per_mask=True)
        assert np.array_equal(dev, ref)
    # the same shape with a short time range, where long walks exist: sampled
    # points are non-zero and must agree bit for bit
    g2 = W.uniform(100_000, 1_000_000, 30, 1, 20, 0x5EED0002 + 100)
    with _graph(g2) as G:
        masks = [3, 129, 254]
        dev = G.point_sums(0, 8, 42, masks)
        _, ref = oracle.sieve(g2, 0, 8, 42, masks=masks, per_mask=True)
        assert np.count_nonzero(ref) > 0
        assert np.array_equal(dev, ref)


def test_full_size_dense_windows_full_witness():
    """n=100,000 / m=1,000,000 with t ~ U[1,30]: windows hold several rows and
    restless walks survive every layer; the whole witness vector must equal the
    oracle's (all 64 points, k=6), and the per-point engine must agree too."""
    g = W.uniform(100_000, 1_000_000, 30, 1, 20, 0x5EED0002 + 200)
    ref = oracle.sieve(g, 7, 6, 31)
    assert np.count_nonzero(ref) > 100
    with _graph(g) as G:
        _, w = G.reach(7, 6, 31)
        assert np.array_equal(w, ref)
    with _graph(g, capi.FLAG_DENSE_STATE) as G:
        _, w = G.reach(7, 6, 31)
        assert np.array_equal(w, ref)


@pytest.mark.parametrize("k", [2, 3, 4, 5, 9, 11])
def test_engines_agree_across_k(k):
    # compact graphs run the reduced-state engine for k >= 2, dense-flag graphs
    # the per-point engine; both must equal the oracle (multi-chunk for k >= 10)
    g = _dense_uniform(800, 9_000, 12, 4, 70 + k, ncolors=2)
    ref = oracle.sieve(g, 1, k, 1000 + k)
    with _graph(g) as G:
        _, w = G.reach(1, k, 1000 + k)
        assert np.array_equal(w, ref)
    with _graph(g, capi.FLAG_DENSE_STATE) as G:
        _, w = G.reach(1, k, 1000 + k)
        assert np.array_equal(w, ref)


def test_graph_replay_and_direct_launch_agree():
    # with kernel timing enabled the library launches kernels one by one; by
    # default it replays a captured CUDA graph per query shape
    g = _dense_uniform(1000, 12_000, 20, 5, 81)
    ref = oracle.sieve(g, 4, 7, 5)
    with _graph(g) as G:
        capi.rr_timing_enable(True)
        try:
            _, w_direct = G.reach(4, 7, 5)
        finally:
            capi.rr_timing_enable(False)
        times = capi.rr_timing_read(reset=True)
        assert times["second_layer"][1] >= 1 and times["last_layer"][1] >= 1
        _, w_graph = G.reach(4, 7, 5)
        _, w_graph2 = G.reach(4, 7, 5)  # replay of the cached graph
        assert np.array_equal(w_direct, ref)
        assert np.array_equal(w_graph, ref) and np.array_equal(w_graph2, ref)


def test_point_shards_xor_to_the_full_witness():
    # the multi-GPU design splits the points into ranges; on one GPU the XOR of
    # the ranges' point sums must equal the full query's witness
    from paper_2010_08423_gb300 import shard
    g = _dense_uniform(1000, 12_000, 20, 5, 91)
    with _graph(g) as G:
        _, full = G.reach(2, 7, 8)
        parts = []
        for r in range(3):
            f, c = shard.point_range(7, r, 3, align=16)
            pm = G.point_sums(2, 7, 8, list(range(f, f + c)))
            parts.append(shard.xor_combine(pm))
        assert np.count_nonzero(full) > 0
        assert np.array_equal(shard.xor_combine(parts), full)


def _hub_graph(seed=5, n=300, hub_in=2000, hub_out=2000, rest=2000, tau=10, delta=3):
    rng = np.random.default_rng(seed)
    src = np.concatenate([rng.integers(1, n, hub_in), np.zeros(hub_out, np.int64),
                          rng.integers(1, n, rest)]).astype(np.uint32)
    dst = np.concatenate([np.zeros(hub_in, np.int64), rng.integers(1, n, hub_out),
                          rng.integers(1, n, rest)]).astype(np.uint32)
    bad = src == dst
    dst[bad] = (dst[bad] % (n - 1)) + 1
    dst[(src == dst)] = (dst[(src == dst)] + 1) % n
    t = rng.integers(1, tau + 1, src.shape[0]).astype(np.uint32)
    return {"n": n, "src": src, "dst": dst, "t": t,
            "delta": np.full(n, delta, np.uint32), "color": rng.integers(0, 3, n).astype(np.uint8)}


def test_cut_hub_segments_two_points_per_lane_odd_groups():
    """Cut hub segments with 2 points per lane and 1, 3 or 7 lane groups per
    chunk (7, 21 or 49 transformed values a row, an odd count) and with 3
    groups of 4 points: the per-point state's carry table that follows the
    transformed buffer stays aligned for its vector loads, and the sums exact."""
    g = _hub_graph()
    with _graph(g) as G:
        nonzero = 0
        for k, ppl, chunk in ((6, 2, 64), (7, 2, 192), (8, 2, 192), (9, 4, 384), (10, 2, 448)):
            capi.rr_set_tuning(G.handle, k, ppl, chunk)
            ref = oracle.sieve(g, 9, k, 90 + k)
            _, w = G.reach(9, k, 90 + k)
            assert np.array_equal(w, ref), (k, ppl, chunk)
            nonzero += int(np.count_nonzero(ref) > 0)
        assert nonzero >= 3


def test_cut_hub_segments_carry_fixup():
    """A vertex with ~2,000 in- and out-rows: its head segment in every row
    list is cut into pieces of 128 rows computed in parallel and stitched by the
    carry fix-up; sums must stay bit-exact, for both engines and the batch."""
    import torch
    g = _hub_graph()
    assert not np.any(g["src"] == g["dst"])
    with _graph(g) as G:
        info = G.info()
        assert info["max_in_degree"] >= 1900
        batch = []
        for s, k in ((3, 3), (5, 4), (7, 5), (9, 6), (0, 5)):
            ref = oracle.sieve(g, s, k, 70 + k)
            _, w = G.reach(s, k, 70 + k)
            assert np.array_equal(w, ref), (s, k)
            batch.append({"source": s, "k": k, "seed": 70 + k, "motif": None, "ref": ref})
        motif = [int(g["color"][4]), 0, 1, 2, 0]
        ref = oracle.sieve(g, 4, 5, 11, motif=motif)
        _, w = G.reach(4, 5, 11, motif=motif)
        assert np.array_equal(w, ref)
        batch.append({"source": 4, "k": 5, "seed": 11, "motif": motif, "ref": ref})
        assert sum(np.count_nonzero(b["ref"]) > 0 for b in batch) >= 4
        torch.cuda.set_device(0)
        d_w = torch.zeros((len(batch), g["n"]), dtype=torch.int64, device="cuda")
        capi.rr_reach_batch_device(G.handle, batch, d_w)
        torch.cuda.synchronize()
        w = d_w.cpu().numpy().view(np.uint64)
        for i, b in enumerate(batch):
            assert np.array_equal(w[i], b["ref"]), i
    with _graph(g, capi.FLAG_DENSE_STATE) as G:
        _, w = G.reach(9, 6, 76)
        assert np.array_equal(w, oracle.sieve(g, 9, 6, 76))


def test_k3_closed_form_cycles_and_parallel_edges():
    """k = 3 sums its last layer in closed form (a 3x3 permanent per edge).
    Walks s -> a -> s repeat z_s and must cancel; parallel edges carry distinct
    y and must not; colored queries take z from the shade table."""
    rng = np.random.default_rng(33)
    n = 40
    src, dst, t = [], [], []
    for a in range(1, 12):
        for rep in range(3):                      # parallel s -> a edges
            src.append(0); dst.append(a); t.append(5 + rep)
        src.append(a); dst.append(0); t.append(7)  # back to the source
        for b in rng.integers(12, n, 4):
            src.append(a); dst.append(int(b)); t.append(int(rng.integers(5, 10)))
    g = {"n": n, "src": np.array(src, np.uint32), "dst": np.array(dst, np.uint32),
         "t": np.array(t, np.uint32), "delta": np.full(n, 3, np.uint32),
         "color": rng.integers(0, 2, n).astype(np.uint8)}
    with _graph(g) as G:
        for seed in (1, 2, 3):
            _, w = G.reach(0, 3, seed)
            ref = oracle.sieve(g, 0, 3, seed)
            assert np.array_equal(w, ref)
            assert w[0] == 0 and np.count_nonzero(ref) > 5
            motif = [int(g["color"][0]), 0, 1]
            _, w = G.reach(0, 3, seed, motif=motif)
            assert np.array_equal(w, oracle.sieve(g, 0, 3, seed, motif=motif))


def test_autotune_picks_a_valid_shape_and_keeps_results():
    g = _dense_uniform(1500, 20_000, 30, 5, 13)
    ref = oracle.sieve(g, 7, 6, 41)
    with _graph(g) as G:
        ppl, chunk = capi.rr_autotune(G.handle, 6)
        assert ppl in (2, 4) and chunk % (32 * ppl) == 0 and chunk <= max(64, 32 * ppl)
        _, w = G.reach(7, 6, 41)
        assert np.array_equal(w, ref)


def test_sync_into_preallocated_pinned_buffers():
    import torch
    g = _dense_uniform(1200, 15_000, 25, 5, 14)
    n = g["n"]
    h_bm = torch.full(((n + 7) // 8,), 255, dtype=torch.uint8, pin_memory=True).numpy()
    h_w = torch.full((n,), -1, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    with _graph(g) as G:
        bm, w = G.reach(5, 6, 21)
        bm2, w2 = G.reach(5, 6, 21, out=(h_bm, h_w))
        assert bm2 is h_bm and w2 is h_w
        assert np.array_equal(w, h_w) and np.array_equal(bm, h_bm)
        assert np.array_equal(w, oracle.sieve(g, 5, 6, 21))
        with pytest.raises(ValueError):
            G.reach(5, 6, 21, out=(h_bm, h_w[:10]))


def test_largest_k_on_a_restless_chain():
    """k = 20, the largest k accepted (2^20 sieve points, 2,048 point chunks of
    512): a 21-vertex chain 0 -> 1 -> ... -> 20 with times 1..20 and waits of at
    most 1, plus a few edges that break restlessness. The witness must equal
    the determinant identity computed by DFS (the sieve oracle would take too
    long at this k): non-zero exactly at vertex 19."""
    src = list(range(20)) + [3, 7, 12]
    dst = list(range(1, 21)) + [9, 15, 2]
    t = list(range(1, 21)) + [40, 2, 1]
    g = {"n": 21, "src": np.array(src, np.uint32), "dst": np.array(dst, np.uint32),
         "t": np.array(t, np.uint32), "delta": np.ones(21, np.uint32)}
    with _graph(g) as G:
        _, w = G.reach(0, 20, 2024)
    reach, sdet, npaths = oracle.dfs_paths(g, 0, 20, 2024, with_det=True)
    assert npaths == 1 and np.nonzero(reach)[0].tolist() == [19]
    assert np.array_equal(w, sdet)
