"""The pair tail: layer k-3 stores its sums over the points of a group that
hold one or two given labels, layer k-2 runs in label space from them, and the
last layer reads its label-space rows (chunks of 256 points or more in at most
8 point groups; other shapes keep the per-point tail). Against the oracle and
against the per-point tail (load flag bit 5), bit for bit: witness and
per-edge sums over k = 6..12, both lane shapes, chunks of 2 to 8 point groups
and shapes on either side of the limits, layer 3 per point or in pair-label
space, cut hub segments, point ranges whose chunks do not start at a multiple
of the chunk size, motif queries, and the persistent batch."""
import numpy as np
import pytest

import oracle
from paper_2010_08423_gb300 import capi
from paper_2010_08423_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    capi.load()
    oracle.build()
    torch.cuda.set_device(0)


def test_info_reports_the_pair_tail():
    g = W.uniform(500, 4000, 20, 0, 4, 5)
    with capi.Graph(g) as G:
        assert G.info()["pair_tail"] == 1
    with capi.Graph(g, capi.FLAG_PAIR_TAIL_OFF) as G:
        assert G.info()["pair_tail"] == 0


# (k, points per lane, points per chunk): 2, 4 and 8 point groups of 256 points
# or more; (6, 2, 64), (7, 4, 128) and (9, 2, 192) are below 256 points and
# (11, 2, 2048) has 32 groups: those keep the per-point tail
SHAPES = [(6, 2, 64), (7, 4, 128), (8, 2, 256), (8, 4, 256), (9, 2, 192), (9, 2, 512),
          (9, 4, 512), (10, 4, 1024), (10, 2, 256), (10, 4, 384), (11, 4, 1024), (11, 2, 2048),
          (12, 4, 512)]


@pytest.mark.parametrize("pair_flag", [capi.FLAG_PAIR_OFF, capi.FLAG_PAIR_ON])
def test_shapes_match_oracle_and_per_point_tail(pair_flag):
    # t ~ U[1,30] on n=1500, m=20000: long restless walks, windows of several rows
    g = W.uniform(1500, 20_000, 30, 0, 5, 12, ncolors=3)
    nonzero = 0
    with capi.Graph(g, pair_flag) as G, capi.Graph(g, pair_flag | capi.FLAG_PAIR_TAIL_OFF) as H:
        for k, ppl, chunk in SHAPES:
            capi.rr_set_tuning(G.handle, k, ppl, chunk)
            capi.rr_set_tuning(H.handle, k, ppl, chunk)
            seed = 1000 + 17 * k + ppl
            ref = oracle.sieve(g, 3, k, seed)
            _, w = G.reach(3, k, seed)
            _, w_off = H.reach(3, k, seed)
            assert np.array_equal(w, ref), (k, ppl, chunk, pair_flag)
            assert np.array_equal(w_off, ref), (k, ppl, chunk, pair_flag)
            nonzero += int(np.count_nonzero(ref) > 0)
        assert nonzero >= len(SHAPES) - 2


def test_motif_queries_and_per_edge_sums():
    g = W.uniform(2000, 30_011, 40, 0, 6, 11, ncolors=3)
    with capi.Graph(g) as G:
        for s, k, seed in ((17, 6, 2), (5, 7, 3), (0, 8, 4)):
            S, E, _, _ = G.arrival(s, k, seed)
            S_ref, E_ref = oracle.sieve(g, s, k, seed, edges=True)
            assert np.array_equal(S, S_ref), (s, k)
            assert np.array_equal(E, E_ref), (s, k)
            assert np.count_nonzero(E_ref) > 0
        for k in (6, 8, 10):
            motif = [int(g["color"][5])] + [j % 3 for j in range(k - 1)]
            _, w = G.reach(5, k, 40 + k, motif=motif)
            assert np.array_equal(w, oracle.sieve(g, 5, k, 40 + k, motif=motif)), k
        motif = [int(g["color"][5])] + [j % 3 for j in range(7)]
        S, E, _, _ = G.arrival(5, 8, 9, motif=motif)
        S_ref, E_ref = oracle.sieve(g, 5, 8, 9, motif=motif, edges=True)
        assert np.array_equal(S, S_ref) and np.array_equal(E, E_ref)


def test_cut_hub_segments():
    """A vertex with ~2,000 in- and out-rows: the pair sums and the
    label-space rows of its cut head segments are stitched by the carry
    fix-up of narrow buffers."""
    from test_gpu_parity import _hub_graph
    g = _hub_graph()
    with capi.Graph(g) as G:
        assert G.info()["max_in_degree"] >= 1900
        nonzero = 0
        for k, ppl, chunk in ((8, 2, 256), (8, 4, 256), (9, 4, 384), (10, 4, 1024), (10, 2, 448)):
            capi.rr_set_tuning(G.handle, k, ppl, chunk)
            ref = oracle.sieve(g, 9, k, 190 + k)
            _, w = G.reach(9, k, 190 + k)
            assert np.array_equal(w, ref), (k, ppl, chunk)
            nonzero += int(np.count_nonzero(ref) > 0)
        assert nonzero >= 3


def test_ranges_off_the_chunk_grid():
    """Point ranges starting at multiples of 128 that are not multiples of the
    chunk: the groups' fixed labels above the in-group ones differ from group
    to group without following the group index."""
    g = W.uniform(3000, 40_000, 40, 1, 6, 0x5EED0000 + 301, ncolors=3)
    with capi.Graph(g) as G:
        capi.rr_set_tuning(G.handle, 10, 4, 1024)
        capi.rr_set_tuning(G.handle, 11, 2, 512)
        for k, first, count in ((10, 640, 384), (10, 128, 896), (11, 384, 1152), (11, 1920, 128)):
            part = G.reach_range(5, k, 77 + k, first, count)
            ref = oracle.sieve(g, 5, k, 77 + k, masks=np.arange(first, first + count, dtype=np.uint32))
            assert np.array_equal(part, ref), (k, first, count)
            assert np.count_nonzero(ref) > 0, (k, first, count)


def test_batch_matches_single_queries_and_oracle():
    """The persistent batch with the pair tail (units of 256 points or more)
    and without it (load flag bit 5), against single queries and the oracle."""
    import torch
    g = W.uniform(1500, 20_000, 30, 0, 5, 12, ncolors=3)
    rng = np.random.default_rng(9)
    qs = []
    for i in range(24):
        k = int(rng.integers(4, 13))
        s = int(rng.integers(0, g["n"]))
        motif = ([int(g["color"][s])] + [int(x) for x in rng.integers(0, 3, k - 1)]) if i % 2 else None
        qs.append({"source": s, "k": k, "seed": int(rng.integers(1, 2**62)), "motif": motif})
    refs = [oracle.sieve(g, q["source"], q["k"], q["seed"], motif=q["motif"]) for q in qs]
    assert sum(int(np.count_nonzero(r) > 0) for r in refs) >= 12
    for flags in (0, capi.FLAG_PAIR_TAIL_OFF):
        with capi.Graph(g, flags) as G:
            for mc in (256, 512, 1024):
                capi.rr_set_batch_tuning(G.handle, 6, 2, mc)
                d_w = torch.zeros((len(qs), g["n"]), dtype=torch.int64, device="cuda")
                capi.rr_reach_batch_device(G.handle, qs, d_w)
                torch.cuda.synchronize()
                w = d_w.cpu().numpy().view(np.uint64)
                for i, r in enumerate(refs):
                    assert np.array_equal(w[i], r), (flags, mc, i, qs[i]["k"])
