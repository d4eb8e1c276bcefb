"""Runs warm-up queries and then one query of a named synthetic workload, for
a profiler to capture (e.g. ``ncu ... python -m paper_2010_08423_gb300.profile_query
--workload powerlaw-2e5 --k 10``). Prints the query's time and its number of
reached vertices (or, with --batch N, times one persistent batched launch of N
mixed queries). Inputs come from ``workloads`` (seeded, synthetic).

Workloads:
  uniform-1e5    n = 1e5, m = 1e6 uniform multigraph, t ~ U[1,1000], delta ~ U{1..20}
  powerlaw-2e5   Chung-Lu exponent 2.5, n = 2e5, m = 2e6, bursty t in [1,1e4],
                 delta ~ U{5..50}, 8 colours (the n = 1e6 motif workload at 1/5 scale)
  powerlaw-1e6   the same at n = 1e6, m = 1e7
"""
import argparse
import sys


def main(argv=None) -> int:
    import torch

    from . import capi
    from . import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="powerlaw-2e5",
                    choices=["uniform-1e5", "powerlaw-2e5", "powerlaw-1e6"])
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--motif", action="store_true", help="a motif query (source colour + k-1 colours)")
    ap.add_argument("--shape", default=None,
                    help="points per lane x points per chunk (e.g. 4x512), as rr_set_tuning")
    ap.add_argument("--batch-shape", default=None,
                    help="blocks per SM, ranges, max chunk of the batch (e.g. 5,2,1024), "
                         "as rr_set_batch_tuning")
    ap.add_argument("--flags", type=int, default=0,
                    help="rr_graph_load flags (capi.FLAG_*), e.g. 512 = k = 5 in closed form")
    ap.add_argument("--batch", type=int, default=0,
                    help="instead: one persistent batched launch of this many queries, "
                         "k ~ U{4..12}, odd ones coloured")
    args = ap.parse_args(argv)

    if args.workload == "uniform-1e5":
        g, s = W.scale_uniform(ncolors=8), 0
    else:
        n = 200_000 if args.workload == "powerlaw-2e5" else 1_000_000
        g = W.chung_lu(n, 10 * n, 2.5, 10_000, 5, 50, W.GRAPH_SEED_BASE + 3, ncolors=8,
                       bursts=(50, 20))
        s = W.first_source(g)
    motif = W.motif_for(g, s, args.k, W.GRAPH_SEED_BASE + 3) if args.motif else None
    torch.cuda.set_device(0)
    if args.batch:
        qs = W.query_set(g, args.batch, 4, 12, W.GRAPH_SEED_BASE + 4)
        with capi.Graph(g, args.flags) as G:
            if args.batch_shape:
                capi.rr_set_batch_tuning(G.handle, *(int(x) for x in args.batch_shape.split(",")))
            d_w = torch.zeros((len(qs), g["n"]), dtype=torch.int64, device="cuda")
            st = torch.cuda.Stream()
            for _ in range(args.warmup):
                capi.rr_reach_batch_device(G.handle, qs, d_w, None, None, st.cuda_stream)
            st.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            capi.rr_reach_batch_device(G.handle, qs, d_w, None, None, st.cuda_stream)
            e1.record(st)
            st.synchronize()
            print(f"{args.workload} batch of {len(qs)} ms {e0.elapsed_time(e1):.3f}")
        return 0
    with capi.Graph(g, args.flags) as G:
        if args.shape:
            ppl, chunk = (int(x) for x in args.shape.lower().split("x"))
            capi.rr_set_tuning(G.handle, args.k, ppl, chunk)
        d_w = torch.zeros(g["n"], dtype=torch.int64, device="cuda")
        st = torch.cuda.Stream()
        for i in range(args.warmup):
            capi.rr_reach_device(G.handle, s, args.k, 5 + i, d_w, None, st.cuda_stream, motif=motif)
        st.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        capi.rr_reach_device(G.handle, s, args.k, 99, d_w, None, st.cuda_stream, motif=motif)
        e1.record(st)
        st.synchronize()
        print(f"{args.workload} k={args.k} ms {e0.elapsed_time(e1):.3f} "
              f"reached {int((d_w != 0).sum().item())} info {G.info()}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
