#!/usr/bin/env python3
"""Benchmark: restless-reachability sieve queries on a resident temporal graph.

Headline workload (one step = one complete query: z-table, every layer over
all 2^k sieve points, fused per-vertex reduce, reach bitmap):
  Chung-Lu power-law temporal multigraph (degree exponent 2.5), n = 1,000,000,
  m = 10,000,000, timestamps in [1, 10000] drawn as Poisson(50) bursts of width
  20, delta(v) ~ U{5..50}, 8 vertex colours; k-RestlessMotifReach with k = 10
  from the first vertex with an out-edge, motif = its colour + 9 uniform
  colours; GF(2^64) mod x^64+x^4+x^3+x+1, splitmix64-seeded values (the seed
  differs per step).

Metric: GF(2^64) edge-updates/s counted as the nominal 2^k * k * m per query.
`value` is device-timed (CUDA events on the launching stream, L2 flushed
between steps, graph resident in HBM); `work` states what one query performs
(GF(2^64) multiplications and stored state values, from the per-kernel counts)
beside the nominal count, and `value_performed` the performed multiplications
per second; `e2e` is the same metric through the host-buffer C-ABI call
rr_reach_sync (descriptor uploaded and results copied back into pinned host
buffers every step). `roofline` reports the dominant kernel against the
measured copy bandwidth or the measured GF(2^64) multiply rate, whichever
binds. Extra lines: the uniform k = 8 query, the dense per-point engine on the
headline query, the small n = 1,000 graph with the full oracle, batched,
served (with the same query list one at a time), at-most-k / bounded and
fine-grained queries, and serving on an n = 1e7 graph.

--gpus N (under torchrun): one query split over the ranks by sieve points
(rr_reach_range_device), partial witnesses all-gathered and XOR-combined each
step (strong scaling: the whole job answers one query per step).

--impl reference times the CPU oracle (oracle/) on a bounded sample of the
headline query (one sieve point per step); the cpu_baseline leg does the same
on one point per core and on one point on one core. These are the only places
this file runs oracle code.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2010_08423_gb300 import workloads as W  # noqa: E402

METRIC = "GF(2^64) edge-updates/s (2^k*k*m per query)"
UNIT = "edge-updates/s"
K = 10
GRAPH_SEED = W.GRAPH_SEED_BASE + 3
WORKLOAD = ("Chung-Lu exponent 2.5 temporal multigraph n=1000000 m=10000000, t in [1,10000] as "
            "Poisson(50) bursts of width 20, delta~U{5..50}, 8 colours; k-RestlessMotifReach k=10 "
            "from the first vertex with an out-edge, motif = its colour + 9 uniform colours")
# the uniform n=1e5 / m=1e6 query (single source vertex 0, plain, k = 8)
K_UNIFORM = 8
UNIFORM_SEED = W.GRAPH_SEED_BASE + 2
UNIFORM_WORKLOAD = ("uniform temporal multigraph n=100000 m=1000000 t~U[1,1000] delta~U{1..20}; "
                    "plain k-RestlessReach k=8 from s=0")
# bytes of the query descriptor the library uploads per query (source, k,
# flags, 4 family keys, 4 pointers, 512-entry shade table)
DESC_BYTES = 16 + 32 + 32 + 512 * 4


def units_per_query(k: int, m: int) -> float:
    return float(2 ** k) * k * m


def headline_query():
    """The motif workload: graph, source, motif; query seeds graph_seed ^ (i+1)."""
    g = W.motif_powerlaw()
    s = W.first_source(g)
    motif = W.motif_for(g, s, K, GRAPH_SEED)
    return g, s, motif


def step_seed(i: int, base: int = GRAPH_SEED) -> int:
    return (base ^ (i + 1)) & ((1 << 64) - 1)


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# the sources whose change invalidates a recorded ncu capture of the query
# kernels (their code, the device arithmetic and the row lists they read)
KERNEL_SOURCES = ("rr_device.cuh", "rr_v2_device.cuh", "rr_sieve2.cu", "rr_graph.cu", "rr_internal.h")


def code_tokens(text: str) -> str:
    """C/C++ source without comments and with whitespace runs collapsed: two
    files with equal code_tokens compile to the same kernels."""
    import re
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"' or c == "'":  # string or character literal, kept whole
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return re.sub(r"\s+", " ", "".join(out)).strip()


def kernel_sources_sha1() -> str:
    """Fingerprint of the code (not the comments) of the engine's kernel sources."""
    import hashlib
    h = hashlib.sha1()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2010_08423_gb300", "csrc", name), encoding="utf-8") as fh:
            h.update(code_tokens(fh.read()).encode())
    return h.hexdigest()


TRAFFIC_RECORDS = {
    "motif": "ncu_traffic_k10_motif_powerlaw_n1e6_m1e7.json",
    "uniform": "ncu_traffic_k8_uniform_n1e5_m1e6.json",
}


def recorded_traffic(workload: str, kernel: str, ppl: int, chunk: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary of
    `workload`, or None if the kernel sources or the query shape differ from
    that capture's."""
    try:
        with open(os.path.join(ROOT, "profiles", TRAFFIC_RECORDS[workload])) as fh:
            rec = json.load(fh)
    except (OSError, KeyError):
        return None
    if kernel_sources_sha1() != rec.get("source_sha1"):
        return None
    if rec.get("shape") != [ppl, chunk]:
        return None
    return rec.get("dram_bytes_per_launch", {}).get(kernel)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def wait_first(self, timeout_s=3.0):
        """Returns once nvidia-smi has written its first sample (or on timeout)."""
        t_end = time.perf_counter() + timeout_s
        while self.proc is not None and time.perf_counter() < t_end:
            self.fh.flush()
            if os.path.getsize(self.path) > 0:
                return
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx = float(f[2])
                except ValueError:
                    continue
                for name, val in zip(names, f[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm),
                "window": "every 50 ms from 0.4 s of untimed steps of the same query just "
                          "before the timed region through its end"}


def kernel_rooflines_dense(info, k, chunk, ppl, m, n, kt, queries, hbm_peak, mul_peak, out_deg_s,
                           ztable_mults=0):
    """Per kernel kind of the per-point engine (dense state: every row a state
    row; rows with a non-empty window multiply once per point): average launch
    time, algorithmic bytes and GF(2^64) multiplications per launch (one
    layer over one point chunk), fractions of the measured peaks."""
    c = chunk
    Wr = info["window_rows"]  # rows with a non-empty window
    lanes = c // (32 * ppl)   # lane groups: the y z_v label products once per row and group
    meta = 20 * m + 4 * (n + 1)
    alg = {
        # layer 1: the source's out-edges multiply, every row stores its prefix
        "first_layer": (m * c * 8 + meta, out_deg_s * (c + k * lanes)),
        # middle layers: two gathered prefix rows per row with a window, every row stored
        "mid_layer": (m * c * 8 + Wr * 2 * c * 8 + meta, Wr * (c + k * lanes)),
        # last layer: gathers and multiplies, per-vertex XOR into the witness
        "last_layer": (Wr * 2 * c * 8 + meta + n * 8, Wr * (c + k * lanes)),
        "ztable": (n * k * 8, ztable_mults),
    }
    out = {}
    for name, (kms, kn) in kt.items():
        if not kn or name not in alg:
            continue
        avg_s = kms / kn / 1e3
        b, mu = alg[name]
        gbs = b / avg_s / 1e9
        gms = mu / avg_s / 1e9
        fh, fa = gbs / hbm_peak, gms / (mul_peak / 1e9)
        out[name] = {"avg_launch_us": round(avg_s * 1e6, 2), "launches_per_query": kn / queries,
                     "alg_bytes_per_launch": int(b), "achieved_gbs": round(gbs, 1),
                     "hbm_frac": round(fh, 4), "alg_gf_mults_per_launch": int(mu),
                     "achieved_gmul_s": round(gms, 2), "alu_frac": round(fa, 4),
                     "bound": "alu" if fa >= fh else "hbm", "time_ms_per_query": round(kms / queries, 4)}
    return out


def work_accounting(by_kernel, k, m, info, ms_per_query):
    """What one query performs against the nominal count: GF(2^64)
    multiplications and stored state values summed over the kernels' per-launch
    counts, and what the dense per-point engine multiplies for the same query."""
    mults = sum(v["alg_gf_mults_per_launch"] * v["launches_per_query"] for v in by_kernel.values())
    nominal = units_per_query(k, m)
    method = float(2 ** k) * (k - 1) * m
    # the per-point engine multiplies once per point for every row with a
    # non-empty window at layers 2..k-1 (layer 1: the source's out-edges)
    dense = float(2 ** k) * (k - 2) * info["window_rows"]
    return {
        "nominal_units_per_query": nominal,
        "method_edge_point_layer_values_per_query": method,
        "performed_gf_mults_per_query": mults,
        "dense_engine_gf_mults_per_query": dense,
        "dense_over_performed_mults": dense / max(1.0, mults),
        "nominal_over_performed": nominal / max(1.0, mults),
        "value_performed": {"value": mults / (ms_per_query / 1e3), "unit": "GF(2^64) multiplications/s"},
        "note": "performed = the per-launch multiplication counts of the roofline table times the "
                "launches per query (reduced-state engine: structurally zero rows and points are "
                "not evaluated); nominal = 2^k*k*m",
    }


def timed_queries(torch, stream, run, nsteps, flush):
    """Device time (ms) of each of nsteps calls run(i) on `stream`, L2 flushed
    (outside the events) before each."""
    ms = []
    with torch.cuda.stream(stream):
        for i in range(nsteps):
            flush.fill_(i)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run(i)
            e1.record(stream)
            stream.synchronize()
            ms.append(e0.elapsed_time(e1))
    return ms


def kernel_times(capi, torch, stream, run, nq):
    """Per-kind kernel times of nq calls launched kernel by kernel."""
    capi.rr_timing_enable(True)
    capi.rr_timing_read(reset=True)
    try:
        with torch.cuda.stream(stream):
            for i in range(nq):
                run(i)
            stream.synchronize()
        return capi.rr_timing_read(reset=True)
    finally:
        capi.rr_timing_enable(False)


def dominant_roofline(by_kernel, kt, mul_peak, hbm_peak, peak_kind, traffic):
    """The roofline object of the kernel kind with the most time per query."""
    if not by_kernel:
        return None
    dom = max(by_kernel, key=lambda k_: kt[k_][0])
    d = by_kernel[dom]
    common = {"traffic": traffic(dom) if traffic else None, "kernel": dom,
              "avg_launch_us": d["avg_launch_us"],
              "alg_bytes_per_launch": d["alg_bytes_per_launch"],
              "alg_gf_mults_per_launch": d["alg_gf_mults_per_launch"],
              "hbm_frac": d["hbm_frac"], "alu_frac": d["alu_frac"]}
    if d["bound"] == "alu":
        return {"bound": "alu", "achieved": d["achieved_gmul_s"], "peak": round(mul_peak / 1e9, 2),
                "unit": "GF(2^64) Gmul/s", "frac": d["alu_frac"],
                "peak_kind": "measured live: rr_bench_gf_mul, register-only multiply chains on all "
                             "SMs, each operand value in one product (ALU-pipe bound)", **common}
    return {"bound": "hbm", "achieved": d["achieved_gbs"], "peak": hbm_peak, "unit": "GB/s",
            "frac": d["hbm_frac"], "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)", **common}


def motif_ztable_mults(g, motif, k):
    """A coloured z entry multiplies once per shade of its vertex's colour (Eq. 3)."""
    mu = np.bincount(np.asarray(motif, dtype=np.int64), minlength=256)
    return k * int((np.bincount(np.asarray(g["color"], dtype=np.int64), minlength=256) * mu).sum())


def uniform_metrics(capi, torch, g, mul_peak, hbm_peak, peak_kind, steps=20):
    """The uniform n=1e5 / m=1e6 graph, plain k=8 from vertex 0 (no restless
    path of 3 or more vertices leaves it, so the witness is zero; the full
    sieve still runs), autotuned shape."""
    n, m = g["n"], len(g["src"])
    with capi.Graph(g) as G:
        info = G.info()
        ppl, chunk = capi.rr_autotune(G.handle, K_UNIFORM)
        st = torch.cuda.Stream()
        d_w = torch.empty(n, dtype=torch.int64, device="cuda")
        d_bm = torch.empty((n + 7) // 8, dtype=torch.uint8, device="cuda")
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")

        def run(i):
            capi.rr_reach_device(G.handle, 0, K_UNIFORM, step_seed(i, UNIFORM_SEED), d_w, d_bm,
                                 st.cuda_stream)
        timed_queries(torch, st, run, 3, flush)
        ms = timed_queries(torch, st, lambda i: run(100 + i), steps, flush)
        kt = kernel_times(capi, torch, st, lambda i: run(200 + i), 5)
    by_kernel = kernel_rooflines(info, K_UNIFORM, chunk, ppl, n, kt, 5, hbm_peak, mul_peak)
    per_q = sum(ms) / steps
    roof = dominant_roofline(by_kernel, kt, mul_peak, hbm_peak, peak_kind,
                             lambda kern: recorded_traffic("uniform", kern, ppl, chunk))
    return {"workload": UNIFORM_WORKLOAD, "value": units_per_query(K_UNIFORM, m) / (per_q / 1e3),
            "unit": UNIT, "ms_per_query": per_q, "steps": steps,
            "shape": {"points_per_lane": ppl, "points_per_chunk": chunk},
            "work": work_accounting(by_kernel, K_UNIFORM, m, info, per_q),
            "roofline": roof, "roofline_by_kernel": by_kernel,
            "rows": {"state": info["producer_window_rows"] + 1, "deep": info["state_compute_rows"],
                     "deep_compute": info["deep_compute_rows"], "last_layer": info["deep_tail_rows"]},
            "l2": "flushed between queries",
            "parity": "tests/test_gpu_scale_parity.py: full k=8 witness from a source with "
                      "8-vertex paths and from vertex 0, bit-exact vs the oracle"}


def dense_metrics(capi, torch, g, s, motif, mul_peak, hbm_peak, peak_kind, nq=2):
    """The headline query on the per-point engine with the dense state layout
    (every row stored for every point; every row with a non-empty window
    multiplied for every point): no structural pruning."""
    n, m = g["n"], len(g["src"])
    ppl, chunk = 4, 256  # 2 * (m+1) * 256 * 8 bytes of state (41 GB)
    with capi.Graph(g, capi.FLAG_DENSE_STATE) as G:
        info = G.info()
        capi.rr_set_tuning(G.handle, K, ppl, chunk)
        st = torch.cuda.Stream()
        d_w = torch.empty(n, dtype=torch.int64, device="cuda")
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")

        def run(i):
            capi.rr_reach_device(G.handle, s, K, step_seed(300 + i), d_w, None, st.cuda_stream,
                                 motif=motif)
        timed_queries(torch, st, run, 1, flush)
        ms = timed_queries(torch, st, lambda i: run(10 + i), nq, flush)
        kt = kernel_times(capi, torch, st, lambda i: run(20 + i), 1)
    out_deg_s = int(np.count_nonzero(g["src"] == s))
    by_kernel = kernel_rooflines_dense(info, K, chunk, ppl, m, n, kt, 1, hbm_peak, mul_peak,
                                       out_deg_s, motif_ztable_mults(g, motif, K))
    per_q = sum(ms) / nq
    mults = sum(v["alg_gf_mults_per_launch"] * v["launches_per_query"] for v in by_kernel.values())
    return {"workload": "the headline query on the per-point engine, dense state layout",
            "value": units_per_query(K, m) / (per_q / 1e3), "unit": UNIT, "ms_per_query": per_q,
            "steps": nq, "shape": {"points_per_lane": ppl, "points_per_chunk": chunk},
            "performed_gf_mults_per_query": mults,
            "value_performed": {"value": mults / (per_q / 1e3), "unit": "GF(2^64) multiplications/s"},
            "roofline": dominant_roofline(by_kernel, kt, mul_peak, hbm_peak, peak_kind, None),
            "roofline_by_kernel": by_kernel, "l2": "flushed between queries"}


def small_metrics(capi, torch, reps=200):
    """n=1,000 / m=10,000, t ~ U[1,100], delta ~ U{1..5}, plain k=5 from
    vertex 0: the GPU query (device-timed, launch-bound) beside the oracle's
    full sieve (all 32 points, unsampled) on one thread and on all cores."""
    import oracle
    g = W.small_uniform()
    n, m, k = g["n"], len(g["src"]), 5
    with capi.Graph(g) as G:
        st = torch.cuda.Stream()
        d_w = torch.empty(n, dtype=torch.int64, device="cuda")
        d_bm = torch.empty((n + 7) // 8, dtype=torch.uint8, device="cuda")
        with torch.cuda.stream(st):
            for i in range(10):
                capi.rr_reach_device(G.handle, 0, k, i + 1, d_w, d_bm, st.cuda_stream)
            st.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for i in range(reps):
                capi.rr_reach_device(G.handle, 0, k, 100 + i, d_w, d_bm, st.cuda_stream)
            e1.record(st)
            st.synchronize()
        gpu_ms = e0.elapsed_time(e1) / reps
        reached = int((d_w != 0).sum().item())
    oracle.build()
    cores = os.cpu_count() or 1
    t1 = []
    for i in range(3):
        t0 = time.perf_counter()
        oracle.sieve(g, 0, k, 100 + i, threads=1)
        t1.append(time.perf_counter() - t0)
    ta = []
    for i in range(3):
        t0 = time.perf_counter()
        oracle.sieve(g, 0, k, 100 + i, threads=cores)
        ta.append(time.perf_counter() - t0)
    u = units_per_query(k, m)
    return {"workload": "uniform temporal multigraph n=1000 m=10000 t~U[1,100] delta~U{1..5}; plain "
                        "k-RestlessReach k=5 from s=0",
            "value": u / (gpu_ms / 1e3), "unit": UNIT, "ms_per_query": gpu_ms,
            "reachable_vertices": reached,
            "cpu_oracle_full": {"single_thread_ms": 1e3 * min(t1), "all_cores_ms": 1e3 * min(ta),
                                "cores": cores, "value_single_thread": u / min(t1),
                                "value_all_cores": u / min(ta),
                                "sample": "all 32 sieve points (no sampling), best of 3"}}


def cpu_baseline(g, s, motif):
    """The oracle as it stands on the headline query: one sieve point per host
    core (all cores) and one point on one core; values scaled by points to the
    nominal unit (the oracle's work is the same for every point)."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    m = len(g["src"])
    masks = (640 + np.arange(cores)).astype(np.uint32) % (2 ** K)
    t0 = time.perf_counter()
    oracle.sieve(g, s, K, step_seed(0), motif=motif, masks=masks, threads=cores)
    dt_all = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.sieve(g, s, K, step_seed(0), motif=motif, masks=masks[:1], threads=1)
    dt_one = time.perf_counter() - t0
    u = units_per_query(K, m)
    return {"value": u * len(masks) / 2 ** K / dt_all, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"{len(masks)} of {2 ** K} sieve points of one k={K} query of the headline "
                      f"workload, one point per core ({dt_all:.1f} s wall), scaled by points",
            "single_thread": {"value": u / 2 ** K / dt_one, "unit": UNIT, "cores": 1,
                              "sample": f"1 of {2 ** K} sieve points on one core ({dt_one:.1f} s), "
                                        "scaled by points"},
            "cpu_model": cpu_model(), "nproc": cores,
            "oracle": "plain C, one point at a time, windows scanned in time order, bitwise "
                      "shift-and-add GF(2^64) multiply (gcc -O2 -fopenmp)"}


def batch_kernel_alg(info, qs, max_chunk, n):
    """Algorithmic bytes and GF(2^64) multiplications of the persistent batch
    kernel for the queries qs: per unit (one query's chunk of points) the same
    per-layer counts as the one-query kernels, with layer 3 per point (the
    batch has no pair-label form); k <= 3 and the label-space layer 2 run in
    the prologue kernels and are not counted here."""
    S = info["producer_window_rows"]
    D = info["state_compute_rows"]
    DC = info["deep_compute_rows"]
    T3 = info["deep_tail_rows"]
    T2 = info["tail_rows"]
    R3 = info["deep_head_runs"]
    tot_b = tot_m = 0.0
    for q in qs:
        k = q["k"]
        if k <= 3:
            continue
        npts = 2 ** k
        ppl = 4 if npts >= 128 else 2
        c = max(32 * ppl, min(npts, max_chunk))
        lg = 7 if ppl == 4 else 6
        rs = c // (32 * ppl) * (lg + 1)
        nch = (npts + c - 1) // c
        if k == 4:
            layers = [(S * rs * 8 + S * 20 + 2 * S * 8, S * (1 + k + c)),
                      (2 * T2 * rs * 8 + T2 * 16 + n * 8, T2 * rs)]
        else:
            l3 = (D * (rs if k == 5 else c) * 8 + 2 * D * k * 8 + D * 20, D * (k + 2 * c) + R3 * c)
            mid = (D * c * 8 + 2 * DC * c * 8 + D * 20, DC * (c + k))
            tail = (D * rs * 8 + 2 * DC * c * 8 + D * 20, DC * (c + k))
            last = (2 * T3 * rs * 8 + T3 * 16 + n * 8, T3 * rs)
            layers = [l3] + ([mid] * (k - 6) + [tail] if k >= 6 else []) + [last]
        tot_b += nch * sum(x[0] for x in layers)
        tot_m += nch * sum(x[1] for x in layers)
    return tot_b, tot_m


def batched_metrics(capi, torch, gc, mul_peak, hbm_peak, nq=256, seed=UNIFORM_SEED):
    """The same graph with 8 colours; nq queries, s ~ U, k ~ U{4..12}, odd q
    with a motif (source colour + k-1 uniform colours): one persistent batched
    launch in the automatic shape and in the shape rr_autotune_batch picks on
    this query list, against one launch sequence per query; results compared
    bit for bit."""
    qs = W.query_set(gc, nq, 4, 12, seed)
    n = gc["n"]
    m = len(gc["src"])
    units = sum(units_per_query(q["k"], m) for q in qs)
    with capi.Graph(gc) as G:
        info = G.info()
        stream = torch.cuda.Stream()
        d_b = torch.zeros((nq, n), dtype=torch.int64, device="cuda")
        d_s = torch.zeros((nq, n), dtype=torch.int64, device="cuda")
        d_st = torch.zeros(nq, dtype=torch.int32, device="cuda")

        def batch_ms(reps=3):
            capi.rr_reach_batch_device(G.handle, qs, d_b, None, d_st, stream.cuda_stream)
            stream.synchronize()
            best = 1e30
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                capi.rr_reach_batch_device(G.handle, qs, d_b, None, d_st, stream.cuda_stream)
                e1.record(stream)
                stream.synchronize()
                best = min(best, e0.elapsed_time(e1))
            return best / 1e3
        t_auto = batch_ms()
        t0 = time.perf_counter()
        tuned = capi.rr_autotune_batch(G.handle, qs)
        tune_s = time.perf_counter() - t0
        t_batch = batch_ms()
        # the batch kernel alone, from the library's per-launch events
        capi.rr_timing_enable(True)
        capi.rr_timing_read(reset=True)
        try:
            capi.rr_reach_batch_device(G.handle, qs, d_b, None, d_st, stream.cuda_stream)
            stream.synchronize()
            kt = capi.rr_timing_read(reset=True)
        finally:
            capi.rr_timing_enable(False)
        for q in qs[:8]:
            capi.rr_reach_device(G.handle, q["source"], q["k"], q["seed"], d_s[0], None,
                                 stream.cuda_stream, motif=q["motif"])
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for i, q in enumerate(qs):
                capi.rr_reach_device(G.handle, q["source"], q["k"], q["seed"], d_s[i], None,
                                     stream.cuda_stream, motif=q["motif"])
            e1.record(stream)
            stream.synchronize()
            t_single = e0.elapsed_time(e1) / 1e3
        same = bool(torch.equal(d_b, d_s)) and int(d_st.abs().sum().item()) == 0
    kms, kn = kt.get("batch", (0.0, 0))
    roof = None
    if kn:
        ab, am = batch_kernel_alg(info, qs, tuned["max_chunk"], n)
        ks = kms / kn / 1e3
        fa, fh = am / ks / mul_peak, ab / ks / 1e9 / hbm_peak
        roof = {"kernel": "k_batch", "avg_launch_us": round(ks * 1e6, 1),
                "alg_gf_mults_per_launch": int(am), "alg_bytes_per_launch": int(ab),
                "achieved_gmul_s": round(am / ks / 1e9, 2), "alu_frac": round(fa, 4),
                "achieved_gbs": round(ab / ks / 1e9, 1), "hbm_frac": round(fh, 4),
                "bound": "alu" if fa >= fh else "hbm",
                "peak": "the multiply rate measured live (rr_bench_gf_mul) and the measured copy bandwidth"}
    return {"workload": f"{nq} queries on the n=100000 m=1000000 graph with 8 colours, "
                        "k~U{4..12}, odd queries coloured (motif = source colour + k-1 uniform)",
            "queries_per_s": nq / t_batch, "value": units / t_batch, "unit": UNIT,
            "autotuned_shape": tuned, "autotune_s": round(tune_s, 2),
            "automatic_shape_queries_per_s": nq / t_auto,
            "one_query_per_launch_queries_per_s": nq / t_single,
            "one_query_per_launch_value": units / t_single,
            "speedup": t_single / t_batch, "bit_exact_vs_single": same,
            "roofline": roof,
            "launches": "1 persistent kernel (+ z-table, first-layer and bitmap prologue/epilogue)"}


def served_metrics(capi, g, nq=160, seed=UNIFORM_SEED ^ 0x5E,
                   workload="plain queries, k~U{6..12}, s~U, on the n=100000 m=1000000 graph",
                   warm=8, batching_probe=True):
    """Serving: Poisson arrivals of plain queries (s ~ U, k ~ U{6..12}) at 0.5x,
    0.8x and 1.1x of the server's measured capacity; latency = submit -> done.
    Warm-up: `warm` queries one at a time, then one untimed burst (every slot
    captures its launch sequences). Capacity = a burst of the whole list on the
    server's default (4 slots, batch lanes off); with batching_probe the same
    burst is also timed with batches of up to 64 queries. The same query list is
    then run one query at a time through rr_reach_sync (the plain GPU form:
    one launch sequence per query, results copied to the host), host-timed."""
    import threading
    rng = np.random.default_rng(seed)
    n = g["n"]
    qs = [(int(rng.integers(0, n)), int(rng.integers(6, 13)), int(rng.integers(1, 2**62)))
          for _ in range(nq)]
    out = {"workload": workload, "slots": 4, "queries_per_level": nq}
    with capi.Graph(g) as G:
        srv = capi.rr_server_create(G.handle, 0, 4)
        try:
            for s_, k_, sd in qs[:warm]:  # warm-up: capture each slot's graphs
                capi.rr_query_poll(srv, capi.rr_query_submit(srv, s_, k_, sd), n, -1)
            for t in [capi.rr_query_submit(srv, s_, k_, sd) for s_, k_, sd in qs[:64]]:
                capi.rr_query_poll(srv, t, n, -1)
            a0 = capi.rr_server_stats(srv)
            t0 = time.perf_counter()
            ts = [capi.rr_query_submit(srv, s_, k_, sd) for s_, k_, sd in qs]
            for t in ts:
                capi.rr_query_poll(srv, t, n, -1)
            cap = nq / (time.perf_counter() - t0)
            out["capacity_queries_per_s"] = cap
            a1 = capi.rr_server_stats(srv)
            out["capacity_admission"] = {"single": a1[0] - a0[0], "batched": a1[1] - a0[1],
                                         "batches": a1[2] - a0[2]}
            if batching_probe:
                # the same burst with the batch lanes on (the server's default is
                # off: the slots' concurrent launch sequences), untimed warm burst first
                capi.rr_server_set_batching(srv, 8, 64)
                for t in [capi.rr_query_submit(srv, s_, k_, sd) for s_, k_, sd in qs[:64]]:
                    capi.rr_query_poll(srv, t, n, -1)
                t0 = time.perf_counter()
                ts = [capi.rr_query_submit(srv, s_, k_, sd) for s_, k_, sd in qs]
                for t in ts:
                    capi.rr_query_poll(srv, t, n, -1)
                out["capacity_with_batches_of_up_to_64_queries_per_s"] = nq / (time.perf_counter() - t0)
                capi.rr_server_set_batching(srv, 0, 0)
                a1 = capi.rr_server_stats(srv)
            loads = []
            for frac in (0.5, 0.8, 1.1):
                rate = frac * cap
                gaps = rng.exponential(1.0 / rate, size=nq)
                tickets = []
                lock = threading.Lock()

                def poller():
                    i = 0
                    while i < nq:
                        with lock:
                            have = len(tickets)
                        if i < have:
                            capi.rr_query_poll(srv, tickets[i], n, -1)
                            i += 1
                        else:
                            time.sleep(0.0002)
                th = threading.Thread(target=poller)
                th.start()
                t_start = time.perf_counter()
                nxt = t_start
                for (s_, k_, sd), gap in zip(qs, gaps):
                    nxt += gap
                    while time.perf_counter() < nxt:
                        pass
                    t = capi.rr_query_submit(srv, s_, k_, sd)
                    with lock:
                        tickets.append(t)
                th.join()
                wall = time.perf_counter() - t_start
                lat = np.array([capi.rr_query_times(srv, t)[1] for t in tickets]) / 1e3
                loads.append({"offered_frac": frac, "offered_queries_per_s": rate,
                              "queries_per_s": nq / wall, "p50_ms": float(np.percentile(lat, 50)),
                              "p99_ms": float(np.percentile(lat, 99))})
            out["loads"] = loads
            a2 = capi.rr_server_stats(srv)
            out["loads_admission"] = {"single": a2[0] - a1[0], "batched": a2[1] - a1[1],
                                      "batches": a2[2] - a1[2]}
        finally:
            capi.rr_server_destroy(srv)
        # the identical query list, one query at a time (pinned host outputs)
        import torch
        h_bm = torch.empty((n + 7) // 8, dtype=torch.uint8, pin_memory=True).numpy()
        h_w = torch.empty(n, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
        for s_, k_, sd in qs[:warm]:
            G.reach(s_, k_, sd, out=(h_bm, h_w))
        t0 = time.perf_counter()
        for s_, k_, sd in qs:
            G.reach(s_, k_, sd, out=(h_bm, h_w))
        one = nq / (time.perf_counter() - t0)
    out["one_query_at_a_time_queries_per_s"] = one
    out["one_query_at_a_time_api"] = "rr_reach_sync per query, same list, pinned host outputs"
    out["capacity_over_one_at_a_time"] = out["capacity_queries_per_s"] / one
    for lv in out["loads"]:
        lv["over_one_at_a_time"] = lv["queries_per_s"] / one
    out["note"] = ("below saturation the delivered rate equals the offered rate; capacity (a burst "
                   "of the whole list) is the served form's throughput")
    return out


def gf_mul_peak(capi, torch):
    """Measured peak rate of the device GF(2^64) multiply (multiplications/s):
    the rr_bench_gf_mul microbenchmark (register-only chains, four independent
    products a step, every operand value entering exactly one product as in the
    layer kernels) over the whole GPU, timed with CUDA events."""
    st = torch.cuda.Stream()
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    capi.rr_bench_gf_mul(sms * 8, 256, 64, sink, st.cuda_stream)
    st.synchronize()
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        mults = capi.rr_bench_gf_mul(sms * 8, 256, 2048, sink, st.cuda_stream)
        e1.record(st)
        st.synchronize()
        best = max(best, mults / (e0.elapsed_time(e1) / 1e3))
    return best


def kernel_rooflines(info, k, chunk, ppl, n, kt, queries, hbm_peak, mul_peak, ztable_mults=0):
    """Per kernel kind of the reduced-state engine: average launch time (from
    the library's CUDA-event timing of `queries` queries), algorithmic bytes and
    GF(2^64) multiplications per launch, and the fractions of the measured HBM
    copy bandwidth and of the measured multiply rate; `bound` is the larger."""
    S = info["producer_window_rows"]   # state rows (label-space layer 2)
    D = info["state_compute_rows"]     # deep rows: per-point state of layers >= 3
    DC = info["deep_compute_rows"]     # deep rows that multiply at layers >= 4
    T3 = info["deep_tail_rows"]        # last-layer rows
    P = info["state_rows"]             # rows of the scalar layer-1 prefix
    c = chunk
    lg = 7 if ppl == 4 else 6
    rstride = c // (32 * ppl) * (lg + 1)
    R3 = info["deep_head_runs"]        # head runs over the deep rows' ranges
    pmode = 1 if info["pair_layer3_min_k"] <= k <= 20 else 0
    NP = k * (k + 1) // 2
    # layers >= 4 read two state rows per window and multiply once per point
    mid = (D * c * 8 + 2 * DC * c * 8 + D * 20, DC * (c + k))
    third = None
    table = bool(info.get("head_table")) and pmode == 1
    HD = info.get("deep_heads", 0)
    nchunks = max(1, (1 << k) // c)
    if pmode:
        # per query: layer 3 in pair-label space (2k label-space values in,
        # k(k+1)/2 pair values out per deep row; k + k^2 products per row) and,
        # with the head table, x_h x_s for every deep-row head and point of
        # every chunk; the same timing kind, so per launch = per query / launches
        third = (D * (NP * 8 + 2 * k * 8 + 20) + (HD * c * 8 * nchunks if table else 0),
                 D * (k + k * k) + (HD * c * nchunks if table else 0))
    ng = c // (32 * ppl)               # point groups of a chunk
    # the pair tail: layers k-2 and k-1 from layer k-3's sums over one- and
    # two-label point sets (kernels: per-point layers up to k-3, then layer k-2
    # in label space with 16-value rows)
    ptail = bool(info.get("pair_tail")) and k >= (7 if pmode else 6) and ng <= 8
    ns = 1 + lg + lg * (lg - 1) // 2   # used values of a group's 32-value block
    tail_out = ng * 32 if ptail else rstride  # values the last per-point layer stores per row
    last_pp = k - 3 if ptail else k - 2
    if pmode == 1:
        # layer 4 reads 2 NP pair values per window and multiplies per point by
        # c and by x_u x_s (from the head table: 8 more bytes per point; else
        # formed here: one more product)
        l4 = ((D * c * 8 + 2 * DC * NP * 8 + D * 20 + DC * c * 8, DC * (2 * c + k)) if table else
              (D * c * 8 + 2 * DC * NP * 8 + D * 20, DC * (3 * c + k)))
        mids = [l4] + [mid] * (last_pp - 5) if last_pp >= 5 else []
        tail = ((D * tail_out * 8 + l4[0] - D * c * 8, l4[1]) if last_pp == 4 else
                (D * tail_out * 8 + 2 * DC * c * 8 + D * 20, DC * (c + k)))
    else:
        # layer 3 per point from the label-space prefix: x_u times y rho for every
        # row, x_v x_s once per head run and once per row
        l3 = (D * c * 8 + 2 * D * k * 8 + D * 20, D * (k + 2 * c) + R3 * c)
        mids = [l3] + [mid] * (last_pp - 4) if last_pp >= 4 else []
        tail = ((D * tail_out * 8 + 2 * D * k * 8 + D * 20, D * (k + 2 * c) + R3 * c) if last_pp == 3 else
                (D * tail_out * 8 + 2 * DC * c * 8 + D * 20, DC * (c + k)))
    if mids:
        mid_avg = (sum(x[0] for x in mids) / len(mids), sum(x[1] for x in mids) / len(mids))
    else:
        mid_avg = mid
    if ptail:
        # layer k-2 reads the used values of both window ends' blocks and keeps
        # 16 values per deep row; per row with a window: lg + ng y-scaled
        # multipliers, lg^2 products over the pair and single sums summed over
        # the groups, 2 lg ng over the groups' single sums, ng over their totals
        label_tail = (2 * DC * ng * ns * 8 + D * 16 * 8 + D * 20,
                      DC * (lg + ng + lg * lg + 2 * lg * ng + ng))
        last = (2 * T3 * (lg + ng) * 8 + T3 * 16 + n * 8, T3 * (lg + ng))
    else:
        last = (2 * T3 * rstride * 8 + T3 * 16 + n * 8, T3 * rstride)
    alg = {
        "first_layer": (P * 8 + P * 12, 0),
        "second_layer": (S * k * 8 + S * 20 + 2 * S * 8, S * (1 + k)),
        "mid_layer": mid_avg,
        "tail_layer": tail,
        "last_layer": last,
        "ztable": (n * k * 8, ztable_mults),
    }
    if ptail:
        alg["label_tail_layer"] = label_tail
    if third is not None:
        per_query = kt.get("third_layer", (0, 0))[1] / queries
        if per_query:
            alg["third_layer"] = (third[0] / per_query, third[1] / per_query)
    out = {}
    for name, (kms, kn) in kt.items():
        if not kn or name not in alg:
            continue
        avg_s = kms / kn / 1e3
        b, mu = alg[name]
        gbs = b / avg_s / 1e9
        gms = mu / avg_s / 1e9
        fh, fa = gbs / hbm_peak, gms / (mul_peak / 1e9)
        out[name] = {"avg_launch_us": round(avg_s * 1e6, 2), "launches_per_query": kn / queries,
                     "alg_bytes_per_launch": int(b), "achieved_gbs": round(gbs, 1),
                     "hbm_frac": round(fh, 4), "alg_gf_mults_per_launch": int(mu),
                     "achieved_gmul_s": round(gms, 2), "alu_frac": round(fa, 4),
                     "bound": "alu" if fa >= fh else "hbm", "time_ms_per_query": round(kms / queries, 4)}
    return out


def atmost_metrics(capi, torch, g, k=10, reps=5, source=0):
    """at-most-k (the exact-k' queries for k' = 2..k, run concurrently) against
    the exact-k query on the benchmark graph. The paper's experiments report the
    ratio of the two runtimes (column 4 of its scalability tables; below 2 on
    most graphs), which the nominal work sum_{k'} k' 2^k' / (k 2^k) predicts."""
    n, m = g["n"], len(g["src"])
    with capi.Graph(g) as G:
        st = torch.cuda.Stream()
        d_w = torch.zeros((k - 1, n), dtype=torch.int64, device="cuda")
        d_bm = torch.zeros((n + 7) // 8, dtype=torch.uint8, device="cuda")
        capi.rr_reach_atmost_device(G.handle, source, k, 1, d_w, d_bm, st.cuda_stream)
        capi.rr_reach_device(G.handle, source, k, 1, d_w[0], None, st.cuda_stream)
        st.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        with torch.cuda.stream(st):
            e[0].record(st)
            for i in range(reps):
                capi.rr_reach_atmost_device(G.handle, source, k, 2 + i, d_w, d_bm, st.cuda_stream)
            e[1].record(st)
            e[2].record(st)
            for i in range(reps):
                capi.rr_reach_device(G.handle, source, k, 2 + i, d_w[0], None, st.cuda_stream)
            e[3].record(st)
            st.synchronize()
        t_atm = e[0].elapsed_time(e[1]) / reps
        t_exact = e[2].elapsed_time(e[3]) / reps
        # bounded RestlessReach (minimum arrival and shortest length over k' <= k)
        d_r = torch.zeros(n, dtype=torch.int32, device="cuda")
        d_l = torch.zeros(n, dtype=torch.uint8, device="cuda")
        capi.rr_reach_bounded_device(G.handle, source, k, 1, d_r, d_l, d_bm, st.cuda_stream)
        st.synchronize()
        with torch.cuda.stream(st):
            e[0].record(st)
            for i in range(reps):
                capi.rr_reach_bounded_device(G.handle, source, k, 2 + i, d_r, d_l, d_bm, st.cuda_stream)
            e[1].record(st)
            st.synchronize()
        t_bounded = e[0].elapsed_time(e[1]) / reps
    nominal_ratio = sum(kk * 2 ** kk for kk in range(2, k + 1)) / (k * 2 ** k)
    return {"k": k, "atmost_ms": t_atm, "exact_ms": t_exact, "time_ratio": t_atm / t_exact,
            "bounded_ms": t_bounded, "bounded_time_ratio": t_bounded / t_exact,
            "nominal_work_ratio": nominal_ratio,
            "value": sum(2 ** kk * kk * m for kk in range(2, k + 1)) / (t_atm / 1e3), "unit": UNIT}


def fine_metrics(capi, torch, g, k=K_UNIFORM, reps=10):
    """Fine-grained oracle (Algorithm 1 with per-time outputs: per-edge sums,
    minimum arrival time R, set D) against the plain query on the benchmark
    graph and query."""
    n, m = g["n"], len(g["src"])
    with capi.Graph(g) as G:
        st = torch.cuda.Stream()
        d_w = torch.zeros(n, dtype=torch.int64, device="cuda")
        d_e = torch.zeros(m, dtype=torch.int64, device="cuda")
        d_r = torch.zeros(n, dtype=torch.int32, device="cuda")
        d_b = torch.zeros((n + 7) // 8, dtype=torch.uint8, device="cuda")
        for i in range(3):
            capi.rr_reach_arrival_device(G.handle, 0, k, 1 + i, d_w, d_r, d_e, d_b, st.cuda_stream)
            capi.rr_reach_device(G.handle, 0, k, 1 + i, d_w, None, st.cuda_stream)
        st.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        with torch.cuda.stream(st):
            e[0].record(st)
            for i in range(reps):
                capi.rr_reach_arrival_device(G.handle, 0, k, 7 + i, d_w, d_r, d_e, d_b,
                                             st.cuda_stream)
            e[1].record(st)
            e[2].record(st)
            for i in range(reps):
                capi.rr_reach_device(G.handle, 0, k, 7 + i, d_w, None, st.cuda_stream)
            e[3].record(st)
            st.synchronize()
        t_fine = e[0].elapsed_time(e[1]) / reps
        t_plain = e[2].elapsed_time(e[3]) / reps
        R = d_r.cpu().numpy().view(np.uint32)
        # no restless path of 3 or more vertices leaves s on this graph; k = 2
        # shows the arrival-time output on the same source
        capi.rr_reach_arrival_device(G.handle, 0, 2, 1, d_w, d_r, d_e, d_b, st.cuda_stream)
        st.synchronize()
        R2 = d_r.cpu().numpy().view(np.uint32)
    reached = R != 0xFFFFFFFF
    reached2 = R2 != 0xFFFFFFFF
    return {"k": k, "fine_ms": t_fine, "plain_ms": t_plain, "time_ratio": t_fine / t_plain,
            "vertices_with_arrival": int(reached.sum()),
            "vertices_with_arrival_k2": int(reached2.sum()),
            "median_arrival_k2": float(np.median(R2[reached2])) if reached2.any() else None,
            "value": units_per_query(k, m) / (t_fine / 1e3), "unit": UNIT,
            "outputs": "witness S, per-edge sums E (m), minimum arrival R (n), set D"}


def run_reference(args):
    """The oracle as it stands on the headline query: each step evaluates one
    sieve point (a bounded sample; the oracle's work is the same for every
    point) with the host's cores sharing each layer's edges; value scaled by
    points to the nominal unit. Rank 0 only."""
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    g, s, motif = headline_query()
    m = len(g["src"])
    cores = os.cpu_count() or 1
    for i in range(args.warmup):
        oracle.sieve(g, s, K, step_seed(i), motif=motif,
                     masks=np.array([640 + i % 64], dtype=np.uint32), threads=cores)
    times = []
    for i in range(args.steps):
        t0 = time.perf_counter()
        oracle.sieve(g, s, K, step_seed(i), motif=motif,
                     masks=np.array([(640 + 7 * i) % 2 ** K], dtype=np.uint32), threads=cores)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = units_per_query(K, m) / 2 ** K * args.steps / tot
    sample = f"1 of {2 ** K} sieve points per step, {cores} threads sharing each layer's edges"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "graph_seed": GRAPH_SEED, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample + ", scaled by points", "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="headline line only")
    ap.add_argument("--dense", action="store_true", help="dense state layout (every row stored)")
    ap.add_argument("--shape", default=None,
                    help="points per lane x points per chunk (e.g. 4x512) instead of the autotuner; "
                         "profiling runs pin the shape the autotuner picks without a profiler")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2010_08423_gb300 import capi, shard

    rank, world, local_rank = env_rank()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    capi.load()

    g, s, motif = headline_query()
    m, n = len(g["src"]), g["n"]
    t0 = time.perf_counter()
    G = capi.Graph(g, capi.FLAG_DENSE_STATE if args.dense else 0)
    load_s = time.perf_counter() - t0
    info = G.info()
    if args.shape:
        ppl, chunk = (int(x) for x in args.shape.lower().split("x"))
        capi.rr_set_tuning(G.handle, K, ppl, chunk)
    else:
        ppl, chunk = capi.rr_autotune(G.handle, K)
    first, count = shard.point_range(K, rank, world)

    stream = torch.cuda.Stream()
    d_w = torch.empty(n, dtype=torch.int64, device="cuda")
    d_bm = torch.empty((n + 7) // 8, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")

    def step(i):
        if world == 1:
            capi.rr_reach_device(G.handle, s, K, step_seed(i), d_w, d_bm, stream.cuda_stream,
                                 motif=motif)
        else:
            # this rank's sieve points, then the parts all-gathered and XOR-combined
            shard.reach_sharded(G.handle, n, s, K, step_seed(i), d_w, motif=motif, stream=stream)

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            step(i)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        sampler = ClockSampler(local_rank)
        sampler.start()
        sampler.wait_first()
        # untimed steps of the same query under the sampler
        t_load = time.perf_counter() + 0.4
        j = 0
        while time.perf_counter() < t_load:
            step(1_000_000 + j)
            j += 1
            stream.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        launches0 = capi.rr_kernel_launches()
        for i in range(args.steps):
            flush.fill_(i)  # evict L2 between steps (outside the timed events)
            evs[i][0].record(stream)
            step(args.warmup + i)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        launches = capi.rr_kernel_launches() - launches0
        clocks = sampler.stop()
    reach = int((d_w != 0).sum().item())
    # profiling pass (not timed above): per-kernel CUDA-event durations recorded
    # by the library on the launching stream, this rank's share of the points
    kt = kernel_times(capi, torch, stream,
                      lambda i: capi.rr_reach_range_device(G.handle, s, K, step_seed(10_000 + i), first,
                                                           count, d_w, stream.cuda_stream, motif),
                      2)
    ms = [a.elapsed_time(b) for a, b in evs]
    tot_ms = sum(ms)
    if dist:
        t = torch.tensor([tot_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    units = units_per_query(K, m)
    value = args.steps * units / (tot_ms / 1e3)  # one whole query per step for the job

    # end to end through the host-buffer API: rr_reach_sync (results copied back
    # every step into pinned host buffers allocated once); sharded: the rank's
    # range, the exchange and the combined witness copied to the host
    h_bm = torch.empty((n + 7) // 8, dtype=torch.uint8, pin_memory=True).numpy()
    h_w = torch.empty(n, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    h_wt = torch.from_numpy(h_w.view(np.int64))

    def e2e_step(i):
        if world == 1:
            G.reach(s, K, step_seed(i), motif=motif, out=(h_bm, h_w))
        else:
            full = shard.reach_sharded(G.handle, n, s, K, step_seed(i), d_w, motif=motif,
                                       stream=stream)
            h_wt.copy_(full)
    for i in range(2):
        e2e_step(2000 + i)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e2e_s = 0.0
    for i in range(args.steps):
        flush.fill_(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step(3000 + i)
        e2e_s += time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = args.steps * units / e2e_s

    peaks, peak_kind = measured_peaks()
    mul_peak = gf_mul_peak(capi, torch)
    by_kernel = {} if args.dense else kernel_rooflines(
        info, K, chunk, ppl, n, kt, 2, peaks["hbm_gbs"], mul_peak,
        ztable_mults=motif_ztable_mults(g, motif, K))
    roofline = dominant_roofline(by_kernel, kt, mul_peak, peaks["hbm_gbs"], peak_kind,
                                 lambda kern: recorded_traffic("motif", kern, ppl, chunk))
    tot_k = max(1e-9, sum(v[0] for v in kt.values()))
    kernel_share = {k_: round(v[0] / tot_k, 4) for k_, v in kt.items() if v[1]}
    ms_per_step = tot_ms / args.steps

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "graph_seed": GRAPH_SEED, "source": s, "k": K,
                       "motif": [int(c) for c in motif], "l2": "flushed between steps",
                       "state_layout": "dense" if args.dense else "compact",
                       "points_per_lane": ppl, "points_per_chunk": chunk,
                       "parallelism": "single GPU" if world == 1 else
                       f"sieve points split over {world} ranks, partial witnesses all-gathered "
                       "and XOR-combined every step",
                       "rank0_points": [first, count],
                       "state_rows": info["producer_window_rows"] + 1,
                       "deep_rows": info["state_compute_rows"],
                       "deep_compute_rows": info["deep_compute_rows"],
                       "last_layer_rows": info["deep_tail_rows"],
                       "producer_rows": info["state_rows"] - 1, "window_rows": info["window_rows"],
                       "max_in_degree": info["max_in_degree"],
                       "pair_layer3": info["pair_layer3_min_k"] <= K, "head_table": info["head_table"],
                       "graph_load_s": round(load_s, 3), "reachable_vertices": reach},
            "work": work_accounting(by_kernel, K, m, info, ms_per_step) if by_kernel else None,
            "roofline": roofline,
            "roofline_by_kernel": by_kernel,
            "kernel_time_share": kernel_share,
            "kernel_ms_per_query": round(tot_k / 2, 4),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": DESC_BYTES,
                    "d2h_bytes_per_step": n * 8 + ((n + 7) // 8 if world == 1 else 0),
                    "api": "rr_reach_sync (pinned host outputs, query descriptor uploaded per step)"
                           if world == 1 else "shard.reach_sharded + witness copied to pinned host memory"},
            "gpu_launches": int(launches), "clocks": clocks,
            "parity": "tests/test_gpu_scale_parity.py: sieve points 640..703 of this query on this "
                      "graph, autotuned shape, bit-exact vs the oracle"}
    if world > 1:
        line["work"] = None  # per-rank kernel counts cover one share of the points
    G.close()
    if rank == 0 and not args.no_extra:
        line["uniform_k8"] = uniform_metrics(capi, torch, W.scale_uniform(), mul_peak,
                                             peaks["hbm_gbs"], peak_kind)
        line["dense"] = dense_metrics(capi, torch, g, s, motif, mul_peak, peaks["hbm_gbs"], peak_kind)
        line["dense"]["compact_over_dense"] = line["dense"]["ms_per_query"] / ms_per_step
        line["small"] = small_metrics(capi, torch)
        # at-most-k where the k query's layers are long: the smaller queries
        # come from its own layers (plain k = 10 from the headline source)
        line["atmost_k_powerlaw"] = atmost_metrics(capi, torch, g, source=s)
        line["atmost_k_powerlaw"]["workload"] = ("plain k-RestlessReach from the headline source on the "
                                                 "Chung-Lu n=1e6 m=1e7 graph")
        gu = W.scale_uniform()
        line["batched"] = batched_metrics(capi, torch, W.scale_uniform(ncolors=8), mul_peak,
                                          peaks["hbm_gbs"])
        line["served"] = served_metrics(capi, gu)
        line["atmost_k"] = atmost_metrics(capi, torch, gu)
        line["fine_grained"] = fine_metrics(capi, torch, gu)
        del gu
        g5 = W.served_powerlaw()
        line["served_powerlaw"] = served_metrics(
            capi, g5, nq=100, seed=W.GRAPH_SEED_BASE + 5, warm=4, batching_probe=False,
            workload="plain queries, k~U{6..12}, s~U, on the Chung-Lu exponent 2.3 graph "
                     "n=1e7 m=1e8 t~U[1,1e5] delta~U{10..200}")
        del g5
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, s, motif)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
