#!/usr/bin/env python
"""Benchmark of the theta-join engine on the 1.07M-node road-like workload.

One step = one whole query: validate R and S, build the S bitmap, list R, search every
source (by default one warp per source, delta-stepping in a shared-memory map), emit the
pairs within theta and put them in (u, v) order.  The workload is the 1.07M-node,
2.7M-edge road-like graph with 50,000 + 50,000 clustered R and S nodes and theta for
about 50 S-matches per R node (2.8M pairs).  The headline ``value`` is join pairs/s
with R and S already in device memory (CUDA events on the query stream, L2 flushed
between steps); ``e2e`` is the same metric through the host-buffer call, with the
copies of R and S to the device and of the pairs back to the host inside the timed
region.  Secondary legs: the 264k-node join, k closest pairs on the 1.07M-node graph,
512 batched joins against plain calls, and a served request stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl engine|reference]

Under torchrun (N > 1) every rank joins its own R and S (same sizes, other seeds) over
the same graph -- weak scaling with no collective on the data path; rank 0 prints the
line, with the slowest rank's time.  ``--impl reference`` times the CPU oracle on every
host core (the paper publishes no code and no absolute numbers to compare against).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "join pairs/s"
UNIT = "pairs/s"
WORKLOADS = json.load(open(os.path.join(ROOT, "tests", "golden", "workloads.json")))
ENGINE_SRC = os.path.join(ROOT, "paper_1607_07696_gb300", "csrc", "rn_engine.cu")
PROFILES = {"road1070k_join": os.path.join(ROOT, "profiles", "search_road1070k.json"),
            "road1070k_kcp_k1000000": os.path.join(ROOT, "profiles", "search_road1070k_kcp.json")}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--workload", default="road1070k_join",
                    choices=["road264k_join", "grid4096_theta1500", "road1070k_join"])
    ap.add_argument("--tile-width", type=int, default=0)
    ap.add_argument("--delta", type=int, default=0)
    ap.add_argument("--tile-sources", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-instance batched leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-hier", action="store_true", help="skip the hierarchical-variant leg")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--no-legs", action="store_true",
                    help="only the headline workload: no secondary legs and no CPU baseline")
    ap.add_argument("--leg", default="", choices=["", "kcp_1m", "batched", "join_264k", "hierarchical", "served",
                                                  "large_balls"],
                    help="run this one secondary leg alone (one GPU) and print its JSON object")
    return ap.parse_args()


def make_workload(name: str, rank: int):
    from paper_1607_07696_gb300 import inputs as I

    if name == "road264k_join":
        spec = WORKLOADS["road264k_join"]
        w = I.c2_road_join(spec["theta"])
        if rank:
            w.R, w.S = I.disjoint_sets(w.graph.n, len(w.R), len(w.S), I.BASE_SEED + 1000 + 7919 * rank)
        return w, spec
    if name == "grid4096_theta1500":
        spec = WORKLOADS["grid4096_theta1500"]
        w = I.c1_grid_join()
        if rank:
            w.R, w.S = I.disjoint_sets(w.graph.n, len(w.R), len(w.S), I.BASE_SEED + 7919 * rank)
        return w, spec
    spec = dict(WORKLOADS["road1070k_clustered"])
    w = I.c3_road_clustered(theta=spec["theta_join"])
    spec["theta"] = spec["theta_join"]
    if rank:
        w.R, w.S = I.clustered_sets(w.graph.xy, len(w.R), len(w.S), I.BASE_SEED + 3000 + 7919 * rank)
    return w, spec


# ------------------------------------------------------------------ clocks ----

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers ----

def measured_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def graph_digest(e) -> dict:
    import numpy as np

    return {"n": int(e.n), "m": int(e.m), "wsum": int(e.w.astype(np.uint64).sum()),
            "xsum": int((e.src.astype(np.uint64) * 3 + e.dst.astype(np.uint64)).sum())}


def algorithmic_bytes(st: dict, pairs: int) -> float:
    """Bytes the search must move, summed over tiles (a source alone is a tile of one
    lane): 8 per reached node (CSR offsets) and per arc leaving it (column, weight), 8
    per node and lane (its distance written, then read at emission), a bit per node (S
    membership) and 12 per pair."""
    return (8 * st["slots"] + 8 * st["slot_arcs"] + 8 * st["slot_lanes"] + st["slots"] / 8
            + 12 * pairs)


def search_kernel(st: dict) -> str:
    return "k_source_search" if st["tile_width"] == 1 else "k_tile_search"


def engine_hash() -> str:
    """Hash of the engine source's warp-search section (`k_source_search` and its device
    helpers: the kernel the committed ncu summaries profile)."""
    src = open(ENGINE_SRC).read()
    a = src.index("// ----------------------------------------------------------- source search ----")
    b = src.index("// ---------------------------------------------------- cooperative source search ----")
    return hashlib.sha256(src[a:b].encode()).hexdigest()[:16]


def profile_of(workload: str, kernel: str):
    """The committed ncu summary of the search kernel on this workload, or None when there
    is none, it covers another kernel or the kernel source changed since."""
    path = PROFILES.get(workload)
    if not path or not os.path.exists(path):
        return None
    p = json.load(open(path))
    if (p.get("workload") != workload or p.get("engine_sha") != engine_hash()
            or not str(p.get("kernel", "")).startswith(kernel)):
        return None
    return p


def roofline(st: dict, pairs: int, search_ms: float, workload: str, peak: float, peak_kind: str) -> dict:
    """HBM roofline of the search kernel: algorithmic bytes per launch over its CUDA-event
    time, against the measured copy bandwidth; beside it, from the committed ncu summary
    of the same kernel and workload (when current), its DRAM traffic per launch and its
    L2 traffic per launch over the same time against the L2 peak ncu reports."""
    alg = algorithmic_bytes(st, pairs)
    achieved = alg / (search_ms / 1e3) / 1e9
    kernel = search_kernel(st)
    prof = profile_of(workload, kernel)
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": prof.get("dram_bytes_per_launch") if prof else None, "kernel": kernel,
           "peak_kind": peak_kind, "search_ms": search_ms, "alg_bytes_per_launch": alg}
    if prof and prof.get("l2_bytes_per_launch") and prof.get("l2_peak_gbs"):
        l2 = prof["l2_bytes_per_launch"] / (search_ms / 1e3) / 1e9
        out["l2"] = {"achieved": l2, "peak": prof["l2_peak_gbs"], "unit": "GB/s",
                     "frac": l2 / prof["l2_peak_gbs"], "bytes_per_launch": prof["l2_bytes_per_launch"],
                     "peak_kind": "ncu lts__t_bytes peak"}
    return out


def cpu_baseline(w, spec) -> dict:
    """The CPU oracle, as it stands, on the whole workload: its per-source searches on
    every host core (R in chunks, one search state per thread), then on one core."""
    from oracle import oracle as O

    og = O.default().graph(w.graph.n, w.graph.src, w.graph.dst, w.graph.w)
    cores = O.host_cores()
    t0 = time.perf_counter()
    p = og.join_mt(w.R, w.S, spec["theta"], cores)
    dt = time.perf_counter() - t0
    t0 = time.perf_counter()
    p1 = og.join(w.R, w.S, spec["theta"])
    dt1 = time.perf_counter() - t0
    assert len(p1) == len(p), "threaded and single-thread oracle disagree"
    return {"value": len(p) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the whole workload: all {len(w.R)} R sources against all {len(w.S)} S nodes, "
                      f"theta {spec['theta']}, {len(p)} pairs; {dt:.2f} s on {cores} threads, "
                      f"{dt1:.2f} s on one",
            "single_core_value": len(p1) / dt1, "cpu_model": O.cpu_model()}


# ------------------------------------------------------------------- engine ----

def batch_leg(rn, steps: int, warmup: int, stream, flush) -> dict:
    """512 independent theta-joins (1k-50k-node graphs, uneven |R| and |S|, per-instance
    theta): pairs/s of the whole batch run as one autotuned, graph-replayed batch, as a
    batch with the default plan, and as 512 plain one-query calls in a row, all with the
    sets already in device memory and L2 flushed before every timed run."""
    import numpy as np
    import torch

    from paper_1607_07696_gb300 import inputs as I

    specs = I.c4_batch_specs()
    thetas = WORKLOADS["batch512"]["theta"]
    qs, dev = [], []
    for sp, th in zip(specs, thetas):
        e, R, S = I.c4_instance(sp)
        g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
        qs.append((g, R, S, th))
        dev.append((torch.as_tensor(R.astype(np.int32), device="cuda"),
                    torch.as_tensor(S.astype(np.int32), device="cuda")))

    def timed(fn) -> float:
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for i in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xFF)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    out = rn.DevicePairs()
    plain_pairs = [0]

    def plain():
        tot = 0
        for (g, R, S, th), (dR, dS) in zip(qs, dev):
            tot += rn.rn_distance_join_dev(g, dR, dS, th, out, stream)
        plain_pairs[0] = tot

    plain_ms = timed(plain)
    plain_launches = 0
    for (g, R, S, th), (dR, dS) in zip(qs[:1], dev[:1]):
        rn.rn_distance_join_dev(g, dR, dS, th, out, stream)
        plain_launches = rn.rn_last_query_stats()["launches"] * len(qs)

    b0 = rn.rn_batch_create(qs)
    default_ms = timed(lambda: rn.rn_batch_run(b0, stream))
    s0 = rn.rn_batch_stats_get(b0)
    t0 = time.perf_counter()
    b1 = rn.rn_batch_create(qs, autotune=True)
    rn.rn_batch_run(b1, stream)
    tune_s = time.perf_counter() - t0
    tuned_ms = timed(lambda: rn.rn_batch_run(b1, stream))
    s1 = rn.rn_batch_stats_get(b1)
    pairs = int(s1["pairs"])
    assert pairs == plain_pairs[0] == int(s0["pairs"]), "batched and plain pair counts differ"
    res = {
        "workload": "batch512: 512 theta-joins, n 1k-50k log-uniform, |R|,|S| 64-4096",
        "instances": len(qs), "nodes": int(sum(q[0].n for q in qs)), "pairs": pairs,
        "unit": UNIT,
        "batched": pairs / (tuned_ms / 1e3), "batched_ms": tuned_ms,
        "batched_default_plan": pairs / (default_ms / 1e3), "batched_default_ms": default_ms,
        "plain": pairs / (plain_ms / 1e3), "plain_ms": plain_ms,
        "batched_vs_plain": plain_ms / tuned_ms,
        "gteps_batched": WORKLOADS["batch512"]["alg_arcs"] / (tuned_ms / 1e3) / 1e9,
        "gteps_plain": WORKLOADS["batch512"]["alg_arcs"] / (plain_ms / 1e3) / 1e9,
        "gteps_basis": "arcs of searches from every R node (the paper's method, counted by the oracle); "
                       "searching from the smaller set the engine relaxes fewer",
        "tiles": int(s1["tiles"]), "groups": int(s1["groups"]), "graph_runs": int(s1["graph_runs"]),
        "launches_per_run": int(s1["launches_per_run"]), "plain_launches": int(plain_launches),
        "autotune_s": tune_s, "default_plan_groups": int(s0["groups"]),
        "tuned": {1: f"one plan for all (tile width {int(s1['plan_tile_width'])}, buckets of "
                     f"{int(s1['plan_delta_mult'])} median weights, {int(s1['plan_tile_sources'])} sources "
                     f"per tile)",
                  2: "plan per size class", 3: "the default plans (warp search for small balls, tiles of 8 "
                                               "sources for large)"}.get(int(s1["tuned"]), "no"),
    }
    del b0, b1
    return res


def join_264k_leg(rn, steps: int, stream, flush, peak: float, peak_kind: str) -> dict:
    """The theta-join on the 264k-node road-like graph with 10,000 + 10,000 uniform sets
    (theta for about 50 S-matches per R node): pairs/s with device buffers and L2
    flushed, GTEPS, and the search's roofline against the same measured HBM peak."""
    import numpy as np
    import torch

    spec = WORKLOADS["road264k_join"]
    w, _ = make_workload("road264k_join", 0)
    e = w.graph
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    dR = torch.as_tensor(w.R.astype(np.int32), device="cuda")
    dS = torch.as_tensor(w.S.astype(np.int32), device="cuda")
    out = rn.DevicePairs()
    theta = spec["theta"]
    for _ in range(3):
        rn.rn_distance_join_dev(g, dR, dS, theta, out, stream)
    ms, search = [], []
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            n = rn.rn_distance_join_dev(g, dR, dS, theta, out, stream)
            b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
        st = rn.rn_last_query_stats()
        search.append(st["search_ms"] + st["retry_ms"])
    med = statistics.median(ms)
    return {"workload": "road264k_join: 264k nodes, 730k edges, |R| = |S| = 10,000 uniform",
            "theta": theta, "pairs": int(n), "value": n / (med / 1e3), "unit": UNIT,
            "ms_per_join": med, "gteps": spec["alg_arcs"] / (med / 1e3) / 1e9,
            "launches": int(st["launches"]), "retried_tiles": st["retried_tiles"],
            "roofline": roofline(st, n, statistics.mean(search), "road264k_join", peak, peak_kind)}


def large_balls_leg(rn, steps: int, stream, flush, peak: float, peak_kind: str) -> dict:
    """The θ-join on the 1.07M-node graph at a θ whose balls hold about 3,300 nodes (near
    the serving stream's: 4096- and 8192-slot maps, searched by four or eight warps per
    source), from
    the first 5,000 of the clustered R nodes against all 50,000 S nodes: pairs/s and the
    cooperative search's roofline."""
    import numpy as np
    import torch

    from paper_1607_07696_gb300 import inputs as I

    w = I.c3_road_clustered()
    e = w.graph
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n, cfg={"search_from": rn.RN_FROM_R})
    R = w.R[:5000]
    dR = torch.as_tensor(R.astype(np.int32), device="cuda")
    dS = torch.as_tensor(w.S.astype(np.int32), device="cuda")
    out = rn.DevicePairs()
    theta = 340_000
    for _ in range(3):
        rn.rn_distance_join_dev(g, dR, dS, theta, out, stream)
    ms, search = [], []
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            n = rn.rn_distance_join_dev(g, dR, dS, theta, out, stream)
            b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
        st = rn.rn_last_query_stats()
        search.append(st["search_ms"] + st["retry_ms"])
    med = statistics.median(ms)
    return {"workload": "road1070k_large_balls: 1.07M nodes, |R| = 5,000 of the clustered R, |S| = 50,000, "
                        "theta 340,000 (balls of about 3,300 nodes, a few far larger)",
            "theta": theta, "pairs": int(n), "value": n / (med / 1e3), "unit": UNIT,
            "ms_per_join": med, "max_ball": int(st["max_ball"]),
            "blocks_per_sm": int(st["blocks_per_sm"]), "launches": int(st["launches"]),
            "retried_tiles": int(st["retried_tiles"]),
            "roofline": dict(roofline(st, n, statistics.mean(search), "road1070k_large_balls", peak, peak_kind),
                             kernel="k_source_coop")}


def hier_leg(rn, steps: int) -> dict:
    """The hierarchical variant (searches local to the parts of the partition hierarchy,
    the searches from the far ends of the arcs that leave a part shared by every source,
    min-plus combination) on the 264k-node join, at several part sizes, beside the flat
    warp search on the same graph: device time per join (CUDA events inside the query),
    pairs/s and the phase counters; every result checked equal to the flat join's."""
    import numpy as np

    spec = WORKLOADS["road264k_join"]
    w, _ = make_workload("road264k_join", 0)
    e = w.graph
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    theta = spec["theta"]
    flat = rn.rn_distance_join(g, w.R, w.S, theta)
    fl = []
    for _ in range(steps):
        rn.rn_distance_join(g, w.R, w.S, theta)
        fl.append(rn.rn_last_query_stats()["device_ms"])
    res = {"workload": "road264k_join: 264k nodes, |R| = |S| = 10,000 uniform, theta for ~50 matches",
           "pairs": len(flat[0]), "unit": UNIT, "flat_ms": statistics.median(fl),
           "flat": len(flat[0]) / (statistics.median(fl) / 1e3)}
    for part in (0, 2048, 6000):
        got = rn.rn_distance_join_hier(g, w.R, w.S, theta, part)
        assert all(np.array_equal(x, y) for x, y in zip(got, flat)), f"hierarchical join (parts {part}) differs"
        ms = []
        for _ in range(steps):
            rn.rn_distance_join_hier(g, w.R, w.S, theta, part)
            ms.append(rn.rn_last_query_stats()["device_ms"])
        hs = rn.rn_last_hier_stats()
        med = statistics.median(ms)
        res[f"parts_{part or 'leaves'}"] = {
            "ms": med, "value": len(flat[0]) / (med / 1e3), "vs_flat": statistics.median(fl) / med,
            "parts": hs["parts"], "max_part": hs["max_part"], "local_pairs": hs["local_pairs"],
            "border_routes": hs["border_routes"], "exit_routes": hs["exit_routes"],
            "exit_searches": hs["exit_searches"], "candidates": hs["candidates"],
            "local_ms": hs["local_ms"], "exit_ms": hs["exit_ms"], "combine_ms": hs["combine_ms"]}
    return res


def kcp_1m_leg(rn, steps: int, stream, flush, peak: float, peak_kind: str) -> dict:
    """k closest pairs on the 1.07M-node graph with 50,000 + 50,000 clustered sets, for
    k = 100, 10^4 and 10^6 (unbounded theta): device time per query (sets in device
    memory, L2 flushed), the radius passes it took, the k-th distance, and the roofline
    of the search launch of the last pass (the candidates it emitted, before the
    selection, count as its pairs)."""
    import numpy as np
    import torch

    from paper_1607_07696_gb300 import inputs as I

    w = I.c3_road_clustered()
    e = w.graph
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    dR = torch.as_tensor(w.R.astype(np.int32), device="cuda")
    dS = torch.as_tensor(w.S.astype(np.int32), device="cuda")
    out = rn.DevicePairs()
    res = {"workload": "road1070k_kcp: 1.07M nodes, |R| = |S| = 50,000 clustered, theta unbounded"}
    for k in (100, 10_000, 1_000_000):
        for _ in range(2):
            rn.rn_kcp_dev(g, dR, dS, k, rn.RN_INF, out, stream)
        ms, sms = [], []
        for i in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xFF)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                n = rn.rn_kcp_dev(g, dR, dS, k, rn.RN_INF, out, stream)
                b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
            sms.append(rn.rn_last_query_stats()["search_ms"])
        st = rn.rn_last_query_stats()
        res[f"k={k}"] = {"ms": statistics.median(ms), "pairs": int(n), "passes": st["passes"],
                         "kth_distance": st["theta_final"], "launches": st["launches"],
                         "tile_width": st["tile_width"], "candidates": int(st["search_pairs"]),
                         "roofline": roofline(st, int(st["search_pairs"]), statistics.mean(sms),
                                              f"road1070k_kcp_k{k}", peak, peak_kind)}
    return res


def serve_leg(rn, count: int) -> dict:
    """Serving on the 6M-node graph: a stream of 70% theta-joins and 30% k-closest-pairs
    requests (|R|, |S| 100-20000).  Saturated throughput (every request submitted at
    once), then Poisson arrivals at 50% and 90% of that rate with p50/p99 latency
    (submit to host result), then the same requests one at a time through the plain
    host calls.  Latencies and rates are host wall clock: inputs start and results end
    in host memory."""
    import threading

    from paper_1607_07696_gb300 import inputs as I

    spec = WORKLOADS["serve6m"]
    e = I.c5_serve_graph()
    t0 = time.perf_counter()
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    load_s = time.perf_counter() - t0
    reqs = I.c5_requests(e.n, count, spec["ball_coeff"])
    srv = rn.rn_serve_create(g)
    for r in reqs[:8]:  # warm-up: every worker's buffers
        rn.rn_serve_wait(srv, rn.rn_serve_submit(srv, r.R, r.S, r.theta, r.k))

    def run_stream(arrivals):
        rn.rn_serve_reset_stats(srv)
        tickets = [None] * count
        ready = threading.Semaphore(0)

        def submitter():
            start = time.perf_counter()
            for i, r in enumerate(reqs):
                if arrivals is not None:
                    delay = start + arrivals[i] - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                tickets[i] = rn.rn_serve_submit(srv, r.R, r.S, r.theta, r.k)
                ready.release()

        failure = []

        def guarded_submitter():
            try:
                submitter()
            except BaseException as ex:  # noqa: BLE001 - re-raised in the main thread
                failure.append(ex)
                for _ in range(count):
                    ready.release()

        th = threading.Thread(target=guarded_submitter)
        t0 = time.perf_counter()
        th.start()
        npairs = []
        for i in range(count):
            ready.acquire()
            if failure:
                th.join()
                raise failure[0]
            npairs.append(len(rn.rn_serve_wait(srv, tickets[i])[0]))
        wall = time.perf_counter() - t0
        th.join()
        st = rn.rn_serve_stats_get(srv)
        return wall, st, npairs

    print(f"serve: graph loaded in {load_s:.1f}s, {count} requests", file=sys.stderr, flush=True)
    wall, st, served_pairs = run_stream(None)
    print(f"serve: saturated {count / wall:.1f} q/s", file=sys.stderr, flush=True)
    sat = count / wall
    phases = {"saturated": {"offered_qps": None, "qps": sat, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                            "max_running": st["max_running"], "slab_peak_mb": st["slab_bytes_peak"] / 2**20}}
    for frac in (0.5, 0.9):
        arr = I.poisson_arrivals(count, frac * sat, seed=int(frac * 100))
        wall, st, _ = run_stream(arr)
        phases[f"poisson_{int(frac * 100)}pct"] = {
            "offered_qps": frac * sat, "qps": count / wall, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "mean_queue_ms": st["mean_queue_ms"], "max_running": st["max_running"]}
    srv.close()
    # the plain form: one query per call, one after the other
    t0 = time.perf_counter()
    plain_pairs, plain_dev_ms, kcp_dev_ms = [], 0.0, 0.0
    for r in reqs:
        out = rn.rn_distance_join(g, r.R, r.S, r.theta) if r.k == 0 else rn.rn_kcp(g, r.R, r.S, r.k, r.theta)
        plain_pairs.append(len(out[0]))
        dms = rn.rn_last_query_stats()["device_ms"]
        plain_dev_ms += dms
        kcp_dev_ms += dms if r.k else 0.0
    plain_s = time.perf_counter() - t0
    assert plain_pairs == served_pairs, "served and plain pair counts differ"
    joins = [r for r in reqs if r.k == 0]
    return {
        "workload": "serve6m: 6M-node road-like graph, 70% theta-joins / 30% kCP, |R|,|S| 100-20000, "
                    f"k 10-1e5, {count} requests",
        "unit": "queries/s", "requests": count, "joins": len(joins), "pairs": int(sum(served_pairs)),
        "served_qps": sat, "plain_qps": count / plain_s, "served_vs_plain": sat / (count / plain_s),
        "plain_device_s": plain_dev_ms / 1e3, "plain_kcp_device_s": kcp_dev_ms / 1e3, "plain_wall_s": plain_s,
        "phases": phases, "graph_load_s": load_s,
        "config": {"workers": 8, "max_blocks": "one per SM", "slab_mb": 4096},
    }


def run_engine(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_1607_07696_gb300 import rn

    if not os.path.exists(rn.LIB_PATH):
        from paper_1607_07696_gb300 import build as B

        B.build()
    w, spec = make_workload(args.workload, rank)
    e = w.graph
    cfg = {"tile_width": args.tile_width, "delta": args.delta, "tile_sources": args.tile_sources}
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n, cfg=cfg)
    info = rn.rn_graph_info(g)
    stream = torch.cuda.Stream()
    dR = torch.as_tensor(w.R.astype(np.int32), device="cuda")
    dS = torch.as_tensor(w.S.astype(np.int32), device="cuda")
    out = rn.DevicePairs()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # 256 MB > 129 MB L2
    theta = spec["theta"]

    def step():
        return rn.rn_distance_join_dev(g, dR, dS, theta, out, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times, search_ms, stats = [], [], None
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xFF)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                npairs = step()
                b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
            stats = rn.rn_last_query_stats()
            search_ms.append(stats["search_ms"])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms = sum(times)
    pairs_all = npairs
    if dist:
        from paper_1607_07696_gb300 import shard

        total_ms, pairs_all = shard.job_time_and_pairs(total_ms, npairs, device="cuda")
    value = pairs_all * args.steps / (total_ms / 1e3)

    # end to end through the host-buffer call: R, S in pinned memory, pairs to the host
    Rh = torch.as_tensor(w.R.astype(np.int32)).pin_memory().numpy()
    Sh = torch.as_tensor(w.S.astype(np.int32)).pin_memory().numpy()
    rn.rn_distance_join(g, Rh, Sh, theta)  # warm the host path's buffers
    e2e_t = []
    for i in range(min(50, max(3, args.steps // 2))):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u, v, d = rn.rn_distance_join(g, Rh, Sh, theta)
        e2e_t.append(time.perf_counter() - t0)
    e2e_value = len(u) / statistics.median(e2e_t)
    assert len(u) == npairs

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    T = stats["tile_width"]
    smean = statistics.mean(search_ms)
    peak, peak_kind = measured_peak_gbs()
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": {
            "workload": args.workload,
            "n": e.n, "m": e.m, "nR": len(w.R), "nS": len(w.S), "theta": theta,
            "pairs": npairs, "tile_width": T, "tile_sources": stats["tile_sources"],
            "tiles": stats["tiles"], "delta": stats["delta"],
            "graph_matches_calibration": graph_digest(e) == spec.get("graph"),
            "blocks_per_sm": stats["blocks_per_sm"],
            "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
            "l2": "flushed between steps (256 MB write outside the timed events)",
        },
        "gteps": (spec.get("alg_arcs", 0) / (total_ms / args.steps / 1e3) / 1e9) if spec.get("alg_arcs") else None,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * (len(w.R) + len(w.S)),
                "d2h_bytes_per_step": 12 * npairs},
        "gpu_launches": int(stats["launches"]) * args.steps,
        "roofline": roofline(stats, npairs, smean, args.workload, peak, peak_kind),
        "clocks": clk.summary(),
        "engine": {"reorder_ms": info["reorder_ms"], "slots": stats["slots"],
                   "slot_arcs": stats["slot_arcs"], "scans": stats["scans"],
                   "retried_tiles": stats["retried_tiles"], "device_ms": stats["device_ms"],
                   "rounds": stats["rounds"], "round_items": stats["round_items"],
                   "boundaries": stats["boundaries"], "cycles_rounds": stats["cycles_rounds"],
                   "cycles_boundaries": stats["cycles_boundaries"],
                   "cycles_emission": stats["cycles_emission"],
                   "cycles_step_a": stats["cycles_step_a"], "round_arcs": stats["round_arcs"]},
    }
    legs = world == 1 and not args.no_legs
    if legs and args.workload != "road264k_join":
        line["join_264k"] = join_264k_leg(rn, min(50, max(3, args.steps // 2)), stream, flush, peak, peak_kind)
    if legs:
        line["kcp_1m"] = kcp_1m_leg(rn, min(10, max(3, args.steps // 2)), stream, flush, peak, peak_kind)
    if legs and not args.no_hier:
        line["hierarchical"] = hier_leg(rn, 5)
    if legs and not args.no_batch:
        line["batched"] = batch_leg(rn, 5, 3, stream, flush)
    if legs and not args.no_serve:
        line["served"] = serve_leg(rn, args.serve_requests)
    if legs and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, spec)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------- reference ----

def run_reference(args):
    """The CPU oracle timed on every host core (its per-source searches on one thread per
    core), each step a bounded sample of the same workload: a run of consecutive R
    sources against all of S."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O

    w, spec = make_workload(args.workload, 0)
    og = O.default().graph(w.graph.n, w.graph.src, w.graph.dst, w.graph.w)
    cores = O.host_cores()
    nR = len(w.R)
    per_step = max(100, min(nR, 100_000 // max(1, args.steps)))  # about 100,000 sources in all
    theta = spec["theta"]
    for i in range(args.warmup):
        og.join_mt(w.R[:200], w.S, theta, cores)
    total_pairs, total_s = 0, 0.0
    for i in range(args.steps):
        lo = (i * per_step) % max(1, nR - per_step + 1)
        R = w.R[lo:lo + per_step]
        t0 = time.perf_counter()
        p = og.join_mt(R, w.S, theta, cores)
        total_s += time.perf_counter() - t0
        total_pairs += len(p)
    value = total_pairs / total_s
    world = int(os.environ.get("WORLD_SIZE", "1"))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": args.workload, "n": w.graph.n, "m": w.graph.m, "nR": nR,
                   "nS": len(w.S), "theta": theta, "parallelism": f"{cores} host threads",
                   "l2": "CPU: inputs resident in host memory"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: {per_step} of {nR} R sources against all "
                                   f"{len(w.S)} S nodes", "cpu_model": O.cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_leg(args):
    """One secondary leg alone, for profiling it: prints {"leg": name, ...its figures}."""
    import torch

    from paper_1607_07696_gb300 import rn

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if not os.path.exists(rn.LIB_PATH):
        from paper_1607_07696_gb300 import build as B

        B.build()
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    peak, peak_kind = measured_peak_gbs()
    steps = min(10, max(3, args.steps))
    if args.leg == "kcp_1m":
        res = kcp_1m_leg(rn, steps, stream, flush, peak, peak_kind)
    elif args.leg == "batched":
        res = batch_leg(rn, steps, args.warmup, stream, flush)
    elif args.leg == "join_264k":
        res = join_264k_leg(rn, steps, stream, flush, peak, peak_kind)
    elif args.leg == "hierarchical":
        res = hier_leg(rn, steps)
    elif args.leg == "large_balls":
        res = large_balls_leg(rn, steps, stream, flush, peak, peak_kind)
    else:
        res = serve_leg(rn, args.serve_requests)
    print(json.dumps({"leg": args.leg, **res}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.leg:
        run_leg(args)
    else:
        run_engine(args)


if __name__ == "__main__":
    main()
