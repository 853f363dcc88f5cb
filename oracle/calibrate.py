"""Calibrate the distance threshold theta of the synthetic join workloads with the oracle.

TEST INFRASTRUCTURE: run by hand (``python -m oracle.calibrate``) to (re)write
``tests/golden/workloads.json``.  Only the oracle computes distances here.

For a workload whose theta is meant to give about t S-matches per R node, theta is the
median, over a sample of R nodes, of the distance from that node to its t-th nearest S
node (the oracle's k-closest-pairs search with a single source and k = t).  The graph's
edge count and weight sum are stored beside theta so a run can tell whether it
regenerated the same graph.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1607_07696_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "workloads.json")


def graph_digest(e: I.EdgeList) -> dict:
    return {"n": int(e.n), "m": int(e.m), "wsum": int(e.w.astype(np.uint64).sum()),
            "xsum": int((e.src.astype(np.uint64) * 3 + e.dst.astype(np.uint64)).sum())}


def theta_for_matches(g: O.OGraph, R, S, t: int, sample: int) -> tuple[int, list[int]]:
    ds = []
    for u in list(R[:sample]):
        p = g.kcp([int(u)], S, t)
        if len(p) == t:
            ds.append(int(p.d[-1]))
    return int(np.median(ds)), ds


def main(parts: list[str] | None = None) -> None:
    """Recompute the stored workload parameters: every part (a few minutes), or only the
    parts named (grid, road264k, road1070k, batch, serve)."""
    o = O.default()
    out = {}
    t0 = time.time()
    want = (lambda name: not parts or name in parts)
    if want("grid"):
        _grid(o, out)
    if want("road264k"):
        _road264k(o, out, t0)
    if want("road1070k"):
        _road1070k(o, out, t0)
    if want("batch"):
        _batch(o, out, t0)
    if want("serve"):
        _serve(o, out, t0)
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    old = json.load(open(OUT)) if os.path.exists(OUT) else {}
    old.update(out)
    with open(OUT, "w") as f:
        json.dump(old, f, indent=1, sort_keys=True)
        f.write("\n")


def _grid(o, out) -> None:
    w = I.c1_grid_join()
    g = o.graph(w.graph.n, w.graph.src, w.graph.dst, w.graph.w)
    full = g.join(w.R, w.S, w.theta)
    out["grid4096_theta1500"] = {"theta": 1500, "pairs": len(full), "alg_arcs": full.arcs,
                                 "graph": graph_digest(w.graph)}


def _road264k(o, out, t0) -> None:
    w = I.c2_road_join(None)
    g = o.graph(w.graph.n, w.graph.src, w.graph.dst, w.graph.w)
    th, _ = theta_for_matches(g, w.R, w.S, 50, 256)
    full = g.join(w.R, w.S, th)
    # alg_arcs: the arcs the plain per-source searches of the oracle look at (the sum
    # over sources of the out-degrees of the nodes within theta), the GTEPS numerator
    out["road264k_join"] = {"theta": th, "matches_per_u": 50, "sample": 256,
                            "pairs": len(full), "alg_arcs": full.arcs,
                            "graph": graph_digest(w.graph)}
    print("road264k_join theta", th, f"{time.time() - t0:.1f}s", flush=True)


def _road1070k(o, out, t0) -> None:
    w = I.c3_road_clustered()
    g = o.graph(w.graph.n, w.graph.src, w.graph.dst, w.graph.w)
    th, _ = theta_for_matches(g, w.R, w.S, 50, 256)
    full = g.join_mt(w.R, w.S, th, O.host_cores())
    out["road1070k_clustered"] = {"theta_join": th, "matches_per_u": 50, "sample": 256,
                                  "pairs": len(full), "alg_arcs": full.arcs,
                                  "k": [100, 10_000, 1_000_000], "graph": graph_digest(w.graph)}
    print("road1070k_clustered theta", th, f"{time.time() - t0:.1f}s", flush=True)


def _batch(o, out, t0) -> None:
    # the batch: theta per instance for its target matches per R node (32 sampled R);
    # an instance whose sampled sources reach fewer S nodes than the target gets the
    # largest distance its samples reached
    thetas, digests = [], []
    for sp in I.c4_batch_specs():
        e, R, S = I.c4_instance(sp)
        g = o.graph(e.n, e.src, e.dst, e.w)
        t = max(1, int(round(sp.matches)))
        ds, far = [], 0
        for u in list(R[:32]):
            p = g.kcp([int(u)], S, t)
            if len(p):
                far = max(far, int(p.d[-1]))
            if len(p) == t:
                ds.append(int(p.d[-1]))
        thetas.append(int(np.median(ds)) if ds else far)
        digests.append(graph_digest(e)["wsum"])
    # the batch's algorithmic arcs (GTEPS numerator): every instance's join at its theta
    alg_arcs, pairs = 0, 0
    for sp, th in zip(I.c4_batch_specs(), thetas):
        e, R, S = I.c4_instance(sp)
        p = o.graph(e.n, e.src, e.dst, e.w).join_mt(R, S, th, O.host_cores())
        alg_arcs += p.arcs
        pairs += len(p)
    out["batch512"] = {"theta": thetas, "sample": 32, "graph_wsum": digests, "alg_arcs": alg_arcs,
                       "pairs": pairs}
    print("batch512", len(thetas), f"{time.time() - t0:.1f}s", flush=True)


def _serve(o, out, t0) -> None:
    # serving: ball growth of the 6M-node graph, nodes within theta ~ c * theta^2, from
    # the oracle's distances of 32 sampled sources at radii holding 1k..50k nodes
    e = I.c5_serve_graph()
    g = o.graph(e.n, e.src, e.dst, e.w)
    rng = np.random.default_rng(I.BASE_SEED + 6)
    ratios = []
    for u in rng.choice(e.n, size=32, replace=False):
        dist, _ = g.sssp(int(u), 3_000_000)
        d = np.sort(dist[dist <= 3_000_000].astype(np.float64))
        for b in (1_000, 2_000, 4_000, 8_000, 16_000, 32_000, 50_000):
            if len(d) > b and d[b - 1] > 0:
                ratios.append(b / d[b - 1] ** 2)
    out["serve6m"] = {"ball_coeff": float(np.median(ratios)), "samples": len(ratios),
                      "graph": graph_digest(e)}
    print("serve6m ball_coeff", out["serve6m"]["ball_coeff"], f"{time.time() - t0:.1f}s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
