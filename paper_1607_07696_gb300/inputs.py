"""Seeded synthetic inputs: road-like graphs and the R / S node sets joined over them.

This module holds no shortest-path arithmetic at all; it only draws graphs and sets.
Both the CUDA engine's tests and the CPU oracle are fed from here, and nothing else is
shared between them.  The real road networks of the paper's experiments (North
America, 175,813 nodes / 179,179 edges and San Francisco, 174,956 nodes / 223,001
edges, Section 5) are not available, so these generators stand in for them:

* ``grid_graph``     a 64 x 64 jittered lattice with ~10% of its edges removed and
                     diagonals in ~3% of its cells, weights round(100 * length) clamped
                     to [50, 150];
* ``road_graph``     uniform random points in the unit square joined by a symmetrised
                     k-nearest-neighbour graph (k = 4), thinned by dropping the longest
                     edges to a target edge count (average degree ~2.8, close to the
                     planar sparsity of road maps), weights = scaled Euclidean length in
                     [1, 10^4];
* ``disjoint_sets``  R and S drawn uniformly without overlap;
* ``clustered_sets`` R and S drawn from 20 Gaussian clusters, each draw snapped to the
                     nearest node not yet used.

Every generator is a pure function of its arguments and seed; numpy's PCG64 stream
is the same on every platform.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 0x16070769


@dataclass
class EdgeList:
    """An undirected weighted graph as an edge list (ids 0..n-1), with coordinates."""

    n: int
    src: np.ndarray  # uint32[m]
    dst: np.ndarray  # uint32[m]
    w: np.ndarray  # uint32[m]
    xy: np.ndarray | None = None  # float64[n, 2]
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(len(self.src))


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


# ---------------------------------------------------------------------- graphs ----

def grid_graph(seed: int = BASE_SEED + 0, side: int = 64, drop: float = 0.10,
               diag: float = 0.03, jitter: float = 0.2) -> EdgeList:
    """Jittered side x side lattice: node (i, j) has id i * side + j and sits at
    (i + U[-j, j], j + U[-j, j]); each 4-neighbour edge is removed with probability
    ``drop``; a random one of the two diagonals is added in a fraction ``diag`` of the
    cells; weight = clamp(round(100 * Euclidean length), 50, 150)."""
    rng = np.random.default_rng(seed)
    n = side * side
    ii, jj = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    xy = np.stack([ii.ravel(), jj.ravel()], axis=1).astype(np.float64)
    xy += rng.uniform(-jitter, jitter, size=(n, 2))
    ids = (ii * side + jj)
    horiz = np.stack([ids[:, :-1].ravel(), ids[:, 1:].ravel()], axis=1)
    vert = np.stack([ids[:-1, :].ravel(), ids[1:, :].ravel()], axis=1)
    lat = np.concatenate([horiz, vert])
    lat = lat[rng.random(len(lat)) >= drop]
    cells = (side - 1) * (side - 1)
    pick = np.nonzero(rng.random(cells) < diag)[0]
    ci, cj = pick // (side - 1), pick % (side - 1)
    which = rng.integers(0, 2, size=len(pick))
    a = np.where(which == 0, ci * side + cj, ci * side + cj + 1)
    b = np.where(which == 0, (ci + 1) * side + cj + 1, (ci + 1) * side + cj)
    e = np.concatenate([lat, np.stack([a, b], axis=1)])
    d = xy[e[:, 0]] - xy[e[:, 1]]
    length = np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1])
    w = np.clip(np.rint(100.0 * length), 50, 150)
    return EdgeList(n, _u32(e[:, 0]), _u32(e[:, 1]), _u32(w), xy,
                    {"kind": "grid", "side": side, "seed": seed})


def _knn_table(xy: np.ndarray, k: int) -> np.ndarray:
    """Indices of the k nearest other points of every point (column 0 = nearest)."""
    from scipy.spatial import cKDTree

    n = len(xy)
    _, idx = cKDTree(xy).query(xy, k=min(k + 1, n), workers=-1)  # per-point results: thread-count independent
    return np.asarray(idx).reshape(n, -1)[:, 1:]


def _knn_edges(idx: np.ndarray, k: int) -> np.ndarray:
    """Undirected edge set {a, b} (a < b) of the symmetrised k-NN relation."""
    n = len(idx)
    src = np.repeat(np.arange(n, dtype=np.int64), k)
    dst = idx[:, :k].ravel().astype(np.int64)
    keep = src != dst
    a = np.minimum(src[keep], dst[keep])
    b = np.maximum(src[keep], dst[keep])
    key = a * n + b
    key.sort()
    key = key[np.concatenate(([True], key[1:] != key[:-1]))] if len(key) else key
    return np.stack([key // n, key % n], axis=1)


def road_graph(n: int, m: int, seed: int, wmax: int = 10_000) -> EdgeList:
    """Road-like graph: n uniform points in the unit square, symmetrised 4-NN edges
    (5-NN, then 6-NN, when 4-NN gives fewer than m), then the longest edges dropped
    (ties: the larger (a, b) first) until exactly m remain.  Weight =
    clamp(round(wmax * length / longest kept length), 1, wmax)."""
    rng = np.random.default_rng(seed)
    xy = rng.random((n, 2))
    idx = _knn_table(xy, 8)
    e = None
    for k in (4, 5, 6, 8):
        e = _knn_edges(idx, min(k, idx.shape[1]))
        if len(e) >= m:
            break
    d = xy[e[:, 0]] - xy[e[:, 1]]
    length = np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1])
    if len(e) > m:
        # the m first edges in (length, a, b) order: every edge shorter than the m-th
        # length, then the ties at that length by (a, b)
        cut = np.partition(length, m - 1)[m - 1]
        short = np.nonzero(length < cut)[0]
        tie = np.nonzero(length == cut)[0]
        tie = tie[np.lexsort((e[tie, 1], e[tie, 0]))][:m - len(short)]
        sel = np.sort(np.concatenate([short, tie]))
        e, length = e[sel], length[sel]
    lmax = float(length.max()) if len(length) else 1.0
    w = np.clip(np.rint(wmax * length / lmax), 1, wmax)
    return EdgeList(n, _u32(e[:, 0]), _u32(e[:, 1]), _u32(w), xy,
                    {"kind": "road", "n": n, "m_target": m, "seed": seed})


def random_graph(n: int, m: int, seed: int, wlo: int = 1, whi: int = 100,
                 loops: bool = True, multi: bool = True) -> EdgeList:
    """Uniform random multigraph for small brute-force tests: m edges with uniform
    endpoints (self-loops and parallel edges allowed unless switched off), weights
    uniform in [wlo, whi]."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, size=m)
    dst = rng.integers(0, n, size=m)
    if not loops:
        bad = src == dst
        dst[bad] = (dst[bad] + 1) % max(n, 1)
    if not multi:
        a, b = np.minimum(src, dst), np.maximum(src, dst)
        _, first = np.unique(a * n + b, return_index=True)
        first = np.sort(first)
        src, dst = src[first], dst[first]
    w = rng.integers(wlo, whi + 1, size=len(src))
    return EdgeList(n, _u32(src), _u32(dst), _u32(w), None,
                    {"kind": "random", "seed": seed})


def full_grid(wd: int, ht: int, c: int) -> EdgeList:
    """Complete wd x ht lattice, every edge of weight c; node (x, y) has id y * wd + x."""
    ids = np.arange(wd * ht).reshape(ht, wd)
    h = np.stack([ids[:, :-1].ravel(), ids[:, 1:].ravel()], axis=1)
    v = np.stack([ids[:-1, :].ravel(), ids[1:, :].ravel()], axis=1)
    e = np.concatenate([h, v])
    return EdgeList(wd * ht, _u32(e[:, 0]), _u32(e[:, 1]), _u32(np.full(len(e), c)), None,
                    {"kind": "full_grid", "wd": wd, "ht": ht, "c": c})


def path_graph(weights) -> EdgeList:
    """Path 0 - 1 - ... - len(weights), edge i of weight weights[i]."""
    w = _u32(weights)
    n = len(w) + 1
    return EdgeList(n, _u32(np.arange(n - 1)), _u32(np.arange(1, n)), w, None, {"kind": "path"})


def star_graph(weights) -> EdgeList:
    """Star with centre 0 and leaves 1..len(weights), leaf i joined by weights[i-1]."""
    w = _u32(weights)
    n = len(w) + 1
    return EdgeList(n, _u32(np.zeros(n - 1)), _u32(np.arange(1, n)), w, None, {"kind": "star"})


# ------------------------------------------------------------------------ sets ----

def disjoint_sets(n: int, nR: int, nS: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """R and S: nR + nS distinct nodes drawn uniformly, the first nR form R."""
    rng = np.random.default_rng(seed)
    pick = rng.choice(n, size=nR + nS, replace=False)
    return _u32(pick[:nR]), _u32(pick[nR:])


def clustered_sets(xy: np.ndarray, nR: int, nS: int, seed: int, clusters: int = 20,
                   sigma: float = 0.05) -> tuple[np.ndarray, np.ndarray]:
    """R and S from Gaussian clusters (centres U[.1, .9]^2, standard deviation sigma).
    Cluster c receives an equal share of each set; within a cluster the draws alternate
    R, S, R, S, ...; every draw is snapped to the nearest node not used yet."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    n = len(xy)
    if nR + nS > n:
        raise ValueError("R and S do not fit in the graph")
    centres = rng.uniform(0.1, 0.9, size=(clusters, 2))
    quota_r = [nR // clusters + (1 if c < nR % clusters else 0) for c in range(clusters)]
    quota_s = [nS // clusters + (1 if c < nS % clusters else 0) for c in range(clusters)]
    order = []  # (cluster, side) in draw order
    for c in range(clusters):
        qr, qs = quota_r[c], quota_s[c]
        for i in range(max(qr, qs)):
            if i < qr:
                order.append((c, 0))
            if i < qs:
                order.append((c, 1))
    pts = np.array([centres[c] for c, _ in order]) + rng.normal(0.0, sigma, size=(len(order), 2))
    tree = cKDTree(xy)
    kq = min(64, n)
    _, cand = tree.query(pts, k=kq)
    cand = np.asarray(cand).reshape(len(order), kq)
    used = np.zeros(n, dtype=bool)
    R, S = [], []
    for i, (c, side) in enumerate(order):
        pick = -1
        for x in cand[i]:
            if not used[x]:
                pick = int(x)
                break
        kk = kq
        while pick < 0:
            kk = min(kk * 4, n)
            _, more = tree.query(pts[i], k=kk)
            for x in np.atleast_1d(more):
                if not used[x]:
                    pick = int(x)
                    break
        used[pick] = True
        (R if side == 0 else S).append(pick)
    return _u32(R), _u32(S)


# ----------------------------------------------------------------- workloads ----

@dataclass
class Workload:
    """A join or kCP instance: a graph, R, S and its parameters."""

    name: str
    graph: EdgeList
    R: np.ndarray
    S: np.ndarray
    theta: int | None = None
    k: int | None = None
    meta: dict = field(default_factory=dict)


def c1_grid_join(seed: int = BASE_SEED + 0) -> Workload:
    """64x64 perturbed grid, |R| = |S| = 256 disjoint uniform nodes, theta = 1,500."""
    g = grid_graph(seed)
    R, S = disjoint_sets(g.n, 256, 256, seed + 1000)
    return Workload("grid4096_theta1500", g, R, S, theta=1500)


def c2_road_join(theta: int | None, seed: int = BASE_SEED + 1) -> Workload:
    """264k-node road-like graph, ~730k edges, |R| = |S| = 10,000 disjoint uniform
    nodes; theta calibrated so the median R node has ~50 S nodes within it."""
    g = road_graph(264_000, 730_000, seed)
    R, S = disjoint_sets(g.n, 10_000, 10_000, seed + 1000)
    return Workload("road264k_join", g, R, S, theta=theta)


def c3_road_clustered(theta: int | None = None, k: int | None = None,
                      seed: int = BASE_SEED + 2) -> Workload:
    """1.07M-node road-like graph, ~2.7M edges, |R| = |S| = 50,000 nodes in 20
    Gaussian clusters."""
    g = road_graph(1_070_000, 2_700_000, seed)
    R, S = clustered_sets(g.xy, 50_000, 50_000, seed + 1000)
    return Workload("road1070k_clustered", g, R, S, theta=theta, k=k)


def log_uniform(rng: np.random.Generator, lo: float, hi: float, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))


@dataclass
class BatchSpec:
    """One instance of the batched workload, before its graph is generated."""

    n: int
    m: int
    graph_seed: int
    nR: int
    nS: int
    set_seed: int
    matches: float  # target S-matches per R node (theta is calibrated for it)


def c4_batch_specs(count: int = 512, seed: int = BASE_SEED + 3) -> list[BatchSpec]:
    """512 joins of uneven size: n log-uniform in [1k, 50k] nodes, m = 2.77 n edges (the
    road-like generator), |R| and |S| log-uniform in [64, 4096] independently, each capped
    at n / 3, and a target of 5 to 200 S-matches per R node, log-uniform."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        n = int(round(log_uniform(rng, 1_000, 50_000)))
        nR = int(min(round(log_uniform(rng, 64, 4096)), n // 3))
        nS = int(min(round(log_uniform(rng, 64, 4096)), n // 3))
        matches = float(log_uniform(rng, 5, 200))
        specs.append(BatchSpec(n, int(round(2.77 * n)), seed + 1 + i, nR, nS, seed + 100_000 + i, matches))
    return specs


def c4_instance(spec: BatchSpec) -> tuple[EdgeList, np.ndarray, np.ndarray]:
    g = road_graph(spec.n, spec.m, spec.graph_seed)
    R, S = disjoint_sets(g.n, spec.nR, spec.nS, spec.set_seed)
    return g, R, S


# ---------------------------------------------------------------- serving ----

C5_N, C5_M = 6_000_000, 14_000_000
C5_BALL_CAP = 4_096  # largest expected ball (nodes per source) a request is sized for


def c5_serve_graph(seed: int = BASE_SEED + 4) -> EdgeList:
    """The resident graph of the serving workload: the road-like generator at 6M nodes,
    14M edges."""
    return road_graph(C5_N, C5_M, seed)


@dataclass
class ServeRequest:
    """One request of the serving stream: a theta-join (k = 0) or k closest pairs."""

    R: np.ndarray
    S: np.ndarray
    theta: int
    k: int
    matches: float  # target S-matches per R node of a join (0 for k closest pairs)


def c5_requests(n: int, count: int, ball_coeff: float, seed: int = BASE_SEED + 5,
                join_frac: float = 0.7) -> list[ServeRequest]:
    """The mixed request stream: 70% theta-joins, 30% k closest pairs; |R| and |S|
    log-uniform in [100, 20000] (disjoint uniform nodes), k log-uniform in [10, 1e5].  A
    join's theta targets log-uniform [5, 200] S-matches per R node: the expected ball
    holding that many S nodes is matches * n / |S| nodes, and a ball of b nodes has
    radius sqrt(b / ball_coeff) (the graph's measured ball growth, about
    ball_coeff * theta^2 nodes within theta).  k closest pairs run unbounded.  Either
    kind is sized so the expected ball of one source stays within C5_BALL_CAP nodes: a
    join's target lowered to what such a ball holds (theta at the cap's radius), k to
    at most |R| * |S| * C5_BALL_CAP / n (without the cap, small sets with a large
    target make single requests search the whole graph from every source)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nR = int(round(log_uniform(rng, 100, 20_000)))
        nS = int(round(log_uniform(rng, 100, 20_000)))
        R, S = disjoint_sets(n, nR, nS, seed + 1 + i)
        if rng.random() < join_frac:
            matches = float(log_uniform(rng, 5, 200))
            ball = min(matches * n / nS, C5_BALL_CAP)
            theta = int(round(np.sqrt(ball / ball_coeff)))
            out.append(ServeRequest(R, S, theta, 0, matches))
        else:
            k = int(round(log_uniform(rng, 10, 100_000)))
            k = max(1, min(k, int(nR * nS * C5_BALL_CAP / n)))
            out.append(ServeRequest(R, S, 0xFFFFFFFF, k, 0.0))
    return out


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream of the given rate (per second)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))
