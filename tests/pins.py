"""Pins for the CPU oracle: checks against things other than the oracle itself.

Each pin is a plain function of an ``Oracle`` handle that raises ``AssertionError`` on a
mismatch, so the same suite runs on the real oracle (test_oracle_pins.py) and on
planted mutants of it (test_oracle_mutants.py), which must each fail at least one.

What pins what:
* Floyd-Warshall brute force on tiny random (multi)graphs, directed and undirected:
  pins the bounded Dijkstra, the inclusive theta cut (Abstract: dist <= theta;
  Algorithm 4: stop only when the cost is greater than theta), the join's (u, v)
  order and kCP's (d, u, v) order at every k.
* Closed forms: a uniform c-weighted wd x ht lattice has dist = c (|dx| + |dy|); a path
  has prefix-sum distances; a star has dist(leaf i, leaf j) = w_i + w_j.
* Invariants on a road-like graph: the join is its own transpose on an undirected
  graph, it grows monotonically with theta, kCP at k is a prefix of kCP at k + 1 and
  equals the first k of the full join sorted by (d, u, v).
* Input rules: ids out of range, repeated ids, R and S overlapping, bad weights.
* Edge-list cleaning: self-loops dropped and parallel edges reduced to their least
  weight (checked against a numpy reduction of the same edge list).
* Points on edges (Section 1: objects moving on edges): the join and kCP of points equal
  the node search on the graph subdivided at the points (an independent formulation:
  new nodes on chains of shorter edges, the node search itself pinned above); points on
  a path are at the gap between their positions; a point at a node is that node.
"""
from __future__ import annotations

import numpy as np

from paper_1607_07696_gb300 import inputs as I

INF64 = np.uint64((1 << 64) - 1)
THETA_MAX = 1 << 31


def _fw_pairs(D: np.ndarray, R, S, theta: int):
    out = []
    for u in R:
        for v in S:
            d = D[u, v]
            if d != INF64 and int(d) <= theta:
                out.append((int(u), int(v), int(d)))
    return out


def pin_fw_random(o, seeds=range(60)):
    """Oracle join / kCP / sssp equal Floyd-Warshall brute force on tiny graphs."""
    for seed in seeds:
        rng = np.random.default_rng(1000 + seed)
        n = int(rng.integers(2, 34))
        m = int(rng.integers(0, 3 * n))
        undirected = bool(seed % 3 != 0)
        wlo, whi = (1, 9) if seed % 2 else (1, 1000)
        e = I.random_graph(n, m, seed, wlo, whi)
        g = o.graph(n, e.src, e.dst, e.w, undirected)
        D = g.floyd_warshall()
        # sssp rows, unbounded and bounded
        for s in range(min(n, 6)):
            dist, _ = g.sssp(s)
            assert np.array_equal(dist, D[s]), f"seed {seed}: sssp row {s} != Floyd-Warshall"
        perm = rng.permutation(n)
        nR = int(rng.integers(1, n)) if n > 1 else 1
        nS = int(rng.integers(0, n - nR + 1))
        R, S = perm[:nR], perm[nR:nR + nS]
        finite = D[D != INF64]
        choices = [0, 1, THETA_MAX, int(rng.integers(0, 3 * whi + 1))]
        if finite.size:
            choices += [int(np.median(finite)), int(finite.max())]
        for theta in choices:
            want = sorted(_fw_pairs(D, R, S, theta))
            got = g.join(R, S, theta).triples()
            assert got == want, f"seed {seed} theta {theta}: join != brute force"
            got = g.join_mt(R, S, theta, threads=1 + seed % 4).triples()
            assert got == want, f"seed {seed} theta {theta}: threaded join != brute force"
            byd = sorted(want, key=lambda t: (t[2], t[0], t[1]))
            for k in sorted({1, 2, 3, max(1, len(byd)), len(byd) + 1, max(1, len(byd) // 2)}):
                kc = g.kcp(R, S, k, theta).triples()
                assert kc == byd[:k], f"seed {seed} theta {theta} k {k}: kcp != brute force"
                kc = g.kcp_mt(R, S, k, theta, threads=1 + seed % 4).triples()
                assert kc == byd[:k], f"seed {seed} theta {theta} k {k}: threaded kcp != brute force"


def pin_closed_forms(o):
    """Distances that have a closed form."""
    wd, ht, c = 9, 7, 13
    e = I.full_grid(wd, ht, c)
    g = o.graph(e.n, e.src, e.dst, e.w)
    for s in (0, 5, wd * ht - 1, 3 * wd + 4):
        dist, arcs = g.sssp(s)
        sx, sy = s % wd, s // wd
        for x in range(e.n):
            assert int(dist[x]) == c * (abs(x % wd - sx) + abs(x // wd - sy)), "grid distance"
        # unbounded search settles every node: the arcs looked at are all 2m arcs
        assert arcs == 2 * e.m, "grid arc count"
    # bounded: exactly the nodes within Manhattan radius theta / c
    theta = 3 * c
    dist, _ = g.sssp(0, theta)
    reached = {x for x in range(e.n) if dist[x] != INF64}
    want = {x for x in range(e.n) if c * (x % wd + x // wd) <= theta}
    assert reached == want, "grid theta ball"
    # path: prefix sums
    w = np.array([5, 1, 7, 2, 9, 3], np.uint32)
    p = I.path_graph(w)
    g = o.graph(p.n, p.src, p.dst, p.w)
    pre = np.concatenate([[0], np.cumsum(w.astype(np.int64))])
    for s in range(p.n):
        dist, _ = g.sssp(s)
        for x in range(p.n):
            assert int(dist[x]) == abs(int(pre[x]) - int(pre[s])), "path distance"
    R, S = [0, 2], [1, 3, 6]
    want = sorted((u, v, abs(int(pre[v]) - int(pre[u]))) for u in R for v in S
                  if abs(int(pre[v]) - int(pre[u])) <= 14)
    assert g.join(R, S, 14).triples() == want, "path join"
    # star: leaf-to-leaf distance is the sum of the two spokes
    sw = np.array([4, 9, 1, 6, 6], np.uint32)
    st = I.star_graph(sw)
    g = o.graph(st.n, st.src, st.dst, st.w)
    R, S = [1, 2], [3, 4, 5]
    pairs = sorted((u, v, int(sw[u - 1]) + int(sw[v - 1])) for u in R for v in S)
    assert g.join(R, S, THETA_MAX).triples() == pairs, "star join"
    byd = sorted(pairs, key=lambda t: (t[2], t[0], t[1]))
    assert g.kcp(R, S, 3).triples() == byd[:3], "star kcp tie-break"
    # directed path: no way back
    g = o.graph(3, [0, 1], [1, 2], [2, 3], undirected=False)
    assert g.join([2], [0], THETA_MAX).triples() == [], "directed path reversed"
    assert g.join([0], [2], THETA_MAX).triples() == [(0, 2, 5)], "directed path"


def pin_invariants(o, n=3000, seed=7):
    """Transpose symmetry, monotonicity in theta and k, kCP = sorted join prefix."""
    e = I.road_graph(n, int(2.77 * n), seed)
    g = o.graph(e.n, e.src, e.dst, e.w)
    R, S = I.disjoint_sets(e.n, 120, 150, seed + 1)
    thetas = [0, 2000, 9000, 20000, 45000]
    prev = set()
    for theta in thetas:
        j = g.join(R, S, theta).triples()
        assert j == sorted(j), "join not sorted by (u, v)"
        js = set(j)
        assert prev <= js, "join not monotone in theta"
        prev = js
        t = g.join(S, R, theta).triples()
        assert sorted((v, u, d) for (u, v, d) in t) == j, "join not its own transpose"
        assert all(d <= theta for (_, _, d) in j), "pair beyond theta"
        assert g.join_mt(R, S, theta, threads=5).triples() == j, "threaded join differs"
    full = sorted(g.join(R, S, THETA_MAX).triples(), key=lambda t: (t[2], t[0], t[1]))
    last = []
    for k in (1, 2, 5, 50, 51, 400, len(full), len(full) + 7):
        kc = g.kcp(R, S, k).triples()
        assert kc == full[:k], f"kcp k={k} != first k of the sorted join"
        assert kc[: len(last)] == last, "kcp not a prefix in k"
        assert g.kcp_mt(R, S, k, threads=3).triples() == kc, f"threaded kcp k={k} differs"
        last = kc
    kb = g.kcp_bruteforce(R, S, 77, 9000).triples()
    assert g.kcp(R, S, 77, 9000).triples() == kb, "kcp with theta != brute force"
    # kCP through a join at a doubled probe bound: the first k of the sorted join
    for k, probe in ((1, 1), (50, 300), (400, 2000), (len(full) + 7, 5)):
        got = g.kcp_by_join(R, S, k, probe=probe, threads=2).triples()
        assert got == full[:k], f"kcp by join k={k} probe {probe}"
    assert g.kcp_by_join(R, S, 77, 9000, probe=100).triples() == kb, "kcp by join with theta"


def pin_triangle(o, seeds=range(8)):
    """Triangle inequality over FW matrices and over joined pairs."""
    for seed in seeds:
        e = I.random_graph(24, 60, 50 + seed, 1, 50)
        g = o.graph(e.n, e.src, e.dst, e.w)
        D = g.floyd_warshall().astype(object)
        R, S = list(range(0, 12)), list(range(12, 24))
        jd = {(u, v): d for (u, v, d) in g.join(R, S, THETA_MAX).triples()}
        for (u, v), d in jd.items():
            for x in range(e.n):
                if D[u, x] != int(INF64) and D[x, v] != int(INF64):
                    assert d <= D[u, x] + D[x, v], "triangle inequality"


def pin_validation(o):
    """Inputs the problem statement rules out are rejected."""
    from oracle.oracle import OracleError

    e = I.path_graph([1, 2, 3, 4])
    g = o.graph(e.n, e.src, e.dst, e.w)
    bad = [
        ([0, 9], [2]),  # id >= n
        ([0, 0], [2]),  # repeated in R
        ([0], [2, 2]),  # repeated in S
        ([0, 2], [2, 3]),  # R and S overlap
    ]
    for R, S in bad:
        for call in (lambda: g.join(R, S, 10), lambda: g.kcp(R, S, 1, 10)):
            try:
                call()
            except OracleError:
                continue
            raise AssertionError(f"accepted R={R} S={S}")
    for call in (lambda: g.join([0], [1], THETA_MAX + 1), lambda: g.kcp([0], [1], 0)):
        try:
            call()
        except OracleError:
            continue
        raise AssertionError("accepted theta > 2^31 or k = 0")
    for w in (0, 1 << 24):
        try:
            o.graph(2, [0], [1], [w])
        except OracleError:
            continue
        raise AssertionError(f"accepted weight {w}")
    # empty sets are fine and give nothing
    assert g.join([], [1], 10).triples() == [] and g.join([0], [], 10).triples() == []


def pin_cleaning(o, seeds=range(10)):
    """Self-loops and parallel edges: the result equals that of the cleaned edge list."""
    for seed in seeds:
        e = I.random_graph(20, 70, 300 + seed, 1, 30)
        a = np.minimum(e.src, e.dst).astype(np.int64)
        b = np.maximum(e.src, e.dst).astype(np.int64)
        keep = a != b
        key = a[keep] * 20 + b[keep]
        w = e.w[keep].astype(np.int64)
        order = np.lexsort((w, key))
        key, w = key[order], w[order]
        first = np.concatenate([[True], key[1:] != key[:-1]]) if len(key) else np.zeros(0, bool)
        ca, cb, cw = key[first] // 20, key[first] % 20, w[first]
        g1 = o.graph(20, e.src, e.dst, e.w)
        g2 = o.graph(20, ca, cb, cw)
        assert g1.num_arcs == 2 * len(ca), "cleaned arc count"
        R, S = list(range(10)), list(range(10, 20))
        assert g1.join(R, S, THETA_MAX).triples() == g2.join(R, S, THETA_MAX).triples(), \
            "multigraph join != cleaned graph join"


def least_weights(e):
    """The least weight of every undirected edge {p < q} of an edge list."""
    best = {}
    for a, b, w in zip(e.src.tolist(), e.dst.tolist(), e.w.tolist()):
        if a != b:
            k = (min(a, b), max(a, b))
            best[k] = min(best.get(k, 1 << 40), w)
    return best


def subdivide(n, best, points):
    """The graph subdivided at the points: every edge carrying points becomes a chain
    through one new node per distinct inner position (a point at an end is that end).
    Returns (node count, src, dst, w, node of every point)."""
    on = {}
    for i, (a, b, t) in enumerate(points):
        k = (min(a, b), max(a, b))
        on.setdefault(k, []).append((t if a == k[0] else best[k] - t, i))
    src, dst, w = [], [], []
    for (p, q), ww in best.items():
        if (p, q) not in on:
            src.append(p), dst.append(q), w.append(ww)
    node = [0] * len(points)
    nxt = n
    for (p, q), lst in on.items():
        W = best[(p, q)]
        at = {0: p, W: q}
        for pos in sorted({pos for pos, _ in lst}):
            if pos not in at:
                at[pos] = nxt
                nxt += 1
        chain = sorted(at.items())
        for (p0, n0), (p1, n1) in zip(chain, chain[1:]):
            src.append(n0), dst.append(n1), w.append(p1 - p0)
        for pos, i in lst:
            node[i] = at[pos]
    return nxt, np.array(src, np.uint32), np.array(dst, np.uint32), np.array(w, np.uint32), node


def random_points(rng, best, count):
    """Points on random edges: at either end, or anywhere, named from either end."""
    keys = list(best)
    out = []
    for _ in range(count):
        p, q = keys[rng.integers(len(keys))]
        W = best[(p, q)]
        t = int(rng.choice([0, W, rng.integers(0, W + 1), rng.integers(0, W + 1)]))
        out.append((p, q, t) if rng.random() < 0.5 else (q, p, W - t))
    return out


def points_by_subdivision(o, e, R, S, theta):
    """(i, j, d) of the points join, from node searches on the subdivided graph."""
    best = least_weights(e)
    m, src, dst, w, node = subdivide(e.n, best, list(R) + list(S))
    g = o.graph(m, src, dst, w)
    rows = []
    for i in range(len(R)):
        dist, _ = g.sssp(node[i], theta)
        for j in range(len(S)):
            d = dist[node[len(R) + j]]
            if d != INF64:
                rows.append((i, j, int(d)))
    return rows


def pin_points(o, seeds=range(6)):
    for seed in seeds:
        rng = np.random.default_rng(900 + seed)
        n = int(rng.integers(30, 300))
        e = I.road_graph(n, int(2.77 * n), 950 + seed)
        best = least_weights(e)
        pts = random_points(rng, best, int(rng.integers(2, 30)))
        k = list(best)[0]
        pts += [pts[0], pts[1]] + [(k[0], k[1], t) for t in (0, 1, best[k] // 2, best[k])]
        pts += [(k[1], k[0], best[k] // 3)]
        R, S = pts[: len(pts) // 2], pts[len(pts) // 2:]
        og = o.graph(e.n, e.src, e.dst, e.w)
        for theta in (0, int(np.median(e.w)) * 3, THETA_MAX):
            got = og.join_points(R, S, theta)
            ref = points_by_subdivision(o, e, R, S, theta)
            assert list(zip(got.u.tolist(), got.v.tolist(), got.d.tolist())) == ref, f"points seed {seed}"
            refk = sorted(ref, key=lambda r: (r[2], r[0], r[1]))
            for kk in (1, 5, len(ref) + 3):
                gk = og.kcp_points(R, S, kk, theta)
                assert list(zip(gk.u.tolist(), gk.v.tolist(), gk.d.tolist())) == refk[:kk]
    # points on a path: distance = gap between positions along the line
    w = [2, 3, 5, 7]
    e = I.path_graph(w)
    og = o.graph(e.n, e.src, e.dst, e.w)
    start = np.concatenate([[0], np.cumsum(w)])
    pts, pos = [], []
    for i, wi in enumerate(w):
        for t in range(0, wi + 1):
            pts.append((i, i + 1, t) if t % 2 else (i + 1, i, wi - t))
            pos.append(int(start[i]) + t)
    got = og.join_points(pts, pts, THETA_MAX)
    assert len(got) == len(pts) ** 2
    assert all(int(d) == abs(pos[i] - pos[j]) for i, j, d in zip(got.u, got.v, got.d))


ALL_PINS = [pin_fw_random, pin_closed_forms, pin_invariants, pin_triangle, pin_validation,
            pin_cleaning, pin_points]
