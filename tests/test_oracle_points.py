"""Pins of the oracle's queries over points on edges (objects on an edge, searched from
the two ends of their edge: Section 1).

The independent formulation: subdivide every edge that carries points at the points'
positions (a chain of shorter edges through new nodes; a point at an end is that end
node), then the distance between two points is the distance between their nodes in the
subdivided graph, taken from the node search, which is pinned on its own (Floyd-Warshall,
closed forms).  Also closed forms on a path, the transpose symmetry, and the input rules.
"""
import numpy as np
import pytest

from paper_1607_07696_gb300 import inputs as I

from pins import least_weights, points_by_subdivision, random_points  # noqa: E402


@pytest.mark.parametrize("seed", range(12))
def test_join_points_equals_subdivided_graph(oracle, seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(30, 400))
    e = I.road_graph(n, int(2.77 * n), 950 + seed)
    best = least_weights(e)
    pts = random_points(rng, best, int(rng.integers(2, 40)))
    # coincident points and several points on one edge
    pts += [pts[0], pts[1]]
    k = list(best)[0]
    pts += [(k[0], k[1], t) for t in (0, 1, best[k] // 2, best[k])]
    R, S = pts[: len(pts) // 2], pts[len(pts) // 2:]
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    for theta in (0, int(np.median(e.w)) * 3, 1 << 31):
        got = og.join_points(R, S, theta)
        ref = points_by_subdivision(oracle, e, R, S, theta)
        assert [(int(a), int(b), int(c)) for a, b, c in zip(got.u, got.v, got.d)] == ref, f"theta {theta}"
        # k closest pairs: the subdivision pairs ordered by (d, i, j), cut to k
        refk = sorted(ref, key=lambda r: (r[2], r[0], r[1]))
        for kk in (1, 5, len(ref) + 3):
            gk = og.kcp_points(R, S, kk, theta)
            assert [(int(a), int(b), int(c)) for a, b, c in zip(gk.u, gk.v, gk.d)] == refk[:kk]


def test_points_on_a_path(oracle):
    # path 0-1-2-3-4 with weights 2, 3, 5, 7: a point's position on the line is its
    # offset from 0; the distance between two points is the gap between positions
    w = [2, 3, 5, 7]
    e = I.path_graph(w)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    start = np.concatenate([[0], np.cumsum(w)])
    pts, pos = [], []
    for i, wi in enumerate(w):
        for t in range(0, wi + 1):
            pts.append((i, i + 1, t) if t % 2 else (i + 1, i, wi - t))
            pos.append(int(start[i]) + t)
    got = og.join_points(pts, pts, 1 << 31)
    assert len(got) == len(pts) ** 2
    for i, j, d in zip(got.u, got.v, got.d):
        assert int(d) == abs(pos[i] - pos[j])


def test_transpose_symmetry(oracle):
    rng = np.random.default_rng(3)
    e = I.road_graph(300, 831, 4)
    best = least_weights(e)
    R, S = random_points(rng, best, 25), random_points(rng, best, 30)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    a = og.join_points(R, S, 60_000)
    b = og.join_points(S, R, 60_000)
    fwd = sorted(zip(a.u.tolist(), a.v.tolist(), a.d.tolist()))
    bwd = sorted(zip(b.v.tolist(), b.u.tolist(), b.d.tolist()))
    assert fwd == bwd


def test_point_at_a_node_is_that_node(oracle):
    e = I.road_graph(500, 1385, 8)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    best = least_weights(e)
    R, S = I.disjoint_sets(e.n, 20, 30, 9)
    incident = {}
    for (p, q), ww in best.items():
        incident.setdefault(p, (p, q, 0))
        incident.setdefault(q, (q, p, 0))
    keep_R = [x for x in R.tolist() if x in incident]
    keep_S = [x for x in S.tolist() if x in incident]
    got = og.join_points([incident[x] for x in keep_R], [incident[x] for x in keep_S], 50_000)
    ref = og.join(keep_R, keep_S, 50_000)
    idx_R = {x: i for i, x in enumerate(keep_R)}
    idx_S = {x: i for i, x in enumerate(keep_S)}
    assert sorted((idx_R[int(u)], idx_S[int(v)], int(d)) for u, v, d in zip(ref.u, ref.v, ref.d)) == \
        [(int(a), int(b), int(c)) for a, b, c in zip(got.u, got.v, got.d)]


def test_bad_points_rejected(oracle):
    from oracle.oracle import OracleError

    e = I.path_graph([4, 6])
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    for bad in ([(0, 2, 1)], [(0, 1, 5)], [(1, 1, 0)], [(0, 9, 0)]):
        with pytest.raises(OracleError):
            og.join_points(bad, [(0, 1, 0)], 100)
    with pytest.raises(OracleError):
        og.kcp_points([(0, 1, 0)], [(1, 2, 3)], 0)
