"""Queries over points on edges (objects on the road between two nodes, Section 1):
the GPU join and k closest pairs of points against the CPU oracle, bit-exact.
"""
import numpy as np
import pytest

import pins
from paper_1607_07696_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1607_07696_gb300 import build as B

    B.build()
    from paper_1607_07696_gb300 import rn as RN

    return RN


def same(got, ref):
    u, v, d = got
    return (len(u) == len(ref) and np.array_equal(u, ref.u) and np.array_equal(v, ref.v)
            and np.array_equal(d.astype(np.uint64), ref.d))


@pytest.mark.parametrize("seed", range(14))
def test_points_random(rn, oracle, seed):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(50, 4000))
    e = I.road_graph(n, int(2.77 * n), 720 + seed)
    best = pins.least_weights(e)
    pts = pins.random_points(rng, best, int(rng.integers(2, 400)))
    k0 = list(best)[int(rng.integers(len(best)))]
    pts += [pts[0], pts[-1]] + [(k0[0], k0[1], t) for t in (0, 1, best[k0] // 2, best[k0])]
    pts += [(k0[1], k0[0], best[k0] // 3)]
    order = rng.permutation(len(pts))
    cut = int(rng.integers(1, len(pts)))
    R = [pts[i] for i in order[:cut]]
    S = [pts[i] for i in order[cut:]]
    # tile widths 32, 64, 128, and the default path (0: the warp search while the balls
    # fit a warp map)
    T = [32, 64, 128, 0][seed % 4]
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n, cfg={"tile_width": T})
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    med = int(np.median(e.w))
    for theta in (0, 3 * med, 20 * med, rn.RN_INF):
        th = min(theta, rn.RN_THETA_MAX)
        assert same(rn.rn_distance_join_points(g, R, S, theta), og.join_points(R, S, th)), f"join theta {theta}"
    for k in (1, 17, 500):
        for theta in (rn.RN_INF, 10 * med):
            th = min(theta, rn.RN_THETA_MAX)
            assert same(rn.rn_kcp_points(g, R, S, k, theta), og.kcp_points(R, S, k, th)), f"kcp k {k} theta {theta}"


def test_points_larger_and_growing(rn, oracle):
    e = I.road_graph(60_000, 166_200, 77)
    best = pins.least_weights(e)
    rng = np.random.default_rng(78)
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    for count in (10, 300, 3000):  # the subdivided graph's buffers grow between queries
        R = pins.random_points(rng, best, count)
        S = pins.random_points(rng, best, count)
        assert same(rn.rn_distance_join_points(g, R, S, 30_000), og.join_points(R, S, 30_000)), count
    assert same(rn.rn_kcp_points(g, R, S, 2000), og.kcp_points(R, S, 2000))
    # node queries on the same graph are unaffected
    Rn, Sn = I.disjoint_sets(e.n, 200, 300, 79)
    ref = og.join(Rn, Sn, 30_000)
    u, v, d = rn.rn_distance_join(g, Rn, Sn, 30_000)
    assert np.array_equal(u, ref.u) and np.array_equal(v, ref.v) and np.array_equal(d.astype(np.uint64), ref.d)


def test_points_rejected(rn):
    e = I.path_graph([4, 6, 5])
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    ok = [(0, 1, 2)]
    for bad, what in (([(0, 2, 1)], "not an undirected edge"), ([(0, 1, 5)], "longer than its edge"),
                      ([(1, 1, 0)], "a == b"), ([(0, 9, 0)], ">= n")):
        with pytest.raises(rn.RNError) as ex:
            rn.rn_distance_join_points(g, bad, ok, 100)
        assert ex.value.status == rn.RN_EINVAL and what in str(ex.value), str(ex.value)
        with pytest.raises(rn.RNError) as ex:
            rn.rn_kcp_points(g, ok, bad, 3)
        assert ex.value.status == rn.RN_EINVAL
    with pytest.raises(rn.RNError):
        rn.rn_kcp_points(g, ok, ok, 0)
    # one-way arcs do not make an edge a point can lie on
    gd = rn.rn_graph_load(e.src, e.dst, e.w, e.n, flags=rn.RN_REORDER)
    with pytest.raises(rn.RNError) as ex:
        rn.rn_distance_join_points(gd, [(0, 1, 1)], [(1, 2, 1)], 100)
    assert "not an undirected edge" in str(ex.value)
    # empty sets
    assert len(rn.rn_distance_join_points(g, [], ok, 100)[0]) == 0
    assert len(rn.rn_kcp_points(g, ok, [], 5)[0]) == 0
    # points on a path: distances are gaps between positions
    u, v, d = rn.rn_distance_join_points(g, [(0, 1, 1), (2, 3, 5)], [(1, 2, 3), (3, 2, 0)], rn.RN_INF)
    assert list(zip(u.tolist(), v.tolist(), d.tolist())) == [(0, 0, 6), (0, 1, 14), (1, 0, 8), (1, 1, 0)]
