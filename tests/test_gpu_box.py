"""Queries restricted to a rectangle (Section 2: geographically constrained queries touch
only the partitions whose MBR meets the constraint): the GPU join and k closest pairs of
the members of R and S lying in a box, bit-exact against the CPU oracle's answer on the
sets filtered by the same box (a node is in the closed box when xmin <= x <= xmax and
ymin <= y <= ymax, compared in the float32 coordinates both sides are given).
"""
import numpy as np
import pytest

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


def inside(xy32, ids, box):
    p = xy32[np.asarray(ids, dtype=np.int64)]
    m = (p[:, 0] >= box[0]) & (p[:, 0] <= box[2]) & (p[:, 1] >= box[1]) & (p[:, 1] <= box[3])
    return np.asarray(ids)[m]


@pytest.mark.parametrize("reorder", [True, False])
def test_box_join_and_kcp(rn, oracle, reorder):
    e = I.road_graph(40_000, 110_800, 101)
    xy32 = e.xy.astype(np.float32)
    flags = rn.RN_UNDIRECTED | (rn.RN_REORDER if reorder else 0)
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n, flags=flags, xy=xy32)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    R, S = I.disjoint_sets(e.n, 3000, 5000, 102)
    theta = 40_000
    rng = np.random.default_rng(103)
    boxes = [(0.0, 0.0, 1.0, 1.0), (0.2, 0.3, 0.55, 0.6), (0.9, 0.9, 0.95, 0.97), (2.0, 2.0, 3.0, 3.0)]
    for _ in range(4):
        x0, x1 = np.sort(rng.random(2))
        y0, y1 = np.sort(rng.random(2))
        boxes.append((float(x0), float(y0), float(x1), float(y1)))
    px = xy32[int(R[7])]
    boxes.append((float(px[0]), float(px[1]), float(px[0]), float(px[1])))  # one point
    for box in boxes:
        b32 = np.asarray(box, dtype=np.float32)
        for which in (rn.RN_BOX_R | rn.RN_BOX_S, rn.RN_BOX_R, rn.RN_BOX_S):
            Rb = inside(xy32, R, b32) if which & rn.RN_BOX_R else R
            Sb = inside(xy32, S, b32) if which & rn.RN_BOX_S else S
            ref = og.join(Rb, Sb, theta)
            assert same(rn.rn_distance_join_box(g, R, S, theta, b32, which), ref), f"join box {box} which {which}"
        st = rn.rn_last_query_stats()
        if box == (0.2, 0.3, 0.55, 0.6) and reorder:
            # most members were kept or dropped by their leaf's rectangle alone
            assert st["box_leaf_decided"] > (len(R) + len(S)) // 2, st["box_leaf_decided"]
        for k in (1, 100, 5000):
            Rb, Sb = inside(xy32, R, b32), inside(xy32, S, b32)
            ref = og.kcp(Rb, Sb, k, rn.RN_THETA_MAX)
            assert same(rn.rn_kcp_box(g, R, S, k, rn.RN_INF, b32), ref), f"kcp box {box} k {k}"


def test_box_rejections(rn):
    e = I.road_graph(2000, 5540, 104)
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    R, S = I.disjoint_sets(e.n, 10, 10, 105)
    with pytest.raises(rn.RNError) as ex:  # no coordinates were given
        rn.rn_distance_join_box(g, R, S, 1000, (0, 0, 1, 1))
    assert ex.value.status == rn.RN_EINVAL and "coordinates" in str(ex.value)
    gx = rn.rn_graph_load(e.src, e.dst, e.w, e.n, xy=e.xy)
    for box in ((0.5, 0, 0.4, 1), (0, 0.5, 1, 0.4), (0, float("nan"), 1, 1)):
        with pytest.raises(rn.RNError) as ex:
            rn.rn_distance_join_box(gx, R, S, 1000, box)
        assert ex.value.status == rn.RN_EINVAL
    with pytest.raises(rn.RNError) as ex:
        rn.rn_distance_join_box(gx, R, S, 1000, (0, 0, 1, 1), which=4)
    assert ex.value.status == rn.RN_EINVAL
    bad = e.xy.copy()
    bad[3, 1] = np.inf
    with pytest.raises(rn.RNError) as ex:
        rn.rn_graph_load(e.src, e.dst, e.w, e.n, xy=bad)
    assert ex.value.status == rn.RN_EINVAL
