"""Recursive two-seed bisection (Section 3, Algorithm 1; Eq. 1-2), run on the host
through the C ABI (no GPU needed)."""
import numpy as np
import pytest

from paper_1607_07696_gb300 import inputs as I


@pytest.fixture(scope="module")
def rn():
    from paper_1607_07696_gb300 import build as B

    B.build()
    from paper_1607_07696_gb300 import rn as RN

    return RN


def _grid(wd, ht, c, offset=0):
    g = I.full_grid(wd, ht, c)
    return g.src + offset, g.dst + offset, g.w


def test_order_is_a_permutation(rn):
    e = I.road_graph(5000, int(2.77 * 5000), 11)
    for alpha in (0.0, 0.5, 1.0):
        o = rn.rn_bisection_order(e.src, e.dst, e.w, e.n, cfg={"alpha": alpha, "leaf_size": 64})
        assert np.array_equal(np.sort(o), np.arange(e.n, dtype=np.uint32))


def test_bridge_is_the_cut(rn):
    # two 10x10 grids of light edges joined by one heavy edge: the first bisection must
    # cut exactly that edge (Section 3: a single remaining cross-edge is the longest one),
    # so with leaves of 100 nodes each grid is one contiguous id range.
    s1, d1, w1 = _grid(10, 10, 3)
    s2, d2, w2 = _grid(10, 10, 3, offset=100)
    src = np.concatenate([s1, s2, [99]])
    dst = np.concatenate([d1, d2, [100]])
    w = np.concatenate([w1, w2, [1000]])
    perm = np.random.default_rng(0).permutation(200).astype(np.uint32)  # hide the structure
    o = rn.rn_bisection_order(perm[src], perm[dst], w, 200, cfg={"leaf_size": 100})
    inv = np.argsort(perm)  # original id of relabelled node
    first = set(inv[o[:100]].tolist())
    assert first in ({*range(100)}, {*range(100, 200)})


def test_components_stay_whole(rn):
    # three disconnected paths: every component lands in one contiguous range
    src, dst, w = [], [], []
    sizes = [40, 25, 35]
    base = 0
    for s in sizes:
        src += list(range(base, base + s - 1))
        dst += list(range(base + 1, base + s))
        w += [1] * (s - 1)
        base += s
    o = rn.rn_bisection_order(src, dst, w, 100, cfg={"leaf_size": 40})
    comp = np.repeat(np.arange(3), sizes)
    labels = comp[o]
    changes = int(np.count_nonzero(labels[1:] != labels[:-1]))
    assert changes == 2


def test_leaves_are_compact(rn):
    # on a uniform grid, leaves of <= 64 nodes are compact regions and each keeps the order
    # its nodes were grown in: consecutive ids are grid neighbours or nearly (a random
    # order puts them ~42 steps apart), and any 64 consecutive ids -- at most two leaves --
    # span less than half the grid
    wd = 64
    s, d, w = _grid(wd, wd, 1)
    o = rn.rn_bisection_order(s, d, w, wd * wd, cfg={"leaf_size": 64})
    xs, ys = (o % wd).astype(int), (o // wd).astype(int)
    step = np.abs(np.diff(xs)) + np.abs(np.diff(ys))
    assert step.mean() < 6, step.mean()
    spans = []
    for i in range(0, wd * wd, 64):
        spans.append((xs[i:i + 64].max() - xs[i:i + 64].min()) + (ys[i:i + 64].max() - ys[i:i + 64].min()))
    assert np.median(spans) < wd // 2


def test_alpha_out_of_range_rejected(rn):
    with pytest.raises(rn.RNError):
        rn.rn_bisection_order([0], [1], [1], 2, cfg={"alpha": 1.5})


@pytest.mark.parametrize("seed", range(12))
def test_random_multigraphs_directed_and_not(rn, seed):
    # sparse random multigraphs (many components, self-loops, parallel and one-way arcs)
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 3000))
    e = I.random_graph(n, int(rng.integers(0, 3 * n)), seed, 1, 50)
    for flags in (0, rn.RN_UNDIRECTED):
        o = rn.rn_bisection_order(e.src, e.dst, e.w, e.n, flags=flags,
                                  cfg={"leaf_size": int(rng.integers(2, 300))})
        assert np.array_equal(np.sort(o), np.arange(e.n, dtype=np.uint32))
