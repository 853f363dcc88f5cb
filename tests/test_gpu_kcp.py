"""Parity of the GPU k-closest-pairs query (through the C ABI) with the CPU oracle.

The answer is unique under the (d, u, v) order, so the bar is equality of every triple
and of the order.  Small graphs are compared in full; the 1.07M-node clustered workload
is checked on samples: every sampled returned pair's distance against a single-source
oracle search, and completeness below the k-th distance for sampled sources.
"""
import json
import os

import numpy as np
import pytest

from paper_1607_07696_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORKLOADS = json.load(open(os.path.join(ROOT, "tests", "golden", "workloads.json")))


@pytest.fixture(scope="module")
def rn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1607_07696_gb300 import build as B

    B.build()
    from paper_1607_07696_gb300 import rn as RN

    return RN


def dev_kcp(rn, g, R, S, k, theta):
    import torch

    out = rn.DevicePairs()
    dR = torch.as_tensor(np.asarray(R, dtype=np.int64).astype(np.int32), device="cuda")
    dS = torch.as_tensor(np.asarray(S, dtype=np.int64).astype(np.int32), device="cuda")
    rn.rn_kcp_dev(g, dR, dS, k, theta, out)
    return out.numpy()


def assert_same(got, ref, what):
    u, v, d = got
    assert len(u) == len(ref), f"{what}: {len(u)} pairs, oracle {len(ref)}"
    assert np.array_equal(u, ref.u), f"{what}: u differs"
    assert np.array_equal(v, ref.v), f"{what}: v differs"
    assert np.array_equal(d.astype(np.uint64), ref.d), f"{what}: d differs"


@pytest.mark.parametrize("seed", range(16))
def test_random_small(rn, oracle, seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(10, 3000))
    if seed % 2:
        e = I.road_graph(n, int(2.77 * n), seed)
    else:
        e = I.random_graph(n, int(rng.integers(n, 3 * n)), seed, 1, int(rng.choice([3, 100, 5000])))
    directed = seed % 5 == 4
    flags = (0 if directed else rn.RN_UNDIRECTED) | rn.RN_REORDER
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n, flags=flags, cfg={"tile_width": [32, 64, 128][seed % 3]})
    og = oracle.graph(e.n, e.src, e.dst, e.w, undirected=not directed)
    perm = rng.permutation(e.n)
    nR = int(rng.integers(1, e.n // 2))
    nS = int(rng.integers(1, e.n - nR + 1))
    R, S = perm[:nR], perm[nR:nR + nS]
    full = og.join(R, S, rn.RN_THETA_MAX)
    for k in sorted({1, 7, 100, max(1, len(full) // 3), max(1, len(full)), len(full) + 5}):
        for theta in (rn.RN_INF, int(np.median(full.d)) if len(full) else 10):
            ref = og.kcp(R, S, k, min(theta, rn.RN_THETA_MAX))
            assert_same(dev_kcp(rn, g, R, S, k, theta), ref, f"seed {seed} k {k} theta {theta}")


def test_ties_on_a_uniform_grid(rn, oracle):
    # every edge weight 1: distances are Manhattan, so ties at the k-th distance abound
    e = I.full_grid(60, 50, 1)
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    R, S = I.disjoint_sets(e.n, 400, 600, 9)
    for k in (1, 2, 3, 50, 51, 777, 5000):
        assert_same(dev_kcp(rn, g, R, S, k, rn.RN_INF), og.kcp(R, S, k), f"grid ties k {k}")
    # host-buffer entry point too
    u, v, d = rn.rn_kcp(g, R, S, 333)
    assert_same((u, v, d), og.kcp(R, S, 333), "host kcp")


def test_grid4096(rn, oracle):
    w = I.c1_grid_join()
    e = w.graph
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    for k in (1, 10, 100, 1000, 6356, 20000):
        assert_same(dev_kcp(rn, g, w.R, w.S, k, rn.RN_INF), og.kcp(w.R, w.S, k), f"grid4096 k {k}")
    # theta below the k-th distance: every pair within theta, fewer than k
    assert_same(dev_kcp(rn, g, w.R, w.S, 5000, 900), og.kcp(w.R, w.S, 5000, 900), "theta-bounded")
    st = rn.rn_last_query_stats()
    assert st["passes"] >= 1


def test_invalid(rn):
    e = I.path_graph([1, 2, 3])
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    with pytest.raises(rn.RNError) as ex:
        rn.rn_kcp(g, [0], [1], 0)
    assert ex.value.status == rn.RN_EINVAL
    with pytest.raises(rn.RNError) as ex:
        rn.rn_kcp(g, [0, 1], [1], 3)
    assert ex.value.status == rn.RN_EINVAL


@pytest.mark.parametrize("k", [100, 10_000, 1_000_000])
def test_road1070k_clustered_sampled(rn, oracle, k):
    w = I.c3_road_clustered()
    e = w.graph
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    u, v, d = dev_kcp(rn, g, w.R, w.S, k, rn.RN_INF)
    assert len(u) == k
    key = [(int(a), int(b), int(c)) for a, b, c in zip(d, u, v)]
    assert key == sorted(key), "not sorted by (d, u, v)"
    assert len(set(zip(u.tolist(), v.tolist()))) == k, "repeated pair"
    assert np.isin(u, w.R).all() and np.isin(v, w.S).all()
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    rng = np.random.default_rng(k)
    dk = int(d[-1])
    # sampled returned pairs: their distances, one source at a time
    idx = rng.choice(len(u), size=min(40, len(u)), replace=False)
    for i in idx:
        dist, _ = og.sssp(int(u[i]), int(d[i]))
        assert int(dist[v[i]]) == int(d[i]), f"pair {i}: distance differs"
    # completeness: for sampled sources, every S node closer than the k-th distance (or
    # tied with it and earlier in (u, v) order) is in the answer
    got = set(zip(u.tolist(), v.tolist()))
    sources = np.unique(np.concatenate([u[idx], rng.choice(w.R, size=20, replace=False)]))
    S_set = np.zeros(e.n, bool)
    S_set[w.S] = True
    lu, lv = int(u[-1]), int(v[-1])
    for s in sources:
        dist, _ = og.sssp(int(s), dk)
        for x in np.nonzero(S_set & (dist <= dk))[0]:
            dx = int(dist[x])
            if (dx, int(s), int(x)) <= (dk, lu, lv):
                assert (int(s), int(x)) in got, f"missing ({s}, {x}, {dx})"
