"""Parity of the GPU theta-join (through the C ABI) with the CPU oracle: bit-exact.

Distances are integers, so the bar is equality of every (u, v, d) triple and of the
order (sorted by (u, v)).  Sizes run from a handful of nodes to the 264k-node road-like
workload and the 1.07M-node clustered workload in full.
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


def dev_join(rn, g, R, S, theta, out=None):
    import torch

    out = out or rn.DevicePairs()
    dR = torch.as_tensor(np.asarray(R, dtype=np.int64).astype(np.int32), device="cuda")
    dS = torch.as_tensor(np.asarray(S, dtype=np.int64).astype(np.int32), device="cuda")
    rn.rn_distance_join_dev(g, dR, dS, theta, out)
    return out.numpy()


def assert_same(got, ref, what=""):
    u, v, d = got
    assert len(u) == len(ref), f"{what}: {len(u)} pairs, oracle {len(ref)}"
    assert np.array_equal(u, ref.u), f"{what}: u differs"
    assert np.array_equal(v, ref.v), f"{what}: v differs"
    assert np.array_equal(d.astype(np.uint64), ref.d), f"{what}: d differs"


def load(rn, e, flags=None, cfg=None):
    flags = rn.RN_UNDIRECTED | rn.RN_REORDER if flags is None else flags
    return rn.rn_graph_load(e.src, e.dst, e.w, e.n, flags=flags, cfg=cfg)


@pytest.mark.parametrize("T", [1, 32, 64, 128])
def test_grid4096_full(rn, oracle, T):
    w = I.c1_grid_join()
    e = w.graph
    g = load(rn, e, cfg={"tile_width": T})
    ref = oracle.graph(e.n, e.src, e.dst, e.w).join(w.R, w.S, w.theta)
    assert_same(dev_join(rn, g, w.R, w.S, w.theta), ref, f"grid T={T} dev")
    assert_same(rn.rn_distance_join(g, w.R, w.S, w.theta), ref, f"grid T={T} host")
    st = rn.rn_last_query_stats()
    assert st["pairs"] == len(ref) and st["tile_width"] == T
    assert st["slot_lanes"] == (st["slots"] if T == 1 else None) or T > 1


@pytest.mark.parametrize("T,ts", [(32, 1), (32, 7), (64, 33), (128, 100), (32, 32)])
def test_tile_sources(rn, oracle, T, ts):
    e = I.road_graph(30_000, 83_100, 41)
    g = load(rn, e, cfg={"tile_width": T, "tile_sources": ts})
    R, S = I.disjoint_sets(e.n, 700, 2000, 42)
    ref = oracle.graph(e.n, e.src, e.dst, e.w).join(R, S, 60_000)
    assert_same(dev_join(rn, g, R, S, 60_000), ref, f"T={T} sources/tile={ts}")
    assert rn.rn_last_query_stats()["tile_sources"] == min(ts, T)


@pytest.mark.parametrize("seed", range(24))
def test_random_small(rn, oracle, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 3000))
    kind = seed % 3
    if kind == 0:
        e = I.random_graph(n, int(rng.integers(0, 3 * n)), seed, 1, int(rng.integers(1, 1 << 16)))
    elif kind == 1:
        e = I.road_graph(max(n, 16), int(2.77 * max(n, 16)), seed)
    else:
        e = I.random_graph(n, int(2 * n), seed, 1, 7)
    n = e.n
    directed = seed % 4 == 3
    reorder = seed % 5 != 4
    flags = (0 if directed else rn.RN_UNDIRECTED) | (rn.RN_REORDER if reorder else 0)
    T = [1, 32, 64, 128][seed % 4]
    cfg = {"tile_width": T, "delta": int(rng.choice([0, 1, 50, 1 << 20]))}
    g = load(rn, e, flags, cfg)
    og = oracle.graph(n, e.src, e.dst, e.w, undirected=not directed)
    perm = rng.permutation(n)
    nR = int(rng.integers(1, max(2, n // 2)))
    nS = int(rng.integers(0, n - nR + 1))
    R, S = perm[:nR], perm[nR:nR + nS]
    D = og.sssp(int(R[0]))[0]
    finite = D[D != np.uint64(2**64 - 1)]
    thetas = [0, int(np.median(finite)) if finite.size else 5, rn.RN_INF]
    for theta in thetas:
        ref = og.join(R, S, min(theta, rn.RN_THETA_MAX))
        assert_same(dev_join(rn, g, R, S, theta), ref, f"seed {seed} theta {theta}")


def test_edge_cases(rn, oracle):
    e = I.road_graph(2000, 5540, 3)
    g = load(rn, e)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    R, S = I.disjoint_sets(e.n, 333, 400, 4)  # 333 = ragged last tile for every width
    th = 20000
    for (r, s) in [(R, S), (R[:0], S), (R, S[:0]), (R[:0], S[:0]), (R[:1], S), (R[:33], S[:1])]:
        assert_same(dev_join(rn, g, r, s, th), og.join(r, s, th), f"|R|={len(r)} |S|={len(s)}")
    # all but one node in R, the last in S
    allR = np.arange(e.n - 1)
    assert_same(dev_join(rn, g, allR, [e.n - 1], th), og.join(allR, [e.n - 1], th), "R = V - {s}")
    # theta at the largest allowed value and RN_INF agree
    a = dev_join(rn, g, R[:40], S, rn.RN_THETA_MAX)
    b = dev_join(rn, g, R[:40], S, rn.RN_INF)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_invalid_inputs_rejected(rn):
    import torch

    e = I.road_graph(500, 1385, 5)
    g = load(rn, e)
    bad = [([1, 2, 3], [4, 500]), ([1, 1], [4]), ([1], [4, 4]), ([1, 2], [2, 3])]
    for R, S in bad:
        with pytest.raises(rn.RNError) as ex:
            dev_join(rn, g, R, S, 100)
        assert ex.value.status == rn.RN_EINVAL
        with pytest.raises(rn.RNError) as ex:
            rn.rn_distance_join(g, R, S, 100)
        assert ex.value.status == rn.RN_EINVAL
    with pytest.raises(rn.RNError) as ex:
        rn.rn_distance_join(g, [1], [2], rn.RN_THETA_MAX + 1)
    assert ex.value.status == rn.RN_EINVAL
    # the graph still answers correctly after rejected calls
    R, S = [1, 2, 3], [4, 5, 6]
    u, v, d = dev_join(rn, g, R, S, 1 << 31)
    assert len(u) == 9


def test_slab_overflow_retry(rn, oracle):
    # unbounded search from 64 sources on a 40k-node graph: every tile's union ball is
    # the whole component, far beyond the shared-memory map, so tiles are searched
    # again with a global map
    e = I.road_graph(40_000, 110_800, 21)
    g = load(rn, e)
    R, S = I.disjoint_sets(e.n, 64, 3000, 22)
    ref = oracle.graph(e.n, e.src, e.dst, e.w).join(R, S, rn.RN_THETA_MAX)
    assert_same(dev_join(rn, g, R, S, rn.RN_INF), ref, "unbounded")
    assert rn.rn_last_query_stats()["retried_tiles"] > 0
    # and the engine is clean afterwards
    R2, S2 = I.disjoint_sets(e.n, 500, 500, 23)
    ref2 = oracle.graph(e.n, e.src, e.dst, e.w).join(R2, S2, 30000)
    assert_same(dev_join(rn, g, R2, S2, 30000), ref2, "after retry")


def test_pair_buffer_growth_and_repeat(rn, oracle):
    e = I.road_graph(20_000, 55_400, 31)
    g = load(rn, e)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    R, S = I.disjoint_sets(e.n, 40, 8000, 32)
    out = rn.DevicePairs()
    small = dev_join(rn, g, R[:2], S[:2], 100, out)
    ref = og.join(R, S, 400_000)  # hundreds of pairs per source: more than the first estimate
    got1 = dev_join(rn, g, R, S, 400_000, out)
    assert_same(got1, ref, "grown")
    got2 = dev_join(rn, g, R, S, 400_000, out)
    assert all(np.array_equal(x, y) for x, y in zip(got1, got2)), "repeat differs"
    assert len(small[0]) <= 4


def test_road264k_full(rn, oracle):
    spec = WORKLOADS["road264k_join"]
    w = I.c2_road_join(spec["theta"])
    e = w.graph
    assert e.m == spec["graph"]["m"]
    g = load(rn, e)
    ref = oracle.graph(e.n, e.src, e.dst, e.w).join(w.R, w.S, w.theta)
    got = dev_join(rn, g, w.R, w.S, w.theta)
    assert_same(got, ref, "road264k")
    assert_same(rn.rn_distance_join(g, w.R, w.S, w.theta), ref, "road264k host")
    st = rn.rn_last_query_stats()
    # the warp search's segments are placed in order (no 40-bit radix sort of all pairs)
    assert st["tile_width"] == 1 and st["launches"] < 16, st["launches"]


def test_road1070k_join_full(rn, oracle):
    """The 1.07M-node join (50,000 + 50,000 clustered nodes, theta for about 50 matches
    per source) in full: every one of the 2.8M pairs equal to the oracle's, searched on
    every host core."""
    from oracle import oracle as O

    spec = WORKLOADS["road1070k_clustered"]
    w = I.c3_road_clustered()
    e = w.graph
    g = load(rn, e)
    theta = spec["theta_join"]
    got = dev_join(rn, g, w.R, w.S, theta)
    ref = oracle.graph(e.n, e.src, e.dst, e.w).join_mt(w.R, w.S, theta, O.host_cores())
    assert len(ref) > 2_000_000
    assert_same(got, ref, "road1070k")
    assert_same(rn.rn_distance_join(g, w.R, w.S, theta), ref, "road1070k host")


@pytest.mark.parametrize("T,slots", [(32, 16384), (32, 65536), (64, 1 << 17), (128, 65536)])
def test_first_map_size(rn, oracle, T, slots):
    # unbounded search: every tile's ball is the whole 20k-node graph, larger than both
    # shared maps; a first map of 16384 slots overflows and is retried, a global first
    # map large enough is not
    e = I.road_graph(20_000, 55_400, 51)
    g = load(rn, e, cfg={"tile_width": T, "map_slots": slots})
    R, S = I.disjoint_sets(e.n, 300, 1500, 52)
    ref = oracle.graph(e.n, e.src, e.dst, e.w).join(R, S, rn.RN_THETA_MAX)
    assert_same(dev_join(rn, g, R, S, rn.RN_INF), ref, f"T={T} first map {slots}")
    st = rn.rn_last_query_stats()
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    _, comp = connected_components(sp.coo_matrix((np.ones(e.m), (e.src, e.dst)), shape=(e.n, e.n)),
                                   directed=False)
    size = int(np.bincount(comp)[comp[R]].max())  # the largest component holding a source
    assert size <= st["max_ball"] <= e.n
    assert st["retried_tiles"] > 0 or slots * 7 // 8 >= st["max_ball"]
    if slots * 7 // 8 < size:
        assert st["retried_tiles"] > 0
    with pytest.raises(rn.RNError):
        load(rn, e, cfg={"map_slots": 5000})


def test_source_search_routes(rn, oracle):
    """The warp-per-source search: sources whose ball outgrows a 2048-slot warp map are
    searched again with a larger warp map, those past the largest (8192) with the tile
    search; the default path follows the balls met so far."""
    e = I.road_graph(40_000, 110_800, 61)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    R, S = I.disjoint_sets(e.n, 300, 3000, 62)
    D = np.sort(og.sssp(int(R[0]))[0])
    for ball, routed in ((3000, "warp"), (20_000, "tiles")):
        theta = int(D[ball])
        g = load(rn, e, cfg={"tile_width": 1})
        assert_same(dev_join(rn, g, R, S, theta), og.join(R, S, theta), f"ball ~{ball}")
        st = rn.rn_last_query_stats()
        assert st["tile_width"] == 1 and st["retried_tiles"] > 0, st
        assert st["max_ball"] > 1792
    # default path: with no search behind the graph, the ball is estimated from the bound
    # (an unbounded one spans the graph: tiles from the first query on); a small bound
    # stays with the warp search, and then its measured balls decide
    g = load(rn, e)
    ref = og.join(R[:40], S, rn.RN_THETA_MAX)
    for i in range(2):
        assert_same(dev_join(rn, g, R[:40], S, rn.RN_INF), ref, f"unbounded {i}")
        assert rn.rn_last_query_stats()["tile_width"] == 32
    g = load(rn, e)
    for i in range(2):
        assert_same(dev_join(rn, g, R[:40], S, int(D[3000])), og.join(R[:40], S, int(D[3000])), f"small {i}")
        assert rn.rn_last_query_stats()["tile_width"] == 1
    theta = int(D[500])
    assert_same(dev_join(rn, g, R, S, theta), og.join(R, S, theta), "small after unbounded")
    st = rn.rn_last_query_stats()
    assert st["tile_width"] == 1 and st["slot_lanes"] == st["slots"]


@pytest.mark.parametrize("ball", [2500, 3400, 6500])
def test_large_warp_maps(rn, oracle, ball):
    """Balls that need 4096- or 8192-slot warp maps, searched by four warps per source:
    first with no history (a 2048-slot map, overflow, the cooperative search again), then
    with the measured balls (the cooperative search from the start); directed and
    undirected graphs, k closest pairs on the same maps."""
    e = I.road_graph(40_000, 110_800, 63)
    R, S = I.disjoint_sets(e.n, 700, 5000, 64)
    theta = int(np.sort(oracle.graph(e.n, e.src, e.dst, e.w).sssp(int(R[0]))[0])[ball])
    for directed in (False, True):
        og = oracle.graph(e.n, e.src, e.dst, e.w, undirected=not directed)
        flags = rn.RN_REORDER | (0 if directed else rn.RN_UNDIRECTED)
        g = load(rn, e, flags=flags, cfg={"tile_width": 1, "search_from": 1})
        ref = og.join(R, S, theta)
        for i in range(2):
            assert_same(dev_join(rn, g, R, S, theta), ref, f"ball ~{ball} directed {directed} run {i}")
            st = rn.rn_last_query_stats()
            assert st["tile_width"] == 1 and st["blocks_per_sm"] >= 1, st
        if not directed:
            assert st["max_ball"] > 1792
        k = max(1, len(ref) // 2)
        kref = og.kcp(R, S, k, theta)
        u, v, d = rn.rn_kcp(g, R, S, k, theta)
        assert_same((u, v, d), kref, f"kcp ball ~{ball} directed {directed}")


def test_long_segments_sorted(rn, oracle):
    """Sources with more than 256 pairs each (S dense around them): the warp search's
    segments are too long to place, and the pairs are radix sorted instead."""
    e = I.road_graph(30_000, 83_100, 71)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    R, S = I.disjoint_sets(e.n, 200, 20_000, 72)
    D = np.sort(og.sssp(int(R[0]))[0])
    theta = int(D[1200])  # balls of ~1,200 nodes, two thirds of them in S
    g = load(rn, e)
    ref = og.join(R, S, theta)
    assert_same(dev_join(rn, g, R, S, theta), ref, "dense S")
    st = rn.rn_last_query_stats()
    assert st["tile_width"] == 1 and st["launches"] > 16, st["launches"]
    # and both orders agree with the tile search's
    gt = load(rn, e, cfg={"tile_width": 32})
    assert_same(dev_join(rn, gt, R, S, theta), ref, "dense S, tiles")
    small = S[:500]
    assert_same(dev_join(rn, g, R, small, theta), og.join(R, small, theta), "sparse S, placed")
    assert rn.rn_last_query_stats()["launches"] < 16


def test_second_device(rn, oracle):
    """A graph loaded on a second GPU after a query on the first: every search kernel
    sets its shared-memory limit on each device it runs on, so both devices' joins (warp
    search and tile search) equal the oracle."""
    import torch

    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    e = I.road_graph(30_000, 83_100, 81)
    R, S = I.disjoint_sets(e.n, 400, 2000, 82)
    ref = oracle.graph(e.n, e.src, e.dst, e.w).join(R, S, 60_000)
    for dev in (0, 1):
        with torch.cuda.device(dev):
            for T in (1, 32):
                g = load(rn, e, cfg={"tile_width": T})
                assert_same(rn.rn_distance_join(g, R, S, 60_000), ref, f"device {dev} T={T}")
                assert rn.rn_last_query_stats()["blocks_per_sm"] >= 1
