"""Searches from S.  On an undirected graph d(u, v) = d(v, u), so a join or k closest
pairs may run its searches from the nodes of S instead of R (the engine does so by
default when S is at least a fifth smaller, or always with search_from = RN_FROM_S) and
must still return exactly the oracle's (u in R, v in S, d) triples in the oracle's order
-- the oracle always searches from R.  Directed graphs never swap."""
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


def assert_same(got, ref, what):
    u, v, d = got
    assert len(u) == len(ref), f"{what}: {len(u)} pairs, oracle {len(ref)}"
    assert np.array_equal(u, ref.u), f"{what}: u differs"
    assert np.array_equal(v, ref.v), f"{what}: v differs"
    assert np.array_equal(d.astype(np.uint64), ref.d), f"{what}: d differs"


def expect_from_s(sf, nR, nS):
    return {0: nS * 5 < nR * 4, 1: False, 2: True}[sf]


@pytest.mark.parametrize("seed", range(8))
def test_join_from_either_side(rn, oracle, seed):
    rng = np.random.default_rng(7100 + seed)
    n = int(rng.integers(500, 12_000))
    e = I.road_graph(n, int(2.77 * n), 7200 + seed)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    nR = int(rng.integers(1, min(800, n // 3)))
    nS = int(rng.integers(1, min(800, n // 3)))
    if seed % 2:
        nR, nS = max(nR, 4 * nS), nS  # S much smaller
    nR = min(nR, n // 2)
    R, S = I.disjoint_sets(e.n, nR, nS, 7300 + seed)
    full = og.join(R, S, rn.RN_THETA_MAX)
    T = [1, 32, 0, 64][seed % 4]
    for theta in (int(np.percentile(full.d, 3)) if len(full) else 10, int(np.median(full.d)) if len(full) else 10,
                  rn.RN_INF):
        ref = og.join(R, S, min(theta, rn.RN_THETA_MAX))
        for sf in (0, 1, 2):
            g = rn.rn_graph_load(e.src, e.dst, e.w, e.n, cfg={"tile_width": T, "search_from": sf})
            assert_same(rn.rn_distance_join(g, R, S, theta), ref, f"seed {seed} theta {theta} from {sf}")
            assert rn.rn_last_query_stats()["from_s"] == expect_from_s(sf, len(R), len(S))


@pytest.mark.parametrize("seed", range(6))
def test_kcp_from_either_side(rn, oracle, seed):
    rng = np.random.default_rng(7400 + seed)
    n = int(rng.integers(500, 8000))
    e = I.road_graph(n, int(2.77 * n), 7500 + seed) if seed % 3 else I.full_grid(70, 60, 1)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    nS = int(rng.integers(5, 120))
    R, S = I.disjoint_sets(e.n, int(rng.integers(4 * nS, 10 * nS)), nS, 7600 + seed)
    T = [1, 32, 0][seed % 3]
    for k in (1, 17, 500, 5000):
        ref = og.kcp(R, S, k)
        for sf in (0, 1, 2):
            g = rn.rn_graph_load(e.src, e.dst, e.w, e.n, cfg={"tile_width": T, "search_from": sf})
            assert_same(rn.rn_kcp(g, R, S, k), ref, f"seed {seed} k {k} from {sf}")
            assert rn.rn_last_query_stats()["from_s"] == expect_from_s(sf, len(R), len(S))


def test_directed_graphs_search_from_r(rn, oracle):
    e = I.random_graph(3000, 9000, 77, 1, 100)
    og = oracle.graph(e.n, e.src, e.dst, e.w, undirected=False)
    R, S = I.disjoint_sets(e.n, 600, 40, 78)
    with pytest.raises(rn.RNError) as ex:
        rn.rn_graph_load(e.src, e.dst, e.w, e.n, flags=rn.RN_REORDER, cfg={"search_from": 2})
    assert ex.value.status == rn.RN_EINVAL
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n, flags=rn.RN_REORDER)
    with pytest.raises(rn.RNError) as ex:
        rn.rn_graph_set_config(g, {"search_from": 2})
    assert ex.value.status == rn.RN_EINVAL
    with pytest.raises(rn.RNError) as ex:
        rn.rn_graph_set_config(g, {"search_from": 3})
    assert ex.value.status == rn.RN_EINVAL
    ref = og.join(R, S, 400)
    assert_same(rn.rn_distance_join(g, R, S, 400), ref, "directed, |S| < |R|")
    assert rn.rn_last_query_stats()["from_s"] == 0


def test_join_many_with_swapped_queries(rn, oracle):
    e = I.road_graph(20_000, 55_400, 81)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    rng = np.random.default_rng(82)
    qs = []
    for i in range(12):
        nR, nS = int(rng.integers(1, 600)), int(rng.integers(1, 600))
        R, S = I.disjoint_sets(e.n, nR, nS, 8300 + i)
        qs.append((R, S, int(rng.choice([20_000, 60_000, 150_000]))))
    many = rn.rn_join_many(g, qs)
    assert rn.rn_last_query_stats()["from_s"] == any(len(S) * 5 < len(R) * 4 for R, S, _ in qs)
    for i, (R, S, th) in enumerate(qs):
        assert_same(many[i], og.join(R, S, th), f"query {i}")


def test_batch_with_swapped_instances(rn, oracle):
    rng = np.random.default_rng(91)
    qs, refs = [], []
    for i in range(10):
        n = int(rng.integers(1000, 8000))
        e = I.road_graph(n, int(2.77 * n), 9100 + i)
        nS = int(rng.integers(2, 60))
        nR = int(rng.integers(1, n // 4)) if i % 3 else nS  # mostly |S| << |R|
        R, S = I.disjoint_sets(e.n, nR, nS, 9200 + i)
        og = oracle.graph(e.n, e.src, e.dst, e.w)
        th = int(rng.choice([30_000, 200_000, 2_000_000]))
        g = rn.rn_graph_load(e.src, e.dst, e.w, e.n, cfg={"search_from": [0, 1, 2][i % 3]})
        qs.append((g, R, S, th))
        refs.append(og.join(R, S, th))
    b = rn.rn_batch_create(qs)
    for run in range(2):
        rn.rn_batch_run(b)
        for i, ref in enumerate(refs):
            assert_same(rn.rn_batch_pairs(b, i), ref, f"run {run} instance {i}")
