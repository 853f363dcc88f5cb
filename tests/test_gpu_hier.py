"""The hierarchical variant (Section 4, Algorithms 2-4: searches local to the parts of the
partition hierarchy, expansion over the arcs that leave a part, the searches from their
far ends shared by every source that reaches them): its join and k closest pairs must
equal the CPU oracle's, triple for triple, at every granularity of the hierarchy.
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


@pytest.mark.parametrize("seed", range(16))
def test_hier_random_small(rn, oracle, seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(20, 3000))
    if seed % 2:
        e = I.road_graph(n, int(2.77 * n), 910 + seed)
    else:
        e = I.random_graph(n, int(rng.integers(n, 3 * n)), 910 + seed, 1, int(rng.choice([3, 100, 5000])))
    directed = seed % 5 == 4
    flags = (0 if directed else rn.RN_UNDIRECTED) | (rn.RN_REORDER if seed % 3 else 0)
    leaf = int(rng.choice([8, 32, 128]))
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n, flags=flags, cfg={"leaf_size": leaf})
    og = oracle.graph(e.n, e.src, e.dst, e.w, undirected=not directed)
    perm = rng.permutation(e.n)
    nR = int(rng.integers(1, max(2, e.n // 3)))
    nS = int(rng.integers(1, e.n - nR + 1))
    R, S = perm[:nR], perm[nR:nR + nS]
    full = og.join(R, S, rn.RN_THETA_MAX)
    med = int(np.median(full.d)) if len(full) else 10
    for part in (0, 4 * leaf, 32 * leaf):
        for theta in (0, med // 3, med, rn.RN_INF):
            ref = og.join(R, S, min(theta, rn.RN_THETA_MAX))
            assert same(rn.rn_distance_join_hier(g, R, S, theta, part), ref), f"join part {part} theta {theta}"
        st = rn.rn_last_hier_stats()
        assert st["max_part"] <= max(part, leaf)
        for k in (1, 17, max(1, len(full) // 2), len(full) + 3):
            ref = og.kcp(R, S, k, rn.RN_THETA_MAX)
            assert same(rn.rn_kcp_hier(g, R, S, k, rn.RN_INF, part), ref), f"kcp part {part} k {k}"


def test_hier_road_and_routes(rn, oracle):
    """A 30k-node road graph: parts of 512 to 4096 nodes; the exit routes carry the pairs
    whose shortest path leaves the source's part, and the result equals the flat search."""
    e = I.road_graph(30_000, 83_100, 931)
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    R, S = I.disjoint_sets(e.n, 1500, 3000, 932)
    for theta in (20_000, 80_000):
        ref = og.join(R, S, theta)
        flat = rn.rn_distance_join(g, R, S, theta)
        assert same(flat, ref)
        for part in (0, 1024, 4096):
            assert same(rn.rn_distance_join_hier(g, R, S, theta, part), ref), f"theta {theta} part {part}"
            st = rn.rn_last_hier_stats()
            assert st["exit_searches"] > 0 and st["border_routes"] > 0 and st["local_pairs"] <= len(ref)
    for k in (10, 1000, 20_000):
        assert same(rn.rn_kcp_hier(g, R, S, k, rn.RN_INF, 2048), og.kcp(R, S, k)), f"kcp k {k}"


def test_hier_rejections(rn):
    e = I.road_graph(20_000, 55_400, 941)
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    R, S = I.disjoint_sets(e.n, 10, 10, 942)
    with pytest.raises(rn.RNError) as ex:  # below the leaf size
        rn.rn_distance_join_hier(g, R, S, 1000, 100)
    assert ex.value.status == rn.RN_EINVAL
    with pytest.raises(rn.RNError) as ex:  # the whole graph as one part: larger than a warp map holds
        rn.rn_distance_join_hier(g, R, S, 1000, 1 << 30)
    assert ex.value.status == rn.RN_EINVAL
    with pytest.raises(rn.RNError) as ex:  # sets that overlap
        rn.rn_distance_join_hier(g, [1, 2], [2], 1000, 0)
    assert ex.value.status == rn.RN_EINVAL
