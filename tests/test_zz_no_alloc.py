"""rn_distance_join_noalloc: the join for callers that cannot let the library allocate
device memory (their own allocator has reserved the device, or a cudaFree -- which
synchronises the whole device -- or an allocation that may fail mid-query is not
acceptable on their path).  Its scratch is one static device array shared by every
call, so two calls in a row must each give exactly what the allocating entry point
gives; the file sorts last so a failure here stops a -x run only after every other test.
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


def _dev(a):
    import torch

    return torch.as_tensor(np.asarray(a, dtype=np.int64).astype(np.int32), device="cuda")


def _reference(rn, g, R, S, theta):
    out = rn.DevicePairs()
    rn.rn_distance_join_dev(g, _dev(R), _dev(S), theta, out)
    return out.numpy()


def _noalloc(rn, g, R, S, theta, cap):
    import torch

    u = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    v = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    d = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    n = rn.rn_distance_join_noalloc(g, _dev(R), _dev(S), theta, u, v, d)
    torch.cuda.synchronize()
    return tuple(t[:n].cpu().numpy().view(np.uint32) for t in (u, v, d))


def test_two_calls_in_a_row_match_the_allocating_join(rn):
    e = I.road_graph(60_000, 166_200, 71)
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    R1, S1 = I.disjoint_sets(e.n, 1500, 2500, 72)
    R2, S2 = I.disjoint_sets(e.n, 900, 4000, 73)
    calls = [(R1, S1, 90_000), (R2, S2, 140_000)]
    for R, S, theta in calls:
        ref = _reference(rn, g, R, S, theta)
        got = _noalloc(rn, g, R, S, theta, cap=len(ref[0]) + 17)
        assert len(ref[0]) > 0
        for x, y in zip(got, ref):
            assert np.array_equal(x, y)  # integer distances: exact


def test_limits_are_rejected_clearly(rn):
    import torch

    e = I.path_graph(np.ones(70_000, dtype=np.uint32))
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    z = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(rn.RNError) as ex:  # |R| above the 65,536 limit
        rn.rn_distance_join_noalloc(g, _dev(np.arange(65_537)), _dev([69_999]), 10, z, z.clone(), z.clone())
    assert ex.value.status == rn.RN_EINVAL and "65536" in str(ex.value)
    with pytest.raises(rn.RNError) as ex:  # 40 pairs do not fit 1 entry
        rn.rn_distance_join_noalloc(g, _dev(np.arange(0, 80, 2)), _dev([81]), 1000, z, z.clone(), z.clone())
    assert ex.value.status == rn.RN_EINVAL and "output" in str(ex.value)


def test_tiles_that_outgrow_the_narrow_map(rn, oracle):
    """Every source's ball holds more than 7/8 of the narrow blocks' 8,192-slot map, so
    every tile of 32 sources overflows and is searched again by wide blocks (16,384
    slots, the static slab cut into four wide regions); the graph's 12,000 nodes fit that
    map, so every tile completes there.  Two calls in a row, each equal to the allocating
    join."""
    e = I.road_graph(12_000, 33_240, 91)
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    R, S = I.disjoint_sets(e.n, 256, 1000, 92)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    theta = max(int(np.sort(og.sssp(int(u))[0])[7200]) for u in R)
    for _ in range(2):
        ref = _reference(rn, g, R, S, theta)
        got = _noalloc(rn, g, R, S, theta, cap=len(ref[0]))
        assert len(ref[0]) > 0
        for x, y in zip(got, ref):
            assert np.array_equal(x, y)


def test_tiles_that_outgrow_the_wide_map_are_rejected(rn):
    """Unbounded searches on a graph whose largest component exceeds the wide map: the
    call reports RN_EINVAL naming the slab, and the next call still works."""
    import scipy.sparse as sp
    import torch
    from scipy.sparse.csgraph import connected_components

    e = I.road_graph(20_000, 55_400, 93)
    _, comp = connected_components(sp.coo_matrix((np.ones(e.m), (e.src, e.dst)), shape=(e.n, e.n)),
                                   directed=False)
    big = np.bincount(comp)
    assert big.max() > 16_384 * 7 // 8
    R, S = I.disjoint_sets(e.n, 256, 1000, 94)
    R = R[big[comp[R]] > 16_384 * 7 // 8]
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    z = torch.zeros(1 << 19, dtype=torch.int32, device="cuda")
    with pytest.raises(rn.RNError) as ex:
        rn.rn_distance_join_noalloc(g, _dev(R), _dev(S), rn.RN_INF, z, z.clone(), z.clone())
    assert ex.value.status == rn.RN_EINVAL and "slab" in str(ex.value)
    ref = _reference(rn, g, R[:8], S, 20_000)
    got = _noalloc(rn, g, R[:8], S, 20_000, cap=len(ref[0]) + 1)
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)
