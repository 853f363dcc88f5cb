"""Batched theta-joins: many instances of uneven graph and set sizes in one persistent
launch per block shape, replayed from a CUDA graph, with autotuned plans.  Every
instance's pairs must equal the CPU oracle's (integer distances: exactly) and the same
query run alone through the plain entry point.
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


def same(got, ref):
    u, v, d = got
    return (len(u) == len(ref) and np.array_equal(u, ref.u) and np.array_equal(v, ref.v)
            and np.array_equal(d.astype(np.uint64), ref.d))


def small_batch(rn, count=40, seed=0):
    rng = np.random.default_rng(seed)
    inst = []
    for i in range(count):
        n = int(rng.integers(50, 6000))
        e = I.road_graph(n, int(2.77 * n), 1000 * seed + i)
        g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
        nR = int(rng.integers(1, max(2, n // 4)))
        nS = int(rng.integers(0, max(1, n // 4)))
        R, S = I.disjoint_sets(e.n, nR, nS, 77 + i)
        theta = int(rng.choice([0, 3000, 20000, 60000, rn.RN_INF]))
        inst.append((e, g, R, S, theta))
    return inst


def test_batch_matches_oracle_eager_and_replayed(rn, oracle):
    inst = small_batch(rn)
    b = rn.rn_batch_create([(g, R, S, th) for (e, g, R, S, th) in inst])
    refs = [oracle.graph(e.n, e.src, e.dst, e.w).join(R, S, min(th, rn.RN_THETA_MAX))
            for (e, g, R, S, th) in inst]
    for run in range(3):  # eager, then graph replays
        rn.rn_batch_run(b)
        for i, ref in enumerate(refs):
            assert same(rn.rn_batch_pairs(b, i), ref), f"run {run} instance {i}"
    st = rn.rn_batch_stats_get(b)
    assert st["eager_runs"] >= 1 and st["graph_runs"] >= 1, st
    assert st["pairs"] == sum(len(r) for r in refs)


def test_autotuned_batch_and_one_shot(rn, oracle):
    inst = small_batch(rn, count=24, seed=1)
    qs = [(g, R, S, th) for (e, g, R, S, th) in inst]
    refs = [oracle.graph(e.n, e.src, e.dst, e.w).join(R, S, min(th, rn.RN_THETA_MAX))
            for (e, g, R, S, th) in inst]
    b = rn.rn_batch_create(qs, autotune=True)
    rn.rn_batch_run(b)
    assert rn.rn_batch_stats_get(b)["tuned"] in (1, 2, 3)
    for i, ref in enumerate(refs):
        assert same(rn.rn_batch_pairs(b, i), ref), f"tuned instance {i}"
    outs = rn.rn_join_batch(qs)
    for i, ref in enumerate(refs):
        assert same(outs[i], ref), f"one-shot instance {i}"


def test_bad_query_is_named(rn):
    e = I.road_graph(300, 831, 5)
    g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    with pytest.raises(rn.RNError) as ex:
        rn.rn_batch_create([(g, [1, 2], [3], 100), (g, [1, 2], [2], 100)])
    assert ex.value.status == rn.RN_EINVAL and "query 1" in str(ex.value)


def test_batch512_alone_and_in_the_mix(rn, oracle):
    import torch

    specs = I.c4_batch_specs()
    thetas = WORKLOADS["batch512"]["theta"]
    inst = []
    for sp, th in zip(specs, thetas):
        e, R, S = I.c4_instance(sp)
        inst.append((e, rn.rn_graph_load(e.src, e.dst, e.w, e.n), R, S, th))
    b = rn.rn_batch_create([(g, R, S, th) for (e, g, R, S, th) in inst])
    rn.rn_batch_run(b)
    rn.rn_batch_run(b)  # replay
    out = rn.DevicePairs()
    rng = np.random.default_rng(3)
    check = set(rng.choice(len(inst), size=40, replace=False).tolist())
    for i, (e, g, R, S, th) in enumerate(inst):
        u, v, d, n = rn.rn_batch_pairs_dev(b, i)
        dR = torch.as_tensor(R.astype(np.int32), device="cuda")
        dS = torch.as_tensor(S.astype(np.int32), device="cuda")
        alone = rn.rn_distance_join_dev(g, dR, dS, th, out)
        assert alone == n, f"instance {i}: {n} pairs in the batch, {alone} alone"
        got = rn.rn_batch_pairs(b, i)
        assert all(np.array_equal(x, y) for x, y in zip(got, out.numpy())), f"instance {i} differs alone"
        if i in check:
            ref = oracle.graph(e.n, e.src, e.dst, e.w).join(R, S, th)
            assert same(got, ref), f"instance {i} differs from the oracle"


def test_batch_edge_cases(rn, oracle):
    # empty sets, theta 0 and unbounded, one-node and two-node graphs, a graph shared by
    # several instances, an instance whose every source overflows the shared map
    big = I.road_graph(30_000, 83_100, 91)
    gb = rn.rn_graph_load(big.src, big.dst, big.w, big.n)
    tiny = I.path_graph([5])
    gt = rn.rn_graph_load(tiny.src, tiny.dst, tiny.w, tiny.n)
    one = I.random_graph(1, 0, 1)
    g1 = rn.rn_graph_load(one.src, one.dst, one.w, one.n)
    # a random (non-planar) graph: a bound of a few median weights, whose ball the planar
    # estimate puts within a warp map, reaches most of the graph -- the warp search's
    # sources overflow, go to tiles one by one, and the instance moves to tiles
    rnd = I.random_graph(20_000, 60_000, 95, 1, 100)
    gr = rn.rn_graph_load(rnd.src, rnd.dst, rnd.w, rnd.n)
    Rr, Sr = I.disjoint_sets(rnd.n, 64, 400, 96)
    Rb, Sb = I.disjoint_sets(big.n, 300, 500, 92)
    inst = [
        (big, gb, Rb, Sb, 40_000),
        (big, gb, Rb[:0], Sb, 40_000),        # no sources
        (big, gb, Rb[:7], Sb[:0], 40_000),    # no targets
        (big, gb, Rb[:50], Sb, 0),            # theta 0: nothing (sets are disjoint)
        (big, gb, Rb[:40], Sb, rn.RN_INF),    # unbounded: whole-graph balls
        (tiny, gt, np.array([0]), np.array([1]), 5),
        (tiny, gt, np.array([1]), np.array([0]), 4),
        (one, g1, np.array([0]), np.array([], dtype=np.int64), 3),
        (rnd, gr, Rr, Sr, 8 * int(np.median(rnd.w))),
    ]
    b = rn.rn_batch_create([(g, R, S, th) for (e, g, R, S, th) in inst])
    for run in range(3):
        rn.rn_batch_run(b)
        for i, (e, g, R, S, th) in enumerate(inst):
            ref = oracle.graph(e.n, e.src, e.dst, e.w).join(R, S, min(th, rn.RN_THETA_MAX))
            assert same(rn.rn_batch_pairs(b, i), ref), f"run {run} instance {i}"
    with pytest.raises(rn.RNError):
        rn.rn_batch_pairs(b, len(inst))
    with pytest.raises(rn.RNError):
        rn.rn_batch_create([])
