"""Device memory from torch's caching allocator through the allocator hook."""
import gc

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


def test_torch_caching_allocator(rn, oracle):
    import torch

    e = I.road_graph(20_000, 55_400, 101)
    R, S = I.disjoint_sets(e.n, 300, 400, 102)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    ref = og.join(R, S, 40_000)
    refk = og.kcp(R, S, 500)
    base = torch.cuda.memory_allocated()
    rn.use_torch_allocator(True)
    try:
        g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
        assert torch.cuda.memory_allocated() > base, "the graph's arrays did not come from torch"
        u, v, d = rn.rn_distance_join(g, R, S, 40_000)
        assert np.array_equal(u, ref.u) and np.array_equal(v, ref.v) and np.array_equal(d.astype(np.uint64), ref.d)
        u, v, d = rn.rn_kcp(g, R, S, 500)
        assert np.array_equal(u, refk.u) and np.array_equal(d.astype(np.uint64), refk.d)
    finally:
        rn.use_torch_allocator(False)
    # made under the hook, used and freed after it: the blocks go back to torch
    u, v, d = rn.rn_distance_join(g, R, S, 40_000)
    assert np.array_equal(u, ref.u)
    held = torch.cuda.memory_allocated()
    del g
    gc.collect()
    assert torch.cuda.memory_allocated() < held
    # and cudaMalloc serves again
    g2 = rn.rn_graph_load(e.src, e.dst, e.w, e.n)
    u, v, d = rn.rn_distance_join(g2, R, S, 40_000)
    assert np.array_equal(u, ref.u) and np.array_equal(v, ref.v)


def test_hook_rules(rn):
    import ctypes as C

    fn = rn._ALLOC_FN(lambda n, ctx: None)
    with pytest.raises(rn.RNError) as ex:
        rn._check(rn.lib().rn_set_allocator(C.cast(fn, C.c_void_p), None, None))
    assert ex.value.status == rn.RN_EINVAL
    # a hook that has no memory: allocation fails cleanly with RN_ENOMEM
    free = rn._FREE_FN(lambda p, ctx: None)
    rn._check(rn.lib().rn_set_allocator(C.cast(fn, C.c_void_p), C.cast(free, C.c_void_p), None))
    try:
        e = I.path_graph([1, 2, 3])
        with pytest.raises(rn.RNError) as ex:
            rn.rn_graph_load(e.src, e.dst, e.w, e.n)
        assert ex.value.status == rn.RN_ENOMEM
    finally:
        rn._check(rn.lib().rn_set_allocator(None, None, None))


def test_stats_log(rn, tmp_path):
    import json
    import os
    import subprocess
    import sys

    log = tmp_path / "stats.jsonl"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_1607_07696_gb300 import inputs as I, rn\n"
        "e = I.road_graph(5000, 13850, 3); g = rn.rn_graph_load(e.src, e.dst, e.w, e.n)\n"
        "R, S = I.disjoint_sets(e.n, 100, 200, 4)\n"
        "u, v, d = rn.rn_distance_join(g, R, S, 30000); k = rn.rn_kcp(g, R, S, 50)\n"
        "print(len(u))\n" % root)
    env = dict(os.environ, RN_STATS_LOG=str(log))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    assert [x["query"] for x in lines] == ["join", "kcp"]
    assert lines[0]["pairs"] == int(out.stdout.strip()) and lines[1]["pairs"] == 50
    assert all(x["device_ms"] > 0 and x["tiles"] > 0 for x in lines)
