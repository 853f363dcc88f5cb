"""The bounds-checked build (librn_checks.so, -DRN_CHECKS): every CSR, slot-map and node
index of the search is checked on the device.  Joins, k closest pairs, a batch and point
queries run through it must pass every check and equal the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, ROOT); sys.path.insert(0, ROOT + "/tests")
import numpy as np
import pins
from oracle import oracle as O
from paper_1607_07696_gb300 import inputs as I, rn
assert rn.LIB_PATH.endswith("librn_checks.so"), rn.LIB_PATH
o = O.default()
def same(got, ref):
    return all(np.array_equal(x, y.astype(x.dtype) if hasattr(y, "astype") else y) for x, y in zip(got, (ref.u, ref.v, ref.d)))
done = 0
for seed in range(4):
    e = I.road_graph(3000 + 7000 * seed, int(2.77 * (3000 + 7000 * seed)), 300 + seed)
    og = o.graph(e.n, e.src, e.dst, e.w)
    for T in (1, 32, 64, 128):  # 1: one warp per source
        g = rn.rn_graph_load(e.src, e.dst, e.w, e.n, cfg={"tile_width": T})
        R, S = I.disjoint_sets(e.n, 400, 600, 400 + seed)
        for theta in (20_000, rn.RN_INF):  # unbounded: every tile overflows and is retried
            assert same(rn.rn_distance_join(g, R, S, theta), og.join(R, S, min(theta, rn.RN_THETA_MAX)))
            done += 1
        if T == 1:  # several joins in one warp search, then in the tile search
            qs = [(R[:150], S[:200], 20_000), (R[150:], S[200:], 9_000), (R[150:170], S, rn.RN_INF)]
            for got, (r, s, th) in zip(rn.rn_join_many(g, qs), qs):
                assert same(got, og.join(r, s, min(th, rn.RN_THETA_MAX)))
            done += 1
        assert same(rn.rn_kcp(g, R, S, 300), og.kcp(R, S, 300)); done += 1
        best = pins.least_weights(e)
        rng = np.random.default_rng(seed)
        P, Q = pins.random_points(rng, best, 200), pins.random_points(rng, best, 300)
        assert same(rn.rn_distance_join_points(g, P, Q, 30_000), og.join_points(P, Q, 30_000)); done += 1
insts = []
for i in range(12):
    e = I.road_graph(500 + 400 * i, int(2.77 * (500 + 400 * i)), 500 + i)
    R, S = I.disjoint_sets(e.n, 20 + 10 * i, 50, 600 + i)
    insts.append((e, rn.rn_graph_load(e.src, e.dst, e.w, e.n), R, S, [5000, 60000, rn.RN_INF][i % 3]))
b = rn.rn_batch_create([(g, R, S, th) for (e, g, R, S, th) in insts])
for run in range(2):
    rn.rn_batch_run(b)
    for i, (e, g, R, S, th) in enumerate(insts):
        assert same(rn.rn_batch_pairs(b, i), o.graph(e.n, e.src, e.dst, e.w).join(R, S, min(th, rn.RN_THETA_MAX)))
print("checked", done)
"""


def test_checked_build_runs_clean():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1607_07696_gb300 import build as B

    lib = B.build(checks=True)
    env = dict(os.environ, RN_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + SCRIPT], env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout + r.stderr)[-4000:]
    assert "checked 68" in r.stdout
