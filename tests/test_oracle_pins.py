"""The CPU oracle against its pins (no GPU needed)."""
import pytest

import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(oracle, pin):
    pin(oracle)


def test_floyd_warshall_seeds_0_to_999(oracle):
    """Join and kCP (every k up to 150, and spread values beyond) against Floyd-Warshall
    brute force on 1,000 random (multi)graphs of up to 64 nodes, directed and undirected."""
    import numpy as np

    from paper_1607_07696_gb300 import inputs as I
    from pins import INF64, THETA_MAX, _fw_pairs

    for seed in range(1000):
        rng = np.random.default_rng(50_000 + seed)
        n = int(rng.integers(1, 65))
        e = I.random_graph(n, int(rng.integers(0, 4 * n + 1)), 60_000 + seed, 1, int(rng.choice([3, 50, 5000])))
        g = oracle.graph(n, e.src, e.dst, e.w, undirected=bool(seed % 4))
        D = g.floyd_warshall()
        perm = rng.permutation(n)
        nR = int(rng.integers(1, n + 1))
        nS = int(rng.integers(0, n - nR + 1))
        R, S = perm[:nR], perm[nR:nR + nS]
        finite = D[D != INF64]
        for theta in [0, THETA_MAX] + ([int(np.median(finite))] if finite.size else []):
            want = sorted(_fw_pairs(D, R, S, theta))
            assert g.join(R, S, theta).triples() == want, f"seed {seed} theta {theta}"
            byd = sorted(want, key=lambda t: (t[2], t[0], t[1]))
            ks = list(range(1, min(len(byd), 150) + 2)) + [len(byd), len(byd) + 7]
            for k in sorted({max(1, k) for k in ks}):
                assert g.kcp(R, S, k, theta).triples() == byd[:k], f"seed {seed} theta {theta} k {k}"
