"""Multi-process path on CPU: two gloo ranks split R, each answers its share (the CPU
oracle stands in for the rank's GPU), the results are gathered and merged, and the merge
must equal the unsharded answer exactly.  Also the weak-scaling aggregation of the bench
(slowest rank's time, all ranks' pairs).
"""
import os
import socket

import numpy as np
import pytest

from paper_1607_07696_gb300 import inputs as I
from paper_1607_07696_gb300 import shard as SH


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O

        e = I.road_graph(3000, 8310, 71)
        og = O.default().graph(e.n, e.src, e.dst, e.w)
        R, S = I.disjoint_sets(e.n, 301, 400, 72)  # 301: shares of unequal size
        lo, hi = SH.shard_bounds(len(R), rank, world)
        mine = og.join(R[lo:hi], S, 40_000)
        got = SH.gather_arrays([mine.u, mine.v, mine.d.astype(np.uint32)])
        u, v, d = SH.merge_join([tuple(x) for x in got])
        k = 250
        mk = og.kcp(R[lo:hi], S, k)
        gk = SH.gather_arrays([mk.u, mk.v, mk.d.astype(np.uint32)])
        ku, kv, kd = SH.merge_kcp([tuple(x) for x in gk], k)
        t, p = SH.job_time_and_pairs(10.0 + rank, 100 * (rank + 1))
        if rank == 0:
            full = og.join(R, S, 40_000)
            fk = og.kcp(R, S, k)
            ok = (np.array_equal(u, full.u) and np.array_equal(v, full.v)
                  and np.array_equal(d.astype(np.uint64), full.d)
                  and np.array_equal(ku, fk.u) and np.array_equal(kv, fk.v)
                  and np.array_equal(kd.astype(np.uint64), fk.d)
                  and t == 10.0 + world - 1 and p == 100 * world * (world + 1) // 2)
            with open(os.path.join(out_dir, "result"), "w") as f:
                f.write("ok" if ok else f"mismatch {len(u)} {len(full)} {t} {p}")
    finally:
        dist.destroy_process_group()


def test_two_rank_join_and_kcp(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    mp.start_processes(rank_main, args=(2, free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    assert (tmp_path / "result").read_text() == "ok"


def test_shard_bounds_cover_exactly():
    for n in (0, 1, 7, 300, 301):
        for world in (1, 2, 3, 8):
            spans = [SH.shard_bounds(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        SH.shard_bounds(5, 2, 2)
