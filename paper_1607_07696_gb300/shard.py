"""Host logic of multi-GPU runs: one process per GPU, R split across ranks, results gathered.

The sources of a join are independent (each u in R is searched on its own), so a query
shards by splitting R into contiguous parts, one per rank, over a graph every rank holds;
no data moves while the ranks search.  The join's result is then the union of the ranks'
pairs, re-sorted by (u, v); k closest pairs take every rank's k best and keep the k best
of those by (d, u, v) (each rank's k best contain every global winner it holds).  The
bench's weak-scaling run uses the same pieces: every rank joins its own R and S, the job
takes the slowest rank's time and the sum of the pairs.

Everything here is host-side marshalling over ``torch.distributed`` (NCCL between GPUs,
gloo on CPU for tests); the per-rank computation is the engine's.
"""
from __future__ import annotations

import numpy as np


def shard_bounds(n_items: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of rank's contiguous share of n_items (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    base, extra = divmod(n_items, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def gather_arrays(arrays: list[np.ndarray], group=None, device=None) -> list[list[np.ndarray]]:
    """All-gather of uint32 arrays of per-rank lengths: out[r][i] is rank r's arrays[i]."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    n = len(arrays[0])
    if any(len(a) != n for a in arrays):
        raise ValueError("arrays of one rank must have equal lengths")
    sizes = torch.tensor([n], dtype=torch.int64, device=device)
    all_sizes = [torch.zeros_like(sizes) for _ in range(world)]
    dist.all_gather(all_sizes, sizes, group=group)
    lens = [int(s.item()) for s in all_sizes]
    cap = max(lens) if lens else 0
    out: list[list[np.ndarray]] = [[] for _ in range(world)]
    for a in arrays:
        t = torch.zeros(cap, dtype=torch.int64, device=device)
        if n:
            t[:n] = torch.as_tensor(np.asarray(a, dtype=np.int64), device=device)
        parts = [torch.zeros_like(t) for _ in range(world)]
        dist.all_gather(parts, t, group=group)
        for r in range(world):
            out[r].append(parts[r][: lens[r]].cpu().numpy().astype(np.uint32))
    return out


def merge_join(parts: list[tuple[np.ndarray, np.ndarray, np.ndarray]]):
    """Union of the ranks' join pairs, sorted by (u, v)."""
    u = np.concatenate([p[0] for p in parts]) if parts else np.zeros(0, np.uint32)
    v = np.concatenate([p[1] for p in parts]) if parts else np.zeros(0, np.uint32)
    d = np.concatenate([p[2] for p in parts]) if parts else np.zeros(0, np.uint32)
    order = np.lexsort((v, u))
    return u[order], v[order], d[order]


def merge_kcp(parts: list[tuple[np.ndarray, np.ndarray, np.ndarray]], k: int):
    """The k best of the ranks' k best pairs, sorted by (d, u, v)."""
    u, v, d = (np.concatenate([p[i] for p in parts]) for i in range(3))
    order = np.lexsort((v, u, d))[:k]
    return u[order], v[order], d[order]


def job_time_and_pairs(total_ms: float, pairs: int, group=None, device=None) -> tuple[float, int]:
    """Weak scaling: the slowest rank's time and the pairs of all ranks."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    p = torch.tensor([pairs], dtype=torch.int64, device=device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), int(p.item())
