"""The per-source protocol of the warp search (`k_source_search`), replayed on the CPU.

The GPU tests check the kernel itself against the oracle, but with the kernel's own queue
sizes a near-queue overflow is rare.  This sequential model follows the kernel's protocol
step by step -- slot flags (seen, dirty, queued), the double near queue with a capacity,
a push only when the flag update finds the slot unqueued, a full queue leaving the slot
dirty, the bucket boundary's pass that takes the least dirty distance, collects the next
bucket (or skips a gap to the bucket holding that distance) and clears stale queued flags,
the map's fill limit -- and runs it with queues of 1 to 64 entries against the oracle's
bounded Dijkstra (Section 4's local search), so every overflow path is exercised.  With
waves of 256 and 512 items (every item of a wave scanned before any is relaxed) it is
also the protocol of the cooperative search, whose four or eight warps share a wave.  Any
serial order of one warp's atomics is a valid execution of the kernel, so the model's
order is one of them.

What it pins: the dirty flag alone carries correctness (an improvement whose push is
dropped, or that lands beyond the bucket, is found by the next boundary pass); the queued
flag and the queues only save passes.  A model that sets the queued flag without the
dirty one fails here; one that never clears a stale queued flag still passes (it is only
slower), as the design intends.
"""
import numpy as np
import pytest

from paper_1607_07696_gb300 import inputs as I

NODE, SEEN, DIRTY, QUEUED = 0x0FFFFFFF, 0x20000000, 0x40000000, 0x80000000
EMPTY_KEY, INF, M32 = NODE, 0xFFFFFFFF, 0xFFFFFFFF


def csr(e):
    src = np.r_[e.src, e.dst]
    dst = np.r_[e.dst, e.src]
    w = np.r_[e.w, e.w]
    o = np.lexsort((w, dst, src))
    rp = np.zeros(e.n + 1, np.int64)
    np.add.at(rp, src[o] + 1, 1)
    return np.cumsum(rp).tolist(), dst[o].tolist(), w[o].tolist()


def warp_search(rp, adj, wt, y0, bound, delta, ms, qs, max_fill, wave=64):
    """Distances of every node within bound of y0, or None when the ball outgrows the
    map's fill limit (the kernel then reports the source for a larger map).  A round's
    items are taken `wave` at a time, all scanned before any is relaxed: 64 is the warp
    search's chunk, W x 64 the cooperative search's wave of W warps (whose warps' scans
    all precede the wave's relaxations, behind a block barrier)."""
    key = [EMPTY_KEY] * ms
    dist = [INF] * ms
    shift = 32 - (ms.bit_length() - 1)

    def slot(y):
        h = ((y * 0x9E3779B1) & M32) >> shift
        for _ in range(ms):
            if (key[h] & NODE) == y:
                return h, False
            if key[h] == EMPTY_KEY:
                key[h] = y
                return h, True
            h = (h + 1) & (ms - 1)
        return None, False

    h0 = ((y0 * 0x9E3779B1) & M32) >> shift
    key[h0] = y0 | DIRTY | QUEUED
    dist[h0] = 0
    qcur, fill = [h0], 1
    top = bound + 1
    tau = min(delta, top)

    def collect(lim):
        m, q = INF, []
        for h in range(ms):
            k = key[h]
            d = dist[h] if k & DIRTY else INF
            m = min(m, d)
            queued = bool(k & DIRTY) and d < lim and len(q) < qs
            if queued:
                q.append(h)
            key[h] = (k | QUEUED) if queued else (k & ~QUEUED & M32)
        return m, q

    while True:
        while qcur:  # rounds of the bucket
            nxt, nnext = [], 0
            for c0 in range(0, len(qcur), wave):
                items = []
                for x in qcur[c0:c0 + wave]:  # step A: take the item, clear its flags
                    k = key[x]
                    key[x] = (k & NODE) | SEEN
                    items.append((dist[x], k & NODE))
                for dv, y in items:  # step B: relax every arc of the chunk
                    for a in range(rp[y], rp[y + 1]):
                        nd = dv + wt[a]
                        if nd > bound:
                            continue
                        h, ins = slot(adj[a])
                        if h is None:
                            return None
                        fill += ins
                        old = dist[h]
                        dist[h] = min(old, nd)
                        if nd < old:
                            near = nd < tau
                            k0 = key[h]
                            key[h] = k0 | (DIRTY | QUEUED if near else DIRTY)
                            if near and not k0 & QUEUED:
                                if nnext < qs:
                                    nxt.append(h)
                                nnext += 1  # past qs: dropped, the slot stays dirty
                if fill > max_fill:
                    return None
            qcur = nxt[:qs]
        tau2 = min(tau + delta, top)
        m, q = collect(tau2)
        if m == INF:
            break
        if m >= tau2:  # an empty bucket: go to the one holding m
            tau = min((m // delta + 1) * delta, top)
            _, q = collect(tau)
        else:
            tau = tau2
        qcur = q
    return {key[h] & NODE: dist[h] for h in range(ms) if key[h] != EMPTY_KEY}


@pytest.mark.parametrize("seed,wave", [(0, 64), (1, 64), (2, 64), (3, 64), (4, 256), (5, 512)])
def test_protocol_matches_dijkstra(oracle, seed, wave):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(200, 800))
    e = I.road_graph(n, int(2.77 * n), 910 + seed)
    rp, adj, wt = csr(e)
    og = oracle.graph(e.n, e.src, e.dst, e.w)
    med = int(np.median(e.w))
    unreached = np.uint64(2**64 - 1)
    ms = 512
    runs = overflow = 0
    for s in rng.choice(e.n, 3, replace=False):
        for bound in (0, 4 * med, 15 * med):
            D, _ = og.sssp(int(s), bound)
            ref = {int(v): int(D[v]) for v in np.flatnonzero(D != unreached)}
            for delta in (med // 2 + 1, 16 * med, 1 << 24):
                for qs in (1, 4, 64):
                    got = warp_search(rp, adj, wt, int(s), bound, delta, ms, qs, ms * 7 // 8, wave)
                    runs += 1
                    if got is None:  # the ball is larger than the map may hold
                        overflow += 1
                        assert len(ref) > ms * 7 // 8 - 64
                        continue
                    assert got == ref, (seed, int(s), bound, delta, qs)
    assert runs - overflow > runs // 2


def warp_bitonic_model(vals, E):
    """The placement's in-register sort (`warp_bitonic<E>`): 32 lanes of E values, element
    lane * E + e in register e; partners at distance j >= E sit in lane ^ (j / E) (a
    shuffle), closer ones in register e ^ j of the same lane."""
    x = [[vals[lane * E + e] for e in range(E)] for lane in range(32)]
    k = 2
    while k <= 32 * E:
        j = k >> 1
        while j > 0:
            if j >= E:
                lj = j // E
                partner = [[x[lane ^ lj][e] for e in range(E)] for lane in range(32)]  # shfl_xor
                for lane in range(32):
                    lower = (lane & lj) == 0
                    for e in range(E):
                        up = ((lane * E + e) & k) == 0
                        p = partner[lane][e]
                        x[lane][e] = min(x[lane][e], p) if lower == up else max(x[lane][e], p)
            else:
                for lane in range(32):
                    for e in range(E):
                        if e & j == 0:
                            up = ((lane * E + e) & k) == 0
                            lo, hi = x[lane][e], x[lane][e ^ j]
                            if (lo > hi) == up:
                                x[lane][e], x[lane][e ^ j] = hi, lo
            j >>= 1
        k <<= 1
    return [x[lane][e] for lane in range(32) for e in range(E)]


@pytest.mark.parametrize("E", [1, 2, 4, 8])
def test_placement_network_sorts(E):
    rng = np.random.default_rng(E)
    pad = (1 << 64) - 1
    for cnt in sorted({1, 2, 31, 32, 33, 16 * E + 3, 32 * E - 1, 32 * E}):
        if cnt > 32 * E:
            continue
        for _ in range(5):
            v = rng.choice(1 << 40, size=cnt, replace=False).tolist()
            vals = v + [pad] * (32 * E - cnt)
            assert warp_bitonic_model(vals, E)[:cnt] == sorted(v), (E, cnt)
