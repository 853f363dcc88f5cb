"""Python face of the CPU oracle (``rn_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of the
benchmark may import this module; the engine never does.  It shares no code with the
CUDA path.  See ``rn_oracle.c`` for what each function computes and which passage of
the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rn_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")

OG_OK, OG_EINVAL, OG_ENOMEM = 0, 1, 2
INF = (1 << 64) - 1
THETA_MAX = 1 << 31


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


class _Pairs(C.Structure):
    _fields_ = [
        ("n", C.c_uint64),
        ("u", C.POINTER(C.c_uint32)),
        ("v", C.POINTER(C.c_uint32)),
        ("d", C.POINTER(C.c_uint64)),
        ("arcs", C.c_uint64),
    ]


@dataclass
class Pairs:
    """Result of a join or kCP: parallel arrays u, v, d and the algorithmic arc count."""

    u: np.ndarray
    v: np.ndarray
    d: np.ndarray
    arcs: int

    def __len__(self) -> int:
        return len(self.u)

    def triples(self) -> list[tuple[int, int, int]]:
        return list(zip(self.u.tolist(), self.v.tolist(), self.d.tolist()))


def build(src: str = SRC, out: str = LIB_PATH, extra: tuple[str, ...] = ()) -> str:
    """Compile the oracle with gcc into a shared library; returns its path."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if os.path.exists(out) and src == SRC and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", tmp, src, *extra]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(C.POINTER(t))


class Oracle:
    """Handle on one build of the oracle library (the real one, or a planted mutant)."""

    def __init__(self, lib_path: str | None = None):
        path = lib_path or build()
        self.lib = C.CDLL(path)
        L = self.lib
        L.og_graph_build.argtypes = [C.c_uint32, C.c_uint64, C.POINTER(C.c_uint32),
                                     C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.c_int,
                                     C.POINTER(C.c_void_p)]
        L.og_graph_free.argtypes = [C.c_void_p]
        L.og_graph_arcs.argtypes = [C.c_void_p]
        L.og_graph_arcs.restype = C.c_uint64
        L.og_graph_export.argtypes = [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_uint32),
                                      C.POINTER(C.c_uint32)]
        L.og_sssp.argtypes = [C.c_void_p, C.c_uint32, C.c_uint64, C.POINTER(C.c_uint64),
                              C.POINTER(C.c_uint64)]
        for fn in (L.og_join,):
            fn.argtypes = [C.c_void_p, C.POINTER(C.c_uint32), C.c_uint32, C.POINTER(C.c_uint32),
                           C.c_uint32, C.c_uint64, C.POINTER(_Pairs)]
        for fn in (L.og_kcp, L.og_kcp_bruteforce):
            fn.argtypes = [C.c_void_p, C.POINTER(C.c_uint32), C.c_uint32, C.POINTER(C.c_uint32),
                           C.c_uint32, C.c_uint64, C.c_uint64, C.POINTER(_Pairs)]
        L.og_join_mt.argtypes = [C.c_void_p, C.POINTER(C.c_uint32), C.c_uint32, C.POINTER(C.c_uint32),
                                 C.c_uint32, C.c_uint64, C.c_uint32, C.POINTER(_Pairs)]
        L.og_kcp_mt.argtypes = [C.c_void_p, C.POINTER(C.c_uint32), C.c_uint32, C.POINTER(C.c_uint32),
                                C.c_uint32, C.c_uint64, C.c_uint64, C.c_uint32, C.POINTER(_Pairs)]
        L.og_pairs_free.argtypes = [C.POINTER(_Pairs)]
        L.og_floyd_warshall.argtypes = [C.c_void_p, C.POINTER(C.c_uint64)]
        # points on edges: arrays of (a, b, t) uint32 triples
        L.og_join_points.argtypes = [C.c_void_p, C.POINTER(C.c_uint32), C.c_uint32, C.POINTER(C.c_uint32),
                                     C.c_uint32, C.c_uint64, C.POINTER(_Pairs)]
        L.og_kcp_points.argtypes = [C.c_void_p, C.POINTER(C.c_uint32), C.c_uint32, C.POINTER(C.c_uint32),
                                    C.c_uint32, C.c_uint64, C.c_uint64, C.POINTER(_Pairs)]

    def graph(self, n: int, src, dst, w, undirected: bool = True) -> "OGraph":
        return OGraph(self, n, src, dst, w, undirected)


class OGraph:
    """The oracle's own adjacency, built from an edge list."""

    def __init__(self, o: Oracle, n: int, src, dst, w, undirected: bool):
        self.o = o
        self.n = int(n)
        s, d, ww = _u32(src), _u32(dst), _u32(w)
        if not (len(s) == len(d) == len(ww)):
            raise ValueError("edge arrays differ in length")
        h = C.c_void_p()
        rc = o.lib.og_graph_build(self.n, len(s), _ptr(s, C.c_uint32), _ptr(d, C.c_uint32),
                                  _ptr(ww, C.c_uint32), int(bool(undirected)), C.byref(h))
        if rc:
            raise OracleError(rc, "og_graph_build")
        self.h = h

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.o.lib.og_graph_free(h)
            self.h = None

    @property
    def num_arcs(self) -> int:
        return int(self.o.lib.og_graph_arcs(self.h))

    def adjacency(self):
        a = self.num_arcs
        off = np.zeros(self.n + 1, np.uint64)
        to = np.zeros(max(a, 1), np.uint32)
        w = np.zeros(max(a, 1), np.uint32)
        self.o.lib.og_graph_export(self.h, _ptr(off, C.c_uint64), _ptr(to, C.c_uint32),
                                   _ptr(w, C.c_uint32))
        return off, to[:a], w[:a]

    def sssp(self, src: int, bound: int = THETA_MAX) -> tuple[np.ndarray, int]:
        dist = np.zeros(self.n + 1, np.uint64)
        arcs = C.c_uint64(0)
        rc = self.o.lib.og_sssp(self.h, int(src), int(bound), _ptr(dist, C.c_uint64), C.byref(arcs))
        if rc:
            raise OracleError(rc, "og_sssp")
        return dist[: self.n], int(arcs.value)

    def _pairs(self, fn, *args) -> Pairs:
        p = _Pairs()
        rc = fn(self.h, *args, C.byref(p))
        if rc:
            raise OracleError(rc, fn.__name__)
        n = int(p.n)
        try:
            u = np.ctypeslib.as_array(p.u, shape=(max(n, 1),))[:n].copy()
            v = np.ctypeslib.as_array(p.v, shape=(max(n, 1),))[:n].copy()
            d = np.ctypeslib.as_array(p.d, shape=(max(n, 1),))[:n].copy()
        finally:
            self.o.lib.og_pairs_free(C.byref(p))
        return Pairs(u, v, d, int(p.arcs))

    def join(self, R, S, theta: int) -> Pairs:
        r, s = _u32(R), _u32(S)
        return self._pairs(self.o.lib.og_join, _ptr(r, C.c_uint32), len(r), _ptr(s, C.c_uint32),
                           len(s), int(theta))

    def kcp(self, R, S, k: int, theta: int = THETA_MAX) -> Pairs:
        r, s = _u32(R), _u32(S)
        return self._pairs(self.o.lib.og_kcp, _ptr(r, C.c_uint32), len(r), _ptr(s, C.c_uint32),
                           len(s), int(k), int(theta))

    def join_mt(self, R, S, theta: int, threads: int) -> Pairs:
        """The join of ``join`` searched on ``threads`` host threads (same pairs, same order)."""
        r, s = _u32(R), _u32(S)
        return self._pairs(self.o.lib.og_join_mt, _ptr(r, C.c_uint32), len(r), _ptr(s, C.c_uint32),
                           len(s), int(theta), int(threads))

    def kcp_mt(self, R, S, k: int, theta: int = THETA_MAX, threads: int = 1) -> Pairs:
        """kCP of ``kcp`` searched on ``threads`` host threads sharing one bound."""
        r, s = _u32(R), _u32(S)
        return self._pairs(self.o.lib.og_kcp_mt, _ptr(r, C.c_uint32), len(r), _ptr(s, C.c_uint32),
                           len(s), int(k), int(theta), int(threads))

    def kcp_by_join(self, R, S, k: int, theta: int = THETA_MAX, threads: int = 1,
                    probe: int | None = None) -> Pairs:
        """kCP by its definition: the first k of all pairs within theta in (d, u, v)
        order.  The join is computed at a probe bound, doubled until it holds k pairs or
        reaches theta: once the join within the probe holds k pairs, no pair beyond the
        probe can be among the first k, so the answer is the first k of that join."""
        if k < 1:
            raise OracleError(OG_EINVAL, "kcp_by_join")
        theta = int(theta)
        b = theta if probe is None else max(1, min(int(probe), theta))
        while True:
            p = self.join_mt(R, S, b, threads)
            if len(p) >= k or b >= theta:
                break
            b = min(theta, 2 * b)
        order = np.lexsort((p.v, p.u, p.d))[:k]
        return Pairs(p.u[order], p.v[order], p.d[order], p.arcs)

    def kcp_bruteforce(self, R, S, k: int, theta: int = THETA_MAX) -> Pairs:
        r, s = _u32(R), _u32(S)
        return self._pairs(self.o.lib.og_kcp_bruteforce, _ptr(r, C.c_uint32), len(r),
                           _ptr(s, C.c_uint32), len(s), int(k), int(theta))

    def join_points(self, R, S, theta: int) -> Pairs:
        """Join of points on edges: R, S are (count, 3) arrays of (a, b, t); pairs are
        (index in R, index in S, distance)."""
        r, s = _points(R), _points(S)
        return self._pairs(self.o.lib.og_join_points, _ptr(r, C.c_uint32), len(r), _ptr(s, C.c_uint32),
                           len(s), int(theta))

    def kcp_points(self, R, S, k: int, theta: int = THETA_MAX) -> Pairs:
        r, s = _points(R), _points(S)
        return self._pairs(self.o.lib.og_kcp_points, _ptr(r, C.c_uint32), len(r), _ptr(s, C.c_uint32),
                           len(s), int(k), int(theta))

    def floyd_warshall(self) -> np.ndarray:
        D = np.zeros(self.n * self.n, np.uint64)
        self.o.lib.og_floyd_warshall(self.h, _ptr(D, C.c_uint64))
        return D.reshape(self.n, self.n)


def _points(P) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(P, dtype=np.uint32).reshape(-1, 3))
    return a if len(a) else np.zeros((1, 3), np.uint32)[:0]


def host_cores() -> int:
    """Cores this process may run on (its CPU affinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_model() -> str:
    """The host CPU's model name, from /proc/cpuinfo (x86: "model name"; Arm: the
    implementer and part numbers when no name is given)."""
    try:
        txt = open("/proc/cpuinfo").read()
    except OSError:
        return "unknown"
    fields = {}
    for line in txt.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            fields.setdefault(k.strip().lower(), v.strip())
    for key in ("model name", "cpu model", "hardware"):
        if fields.get(key):
            return fields[key]
    if "cpu part" in fields:
        return f"Arm implementer {fields.get('cpu implementer', '?')} part {fields['cpu part']}"
    return "unknown"


_default: Oracle | None = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default
