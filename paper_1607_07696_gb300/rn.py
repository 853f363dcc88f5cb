"""Python binding of the engine's C ABI (include/rn.h): argument marshalling only.

Every function here forwards to the function of the same name in ``librn.so``; all the
work of a query runs in the library's CUDA kernels.  The library is built in-tree by
``paper_1607_07696_gb300.build`` (or ``__graft_entry__.build()``); importing this module
without it raises -- there is no fallback of any kind.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

# RN_LIBRARY may name another build of the engine (the bounds-checked librn_checks.so)
LIB_PATH = os.environ.get("RN_LIBRARY") or os.path.join(os.path.dirname(os.path.abspath(__file__)), "librn.so")

RN_OK, RN_EINVAL, RN_ENOMEM, RN_ECUDA, RN_ETIMEOUT = 0, 1, 2, 3, 4
RN_ECANCELLED, RN_EBUSY, RN_EINTERNAL, RN_ENOTIMPL = 5, 6, 7, 8
RN_UNDIRECTED, RN_REORDER = 1, 2
RN_INF = 0xFFFFFFFF
RN_FROM_AUTO, RN_FROM_R, RN_FROM_S = 0, 1, 2
RN_THETA_MAX = 1 << 31
RN_WEIGHT_LIMIT = 1 << 24  # weights must be below it

_NAMES = {0: "RN_OK", 1: "RN_EINVAL", 2: "RN_ENOMEM", 3: "RN_ECUDA", 4: "RN_ETIMEOUT",
          5: "RN_ECANCELLED", 6: "RN_EBUSY", 7: "RN_EINTERNAL", 8: "RN_ENOTIMPL"}


class RNError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_NAMES.get(status, status)}: {msg}")
        self.status = status


class rn_pairs(C.Structure):
    _fields_ = [("u", C.POINTER(C.c_uint32)), ("v", C.POINTER(C.c_uint32)),
                ("d", C.POINTER(C.c_uint32)), ("n", C.c_uint64)]


class rn_dpairs(C.Structure):
    _fields_ = [("u", C.c_void_p), ("v", C.c_void_p), ("d", C.c_void_p), ("n", C.c_uint64),
                ("cap", C.c_uint64)]


class rn_config(C.Structure):
    _fields_ = [("tile_width", C.c_uint32), ("tile_sources", C.c_uint32), ("delta", C.c_uint32),
                ("leaf_size", C.c_uint32), ("alpha", C.c_float), ("map_slots", C.c_uint32),
                ("search_from", C.c_uint32)]


class rn_graph_stats(C.Structure):
    _fields_ = [("n", C.c_uint32), ("arcs", C.c_uint64), ("max_degree", C.c_uint32),
                ("median_weight", C.c_uint32), ("flags", C.c_uint32), ("reorder_ms", C.c_double),
                ("device_bytes", C.c_uint64)]


class rn_query_stats(C.Structure):
    _fields_ = [("pairs", C.c_uint64), ("tiles", C.c_uint64), ("retried_tiles", C.c_uint64),
                ("scans", C.c_uint64), ("tile_width", C.c_uint32), ("tile_sources", C.c_uint32),
                ("delta", C.c_uint32),
                ("passes", C.c_uint32), ("theta_final", C.c_uint32), ("launches", C.c_uint32),
                ("blocks_per_sm", C.c_uint32),
                ("slots", C.c_uint64), ("slot_arcs", C.c_uint64), ("device_ms", C.c_double),
                ("search_ms", C.c_double), ("rounds", C.c_uint64), ("round_items", C.c_uint64),
                ("boundaries", C.c_uint64), ("cycles_rounds", C.c_uint64),
                ("cycles_boundaries", C.c_uint64), ("cycles_emission", C.c_uint64),
                ("cycles_step_a", C.c_uint64), ("round_arcs", C.c_uint64), ("max_ball", C.c_uint64),
                ("retry_ms", C.c_double), ("dirty_groups", C.c_uint64), ("slot_lanes", C.c_uint64),
                ("box_leaf_decided", C.c_uint64), ("search_pairs", C.c_uint64), ("from_s", C.c_uint32)]


class rn_query(C.Structure):
    _fields_ = [("g", C.c_void_p), ("R", C.POINTER(C.c_uint32)), ("nR", C.c_uint32),
                ("S", C.POINTER(C.c_uint32)), ("nS", C.c_uint32), ("theta", C.c_uint32)]


class rn_batch_config(C.Structure):
    _fields_ = [("autotune", C.c_uint32), ("use_graph", C.c_uint32)]


class rn_batch_stats(C.Structure):
    _fields_ = [("instances", C.c_uint32), ("groups", C.c_uint32), ("tiles", C.c_uint64),
                ("retried_tiles", C.c_uint64), ("pairs", C.c_uint64), ("eager_runs", C.c_uint32),
                ("graph_runs", C.c_uint32), ("launches_per_run", C.c_uint32), ("tuned", C.c_uint32),
                ("candidates", C.c_uint32), ("device_ms", C.c_double), ("plan_tile_width", C.c_uint32),
                ("plan_delta_mult", C.c_uint32), ("plan_tile_sources", C.c_uint32)]


class rn_edges(C.Structure):
    _fields_ = [("n", C.c_uint32), ("flags", C.c_uint32), ("m", C.c_uint64), ("src", C.POINTER(C.c_uint32)),
                ("dst", C.POINTER(C.c_uint32)), ("w", C.POINTER(C.c_uint32))]


class rn_point(C.Structure):
    _fields_ = [("a", C.c_uint32), ("b", C.c_uint32), ("t", C.c_uint32)]


class rn_request(C.Structure):
    _fields_ = [("R", C.POINTER(C.c_uint32)), ("nR", C.c_uint32), ("S", C.POINTER(C.c_uint32)),
                ("nS", C.c_uint32), ("theta", C.c_uint32), ("k", C.c_uint64)]


class rn_hier_stats(C.Structure):
    _fields_ = [("parts", C.c_uint64), ("max_part", C.c_uint64), ("local_pairs", C.c_uint64),
                ("border_routes", C.c_uint64), ("exit_routes", C.c_uint64), ("exit_searches", C.c_uint64),
                ("candidates", C.c_uint64), ("local_ms", C.c_double), ("exit_ms", C.c_double),
                ("combine_ms", C.c_double)]


class rn_serve_config(C.Structure):
    _fields_ = [("slab_bytes", C.c_uint64), ("workers", C.c_uint32), ("max_blocks", C.c_uint32)]


class rn_serve_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("pending", C.c_uint64), ("running", C.c_uint64), ("cancelled", C.c_uint64),
                ("groups", C.c_uint64), ("grouped", C.c_uint64), ("pairs", C.c_uint64),
                ("slab_bytes", C.c_uint64), ("slab_bytes_in_use", C.c_uint64),
                ("slab_bytes_peak", C.c_uint64), ("workers", C.c_uint32), ("max_running", C.c_uint32),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("max_ms", C.c_double),
                ("mean_ms", C.c_double), ("mean_queue_ms", C.c_double), ("busy_s", C.c_double),
                ("span_s", C.c_double)]


# Every symbol include/rn.h declares, with its ctypes signature (restype, argtypes).
_P32 = C.POINTER(C.c_uint32)
_G = C.c_void_p
SIGNATURES = {
    "rn_graph_load": (C.c_int, [_P32, _P32, _P32, C.c_uint64, C.c_uint32, C.c_uint32,
                                C.POINTER(C.c_float), C.POINTER(rn_config), C.POINTER(C.c_void_p)]),
    "rn_graph_free": (None, [_G]),
    "rn_bisection_order": (C.c_int, [_P32, _P32, _P32, C.c_uint64, C.c_uint32, C.c_uint32,
                                     C.POINTER(rn_config), _P32]),
    "rn_graph_info": (C.c_int, [_G, C.POINTER(rn_graph_stats)]),
    "rn_graph_permutation": (C.c_int, [_G, _P32]),
    "rn_graph_set_config": (C.c_int, [_G, C.POINTER(rn_config)]),
    "rn_distance_join": (C.c_int, [_G, _P32, C.c_uint32, _P32, C.c_uint32, C.c_uint32,
                                   C.POINTER(rn_pairs)]),
    "rn_distance_join_dev": (C.c_int, [_G, C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint32,
                                       C.c_uint32, C.POINTER(rn_dpairs), C.c_void_p]),
    "rn_distance_join_noalloc": (C.c_int, [_G, C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint32,
                                           C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_uint64, C.POINTER(C.c_uint64), C.c_void_p]),
    "rn_kcp": (C.c_int, [_G, _P32, C.c_uint32, _P32, C.c_uint32, C.c_uint64, C.c_uint32,
                         C.POINTER(rn_pairs)]),
    "rn_kcp_dev": (C.c_int, [_G, C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint32, C.c_uint64,
                             C.c_uint32, C.POINTER(rn_dpairs), C.c_void_p]),
    "rn_batch_create": (C.c_int, [C.POINTER(rn_query), C.c_uint32, C.POINTER(rn_batch_config),
                                  C.POINTER(C.c_void_p)]),
    "rn_batch_run": (C.c_int, [C.c_void_p, C.c_void_p]),
    "rn_batch_pairs": (C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(rn_pairs)]),
    "rn_batch_pairs_dev": (C.c_int, [C.c_void_p, C.c_uint32, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                     C.POINTER(C.c_void_p), C.POINTER(C.c_uint64)]),
    "rn_batch_stats_get": (C.c_int, [C.c_void_p, C.POINTER(rn_batch_stats)]),
    "rn_batch_free": (None, [C.c_void_p]),
    "rn_join_batch": (C.c_int, [C.POINTER(rn_query), C.c_uint32, C.POINTER(rn_pairs)]),
    "rn_serve_create": (C.c_int, [_G, C.POINTER(rn_serve_config), C.POINTER(C.c_void_p)]),
    "rn_serve_submit": (C.c_int, [C.c_void_p, C.POINTER(rn_request), C.POINTER(C.c_uint64)]),
    "rn_serve_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint32, C.POINTER(rn_pairs)]),
    "rn_serve_cancel": (C.c_int, [C.c_void_p, C.c_uint64]),
    "rn_serve_stats_get": (C.c_int, [C.c_void_p, C.POINTER(rn_serve_stats)]),
    "rn_serve_reset_stats": (C.c_int, [C.c_void_p]),
    "rn_serve_destroy": (None, [C.c_void_p]),
    "rn_distance_join_points": (C.c_int, [_G, C.POINTER(rn_point), C.c_uint32, C.POINTER(rn_point), C.c_uint32,
                                          C.c_uint32, C.POINTER(rn_pairs)]),
    "rn_kcp_points": (C.c_int, [_G, C.POINTER(rn_point), C.c_uint32, C.POINTER(rn_point), C.c_uint32, C.c_uint64,
                                C.c_uint32, C.POINTER(rn_pairs)]),
    "rn_distance_join_box": (C.c_int, [_G, _P32, C.c_uint32, _P32, C.c_uint32, C.c_uint32,
                                       C.POINTER(C.c_float), C.c_uint32, C.POINTER(rn_pairs)]),
    "rn_kcp_box": (C.c_int, [_G, _P32, C.c_uint32, _P32, C.c_uint32, C.c_uint64, C.c_uint32,
                             C.POINTER(C.c_float), C.c_uint32, C.POINTER(rn_pairs)]),
    "rn_file_read": (C.c_int, [C.c_char_p, C.POINTER(rn_edges)]),
    "rn_edges_free": (None, [C.POINTER(rn_edges)]),
    "rn_graph_load_file": (C.c_int, [C.c_char_p, C.POINTER(C.c_void_p)]),
    "rn_graph_write_file": (C.c_int, [C.c_char_p, _P32, _P32, _P32, C.c_uint64, C.c_uint32, C.c_uint32]),
    "rn_set_allocator": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "rn_tune_cache_save": (C.c_int, [C.c_char_p]),
    "rn_tune_cache_load": (C.c_int, [C.c_char_p, C.POINTER(C.c_uint32)]),
    "rn_join_many": (C.c_int, [_G, C.POINTER(rn_request), C.c_uint32, C.POINTER(rn_pairs)]),
    "rn_pairs_free": (None, [C.POINTER(rn_pairs)]),
    "rn_dpairs_free": (None, [C.POINTER(rn_dpairs)]),
    "rn_last_error": (C.c_char_p, []),
    "rn_last_query_stats": (C.c_int, [C.POINTER(rn_query_stats)]),
    "rn_distance_join_hier": (C.c_int, [_G, _P32, C.c_uint32, _P32, C.c_uint32, C.c_uint32, C.c_uint32,
                                        C.POINTER(rn_pairs)]),
    "rn_kcp_hier": (C.c_int, [_G, _P32, C.c_uint32, _P32, C.c_uint32, C.c_uint64, C.c_uint32, C.c_uint32,
                              C.POINTER(rn_pairs)]),
    "rn_last_hier_stats": (C.c_int, [C.POINTER(rn_hier_stats)]),
    "rn_version": (C.c_char_p, []),
}

_lib = None


def lib() -> C.CDLL:
    """The loaded engine library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_1607_07696_gb300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int) -> None:
    if status != RN_OK:
        raise RNError(status, lib().rn_last_error().decode())


def _u32(a) -> np.ndarray:
    a = np.asarray(a)
    if a.dtype == np.uint32:
        return np.ascontiguousarray(a)
    if a.size and (a.min() < 0 or a.max() > 0xFFFFFFFF):
        raise ValueError("ids and weights must fit in uint32")
    if a.dtype == np.int32 and a.flags.c_contiguous:
        return a.view(np.uint32)  # no copy: keeps pinned host memory pinned
    return np.ascontiguousarray(a, dtype=np.uint32)


def _p32(a: np.ndarray):
    return a.ctypes.data_as(_P32)


def _dev_ptr(t) -> int:
    """Device address of a CUDA tensor of 32-bit ints (int32 or uint32)."""
    if not t.is_cuda or t.element_size() != 4 or not t.is_contiguous():
        raise ValueError("device arrays must be contiguous 32-bit CUDA tensors")
    return t.data_ptr()


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    return int(getattr(stream, "cuda_stream", stream))


def _config(cfg: dict | None):
    if cfg is None:
        return None
    c = rn_config()
    c.tile_width = int(cfg.get("tile_width", 0))
    c.tile_sources = int(cfg.get("tile_sources", 0))
    c.delta = int(cfg.get("delta", 0))
    c.leaf_size = int(cfg.get("leaf_size", 0))
    c.alpha = float(cfg.get("alpha", -1.0))
    c.map_slots = int(cfg.get("map_slots", 0))
    c.search_from = int(cfg.get("search_from", 0))
    return C.byref(c)


class Graph:
    """Owner of an ``rn_graph*``; freed with the object."""

    def __init__(self, handle: int, n: int):
        self.handle = C.c_void_p(handle)
        self.n = n

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and h.value and _lib is not None:
            _lib.rn_graph_free(h)
            self.handle = None


def rn_graph_load(src, dst, w, n: int, flags: int = RN_UNDIRECTED | RN_REORDER,
                  cfg: dict | None = None, xy=None) -> Graph:
    """Load a graph; xy (optional, n x 2) gives node coordinates for rectangle queries."""
    s, d, ww = _u32(src), _u32(dst), _u32(w)
    if not (len(s) == len(d) == len(ww)):
        raise ValueError("edge arrays differ in length")
    pxy = None
    if xy is not None:
        xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float32).reshape(-1, 2))
        if len(xy) != int(n):
            raise ValueError("xy needs one (x, y) per node")
        pxy = xy.ctypes.data_as(C.POINTER(C.c_float))
    out = C.c_void_p()
    _check(lib().rn_graph_load(_p32(s), _p32(d), _p32(ww), len(s), int(n), int(flags), pxy,
                               _config(cfg), C.byref(out)))
    return Graph(out.value, int(n))


def rn_bisection_order(src, dst, w, n: int, flags: int = RN_UNDIRECTED,
                       cfg: dict | None = None) -> np.ndarray:
    """Host-only: order[i] = original id placed at internal id i by RN_REORDER."""
    s, d, ww = _u32(src), _u32(dst), _u32(w)
    order = np.zeros(int(n), np.uint32)
    _check(lib().rn_bisection_order(_p32(s), _p32(d), _p32(ww), len(s), int(n), int(flags),
                                    _config(cfg), _p32(order)))
    return order


def rn_graph_info(g: Graph) -> dict:
    st = rn_graph_stats()
    _check(lib().rn_graph_info(g.handle, C.byref(st)))
    return {f: getattr(st, f) for f, _ in rn_graph_stats._fields_}


def rn_graph_permutation(g: Graph) -> np.ndarray:
    p = np.zeros(g.n, np.uint32)
    _check(lib().rn_graph_permutation(g.handle, _p32(p)))
    return p


def rn_graph_set_config(g: Graph, cfg: dict | None) -> None:
    _check(lib().rn_graph_set_config(g.handle, _config(cfg)))


class _PairsOwner:
    """Holds library-owned result buffers (an ``rn_pairs``) until no array views them."""

    def __init__(self, p: rn_pairs):
        self.p = p

    def __del__(self):
        if _lib is not None and getattr(self, "p", None) is not None:
            _lib.rn_pairs_free(C.byref(self.p))
            self.p = None


class _View:
    """numpy array interface over one of the buffers, keeping their owner alive."""

    def __init__(self, owner: _PairsOwner, ptr, n: int):
        self.owner = owner
        self.__array_interface__ = {"shape": (n,), "typestr": "<u4", "version": 3,
                                    "data": (C.cast(ptr, C.c_void_p).value, False)}


def _take_pairs(p: rn_pairs):
    """(u, v, d) numpy views of the library's result buffers (no copy); the buffers are
    freed when the last of the three arrays is gone."""
    n = int(p.n)
    owner = _PairsOwner(p)
    if n == 0:
        z = np.zeros(0, np.uint32)
        return z, z.copy(), z.copy()
    return tuple(np.asarray(_View(owner, ptr, n)) for ptr in (p.u, p.v, p.d))


def rn_distance_join(g: Graph, R, S, theta: int):
    """Host arrays in, host arrays out: (u, v, d) sorted by (u, v)."""
    r, s = _u32(R), _u32(S)
    p = rn_pairs()
    _check(lib().rn_distance_join(g.handle, _p32(r), len(r), _p32(s), len(s), int(theta), C.byref(p)))
    return _take_pairs(p)


def rn_kcp(g: Graph, R, S, k: int, theta: int = RN_INF):
    """Host arrays in, host arrays out: (u, v, d) sorted by (d, u, v)."""
    r, s = _u32(R), _u32(S)
    p = rn_pairs()
    _check(lib().rn_kcp(g.handle, _p32(r), len(r), _p32(s), len(s), int(k), int(theta), C.byref(p)))
    return _take_pairs(p)


RN_BOX_R, RN_BOX_S = 1, 2


def _box(box):
    b = np.ascontiguousarray(np.asarray(box, dtype=np.float32).reshape(4))
    return b, b.ctypes.data_as(C.POINTER(C.c_float))


def rn_distance_join_box(g: Graph, R, S, theta: int, box, which: int = RN_BOX_R | RN_BOX_S):
    """The join of the members of R and S (as ``which`` says) whose node lies in the closed
    rectangle box = (xmin, ymin, xmax, ymax); (u, v, d) sorted by (u, v)."""
    r, s = _u32(R), _u32(S)
    b, pb = _box(box)
    p = rn_pairs()
    _check(lib().rn_distance_join_box(g.handle, _p32(r), len(r), _p32(s), len(s), int(theta), pb, int(which),
                                      C.byref(p)))
    return _take_pairs(p)


def rn_kcp_box(g: Graph, R, S, k: int, theta: int = RN_INF, box=(0, 0, 0, 0), which: int = RN_BOX_R | RN_BOX_S):
    """k closest pairs of the members of R and S in the rectangle; sorted by (d, u, v)."""
    r, s = _u32(R), _u32(S)
    b, pb = _box(box)
    p = rn_pairs()
    _check(lib().rn_kcp_box(g.handle, _p32(r), len(r), _p32(s), len(s), int(k), int(theta), pb, int(which),
                            C.byref(p)))
    return _take_pairs(p)


class DevicePairs:
    """Library-owned device result buffers (an ``rn_dpairs``), reusable across calls."""

    def __init__(self):
        self.s = rn_dpairs()

    def __del__(self):
        if _lib is not None and getattr(self, "s", None) is not None:
            _lib.rn_dpairs_free(C.byref(self.s))

    @property
    def n(self) -> int:
        return int(self.s.n)

    def tensors(self):
        """(u, v, d) as int32 torch views of the device buffers (valid until the next call)."""
        import torch

        n = self.n

        class _View:
            def __init__(self, ptr):
                self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i4",
                                                 "data": (int(ptr or 0), False), "version": 3}

        if n == 0:
            z = torch.zeros(0, dtype=torch.int32, device="cuda")
            return z, z.clone(), z.clone()
        return tuple(torch.as_tensor(_View(p), device="cuda") for p in (self.s.u, self.s.v, self.s.d))

    def numpy(self):
        return tuple(t.cpu().numpy().view(np.uint32) for t in self.tensors())


def rn_distance_join_dev(g: Graph, dR, dS, theta: int, out: DevicePairs, stream=None) -> int:
    """Device tensors in, library-owned device buffers out; returns the pair count."""
    _check(lib().rn_distance_join_dev(g.handle, _dev_ptr(dR), dR.numel(), _dev_ptr(dS), dS.numel(),
                                      int(theta), C.byref(out.s), _stream_ptr(stream)))
    return out.n


def rn_distance_join_noalloc(g: Graph, dR, dS, theta: int, out_u, out_v, out_d, stream=None) -> int:
    """The join into caller-owned device tensors (out_u/out_v/out_d, equal lengths), with no
    allocation by the library; returns the pair count."""
    n = C.c_uint64(0)
    cap = out_u.numel()
    if out_v.numel() != cap or out_d.numel() != cap:
        raise ValueError("output tensors differ in length")
    _check(lib().rn_distance_join_noalloc(g.handle, _dev_ptr(dR), dR.numel(), _dev_ptr(dS), dS.numel(),
                                          int(theta), _dev_ptr(out_u), _dev_ptr(out_v), _dev_ptr(out_d),
                                          cap, C.byref(n), _stream_ptr(stream)))
    return int(n.value)


def rn_kcp_dev(g: Graph, dR, dS, k: int, theta: int, out: DevicePairs, stream=None) -> int:
    _check(lib().rn_kcp_dev(g.handle, _dev_ptr(dR), dR.numel(), _dev_ptr(dS), dS.numel(), int(k),
                            int(theta), C.byref(out.s), _stream_ptr(stream)))
    return out.n


def rn_last_query_stats() -> dict:
    st = rn_query_stats()
    _check(lib().rn_last_query_stats(C.byref(st)))
    return {f: getattr(st, f) for f, _ in rn_query_stats._fields_}


def rn_distance_join_hier(g: Graph, R, S, theta: int, part_size: int = 0):
    """The join by the hierarchical variant (parts of the partition hierarchy of at most
    part_size nodes; 0: its leaves): the same (u, v, d), sorted by (u, v)."""
    r, s = _u32(R), _u32(S)
    p = rn_pairs()
    _check(lib().rn_distance_join_hier(g.handle, _p32(r), len(r), _p32(s), len(s), int(theta), int(part_size),
                                       C.byref(p)))
    return _take_pairs(p)


def rn_kcp_hier(g: Graph, R, S, k: int, theta: int = RN_INF, part_size: int = 0):
    """k closest pairs by the hierarchical variant; sorted by (d, u, v)."""
    r, s = _u32(R), _u32(S)
    p = rn_pairs()
    _check(lib().rn_kcp_hier(g.handle, _p32(r), len(r), _p32(s), len(s), int(k), int(theta), int(part_size),
                             C.byref(p)))
    return _take_pairs(p)


def rn_last_hier_stats() -> dict:
    st = rn_hier_stats()
    _check(lib().rn_last_hier_stats(C.byref(st)))
    return {f: getattr(st, f) for f, _ in rn_hier_stats._fields_}


def rn_version() -> str:
    return lib().rn_version().decode()


def _queries(queries):
    """queries: (Graph, R, S, theta) tuples -> (ctypes array, arrays kept alive)."""
    keep = []
    arr = (rn_query * len(queries))()
    for i, (g, R, S, theta) in enumerate(queries):
        r, s_ = _u32(R), _u32(S)
        keep += [r, s_]
        arr[i].g = g.handle
        arr[i].R = _p32(r)
        arr[i].nR = len(r)
        arr[i].S = _p32(s_)
        arr[i].nS = len(s_)
        arr[i].theta = int(theta)
    return arr, keep


class Batch:
    """Owner of an ``rn_batch*`` (a prepared batch of theta-joins)."""

    def __init__(self, handle: int):
        self.handle = C.c_void_p(handle)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and h.value and _lib is not None:
            _lib.rn_batch_free(h)
            self.handle = None


def rn_batch_create(queries, autotune: bool = False, use_graph: bool = True) -> Batch:
    arr, _keep = _queries(queries)
    cfg = rn_batch_config(int(bool(autotune)), int(bool(use_graph)))
    out = C.c_void_p()
    _check(lib().rn_batch_create(arr, len(queries), C.byref(cfg), C.byref(out)))
    return Batch(out.value)


def rn_batch_run(b: Batch, stream=None) -> None:
    _check(lib().rn_batch_run(b.handle, _stream_ptr(stream)))


def rn_batch_pairs(b: Batch, i: int):
    p = rn_pairs()
    _check(lib().rn_batch_pairs(b.handle, int(i), C.byref(p)))
    return _take_pairs(p)


def rn_batch_pairs_dev(b: Batch, i: int):
    """(u, v, d) device addresses and the count of instance i's pairs (owned by the batch)."""
    u, v, d, n = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_uint64()
    _check(lib().rn_batch_pairs_dev(b.handle, int(i), C.byref(u), C.byref(v), C.byref(d), C.byref(n)))
    return u.value, v.value, d.value, int(n.value)


def rn_batch_stats_get(b: Batch) -> dict:
    st = rn_batch_stats()
    _check(lib().rn_batch_stats_get(b.handle, C.byref(st)))
    return {f: getattr(st, f) for f, _ in rn_batch_stats._fields_}


def rn_join_batch(queries):
    """One call: every query's (u, v, d) host arrays, in query order."""
    arr, _keep = _queries(queries)
    outs = (rn_pairs * len(queries))()
    _check(lib().rn_join_batch(arr, len(queries), outs))
    return [_take_pairs(outs[i]) for i in range(len(queries))]


# ------------------------------------------------------------------ serving ----

WAIT_FOREVER = 0xFFFFFFFF


class Server:
    """Owner of an ``rn_server*`` over one graph (kept alive as long as the server)."""

    def __init__(self, handle: int, graph: Graph):
        self.handle = C.c_void_p(handle)
        self.graph = graph

    def close(self) -> None:
        h = getattr(self, "handle", None)
        if h and h.value and _lib is not None:
            _lib.rn_serve_destroy(h)
        self.handle = None

    def __del__(self):
        self.close()


def rn_serve_create(g: Graph, slab_bytes: int = 0, workers: int = 0, max_blocks: int = 0) -> Server:
    cfg = rn_serve_config(int(slab_bytes), int(workers), int(max_blocks))
    out = C.c_void_p()
    _check(lib().rn_serve_create(g.handle, C.byref(cfg), C.byref(out)))
    return Server(out.value, g)


def rn_serve_submit(srv: Server, R, S, theta: int = RN_INF, k: int = 0) -> int:
    """Queue a theta-join (k = 0) or a k-closest-pairs request; returns its ticket."""
    r, s = _u32(R), _u32(S)
    q = rn_request(_p32(r), len(r), _p32(s), len(s), int(theta), int(k))
    t = C.c_uint64()
    _check(lib().rn_serve_submit(srv.handle, C.byref(q), C.byref(t)))
    return int(t.value)


def rn_serve_wait(srv: Server, ticket: int, timeout_ms: int = WAIT_FOREVER):
    """The request's (u, v, d) once done (the GIL is released while waiting)."""
    p = rn_pairs()
    _check(lib().rn_serve_wait(srv.handle, int(ticket), int(timeout_ms), C.byref(p)))
    return _take_pairs(p)


def rn_serve_cancel(srv: Server, ticket: int) -> None:
    _check(lib().rn_serve_cancel(srv.handle, int(ticket)))


def rn_serve_stats_get(srv: Server) -> dict:
    st = rn_serve_stats()
    _check(lib().rn_serve_stats_get(srv.handle, C.byref(st)))
    return {name: getattr(st, name) for name, _ in rn_serve_stats._fields_}


def rn_serve_reset_stats(srv: Server) -> None:
    _check(lib().rn_serve_reset_stats(srv.handle))


# ------------------------------------------------------------- points on edges ----

def _points(P) -> np.ndarray:
    a = np.asarray(P, dtype=np.int64).reshape(-1, 3)
    if a.size and (a.min() < 0 or a.max() > 0xFFFFFFFF):
        raise ValueError("point fields must fit in uint32")
    return np.ascontiguousarray(a.astype(np.uint32))


def _pp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(rn_point))


def rn_distance_join_points(g: Graph, R, S, theta: int):
    """Points as (count, 3) arrays of (a, b, t): the point on edge {a, b} at distance t
    from a.  Returns (u, v, d) with u, v indices into R and S, sorted by (u, v)."""
    r, s = _points(R), _points(S)
    p = rn_pairs()
    _check(lib().rn_distance_join_points(g.handle, _pp(r), len(r), _pp(s), len(s), int(theta), C.byref(p)))
    return _take_pairs(p)


def rn_kcp_points(g: Graph, R, S, k: int, theta: int = RN_INF):
    """k closest pairs of points, sorted by (d, u, v); u, v index R and S."""
    r, s = _points(R), _points(S)
    p = rn_pairs()
    _check(lib().rn_kcp_points(g.handle, _pp(r), len(r), _pp(s), len(s), int(k), int(theta), C.byref(p)))
    return _take_pairs(p)


# ------------------------------------------------------------------ graph files ----

def rn_file_read(path: str):
    """(n, flags, src, dst, w) of a .rng or DIMACS .gr file (host arrays, copied)."""
    e = rn_edges()
    _check(lib().rn_file_read(os.fsencode(path), C.byref(e)))
    try:
        m = int(e.m)
        arrs = [np.ctypeslib.as_array(p, shape=(max(m, 1),))[:m].copy() for p in (e.src, e.dst, e.w)]
        return int(e.n), int(e.flags), arrs[0], arrs[1], arrs[2]
    finally:
        lib().rn_edges_free(C.byref(e))


def rn_graph_load_file(path: str) -> Graph:
    out = C.c_void_p()
    _check(lib().rn_graph_load_file(os.fsencode(path), C.byref(out)))
    g = Graph(out.value, 0)
    g.n = int(rn_graph_info(g)["n"])
    return g


def rn_graph_write_file(path: str, src, dst, w, n: int, flags: int = RN_UNDIRECTED | RN_REORDER) -> None:
    s, d, ww = _u32(src), _u32(dst), _u32(w)
    if not (len(s) == len(d) == len(ww)):
        raise ValueError("edge arrays differ in length")
    _check(lib().rn_graph_write_file(os.fsencode(path), _p32(s), _p32(d), _p32(ww), len(s), int(n), int(flags)))


# ------------------------------------------------------------- allocator hook ----

_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
_torch_hooks = []  # every hook made: blocks made through one still call it when freed
_torch_hook_open = True


def use_torch_allocator(enable: bool = True) -> None:
    """Take the engine's device memory from torch's caching allocator (enable=True) or
    from cudaMalloc again (False).  Blocks already made keep going back to the allocator
    that made them."""
    import atexit

    import torch

    if not enable:
        _check(lib().rn_set_allocator(None, None, None))
        return

    def alloc(nbytes, ctx):
        try:
            dev = torch.cuda.current_device()
            stream = torch.cuda.default_stream(dev)
            p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
            stream.synchronize()  # the block may have been in use on that stream until now
            return p
        except Exception:  # noqa: BLE001 - reported to the engine as no memory
            return None

    def free(ptr, ctx):
        if _torch_hook_open:
            torch.cuda.caching_allocator_delete(int(ptr))

    if not _torch_hooks:
        def _close():
            global _torch_hook_open
            _torch_hook_open = False  # no calls into torch while the interpreter exits

        atexit.register(_close)
    hook = (_ALLOC_FN(alloc), _FREE_FN(free))
    _torch_hooks.append(hook)
    _check(lib().rn_set_allocator(C.cast(hook[0], C.c_void_p), C.cast(hook[1], C.c_void_p), None))


def rn_tune_cache_save(path: str) -> None:
    _check(lib().rn_tune_cache_save(os.fsencode(path)))


def rn_tune_cache_load(path: str) -> int:
    n = C.c_uint32()
    _check(lib().rn_tune_cache_load(os.fsencode(path), C.byref(n)))
    return int(n.value)


def rn_join_many(g: Graph, queries):
    """Several theta-joins [(R, S, theta), ...] over one graph, searched together; a list
    of (u, v, d), one per query, each sorted by (u, v)."""
    arrs = [(_u32(R), _u32(S), int(theta)) for (R, S, theta) in queries]
    reqs = (rn_request * max(1, len(arrs)))()
    for i, (r, s, th) in enumerate(arrs):
        reqs[i] = rn_request(_p32(r), len(r), _p32(s), len(s), th, 0)
    outs = (rn_pairs * max(1, len(arrs)))()
    _check(lib().rn_join_many(g.handle, reqs, len(arrs), outs))
    return [_take_pairs(outs[i]) for i in range(len(arrs))]
