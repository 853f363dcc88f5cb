"""The C ABI library: it builds, loads, exports every symbol include/rn.h declares, and
rejects bad arguments on the host before touching a GPU (no GPU needed)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rn():
    from paper_1607_07696_gb300 import build as B

    B.build()
    from paper_1607_07696_gb300 import rn as RN

    RN.lib()
    return RN


def declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(rn_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("rn_graph_load", "rn_distance_join", "rn_distance_join_dev", "rn_kcp", "rn_kcp_dev",
                 "rn_last_error", "rn_pairs_free", "rn_graph_free"):
        assert must in names


def test_every_declared_symbol_is_exported(rn):
    import ctypes

    L = ctypes.CDLL(rn.LIB_PATH)
    for name in declared_functions():
        assert hasattr(L, name), f"{name} declared in include/ but not exported"
        assert name in rn.SIGNATURES, f"{name} has no binding signature"


def test_version(rn):
    assert "sm_103a" in rn.rn_version()


def test_graph_load_rejects_bad_input_on_host(rn):
    with pytest.raises(rn.RNError) as e:
        rn.rn_graph_load([0], [5], [1], n=3)
    assert e.value.status == rn.RN_EINVAL
    with pytest.raises(rn.RNError) as e:
        rn.rn_graph_load([0], [1], [0], n=3)
    assert e.value.status == rn.RN_EINVAL
    with pytest.raises(rn.RNError) as e:
        rn.rn_graph_load([0], [1], [1 << 24], n=3)
    assert e.value.status == rn.RN_EINVAL
    with pytest.raises(rn.RNError) as e:
        rn.rn_graph_load([0], [1], [1], n=3, flags=0x80)
    assert e.value.status == rn.RN_EINVAL
    with pytest.raises(rn.RNError) as e:
        rn.rn_graph_load([], [], [], n=0)
    assert e.value.status == rn.RN_EINVAL
    assert "n" in rn.lib().rn_last_error().decode()


def test_no_stats_before_a_query(rn):
    import threading

    out = {}

    def probe():
        try:
            rn.rn_last_query_stats()
        except rn.RNError as e:
            out["status"] = e.status

    t = threading.Thread(target=probe)
    t.start()
    t.join()
    assert out["status"] == rn.RN_EINVAL


def test_library_has_no_cpu_fallback_symbols(rn):
    # the product library must not link the oracle
    import subprocess

    syms = subprocess.run(["nm", "-D", rn.LIB_PATH], capture_output=True, text=True).stdout
    assert "og_" not in syms
