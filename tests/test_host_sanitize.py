"""The host C++ (CSR builder, recursive bisection, relabelling, graph files) under the
address and undefined-behaviour sanitizers, driven by tests/sanitize/host_driver.cpp."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1607_07696_gb300", "csrc")


def cuda_include():
    for d in ("/usr/local/cuda/include", os.path.join(os.environ.get("CUDA_HOME", ""), "include")):
        if os.path.exists(os.path.join(d, "nvtx3", "nvToolsExt.h")):
            return d
    return None


def test_host_code_under_sanitizers(tmp_path):
    cxx = shutil.which("g++")
    inc = cuda_include()
    if not cxx or not inc:
        pytest.skip("g++ or the CUDA headers are missing")
    exe = str(tmp_path / "host_driver")
    cmd = [cxx, "-std=c++17", "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=all", "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", inc,
           os.path.join(ROOT, "tests", "sanitize", "host_driver.cpp"), os.path.join(CSRC, "rn_graph.cpp"),
           os.path.join(CSRC, "rn_file.cpp"), "-o", exe, "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([exe, str(tmp_path)], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, (r.stdout + r.stderr)[-4000:]
    assert "0 failures" in r.stdout
