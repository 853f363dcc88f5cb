"""Build the engine's shared library ``librn.so`` in-tree with nvcc for sm_103a.

Usage: ``python -m paper_1607_07696_gb300.build`` (or ``__graft_entry__.build()``).
Translation units compile in parallel into ``_build/``; the link step makes
``paper_1607_07696_gb300/librn.so`` with the CUDA runtime linked statically, so the
library needs nothing from the environment but the driver.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "librn.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
SOURCES = ["rn_engine.cu", "rn_graph.cpp", "rn_api.cpp", "rn_serve.cpp", "rn_file.cpp"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the engine needs the CUDA toolkit to build")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _headers() -> list[str]:
    hs = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    hs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    return hs


CHECKS_LIB = os.path.join(PKG, "librn_checks.so")


def build(verbose: bool = False, force: bool = False, checks: bool = False) -> str:
    """Compile every translation unit that changed and link librn.so; returns its path.
    checks=True builds librn_checks.so instead: the same engine with device bounds
    checks compiled in (-DRN_CHECKS; a failed check is reported as RN_EINTERNAL)."""
    out_dir = os.path.join(BUILD, "checks") if checks else BUILD
    lib_path = CHECKS_LIB if checks else LIB
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    headers = _headers()
    jobs = []
    objs = []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(out_dir, src + ".o")
        objs.append(obj)
        if force or _stale(obj, [path, *headers]):
            extra = ["-Xptxas", "-v"] if (verbose and src.endswith(".cu")) else []
            defs = ["-DRN_CHECKS"] if checks else []
            jobs.append([cc, *ARCH, *COMMON, *defs, *extra, "-c", path, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for out in ex.map(run, jobs):
            if verbose and out:
                print(out, file=sys.stderr)
    if force or jobs or _stale(lib_path, objs):
        tmp = lib_path + f".tmp{os.getpid()}"
        run([cc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"])
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
