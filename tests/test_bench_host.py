"""The benchmark's host side, without a GPU: the committed ncu summaries match the kernel
source they describe, the roofline arithmetic, and the CPU reference arm's JSON line."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bench():
    sys.path.insert(0, ROOT)
    import bench as B

    return B


def test_committed_profiles_describe_the_current_warp_search():
    B = bench()
    paths = set(B.PROFILES.values())
    assert paths, "no profile registered"
    for path in paths:
        assert os.path.exists(path), path
        p = json.load(open(path))
        assert p["workload"] in B.PROFILES and B.PROFILES[p["workload"]] == path
        assert p["engine_sha"] == B.engine_hash(), f"{path}: captured on another version of the warp search"
        assert p["kernel"].startswith("k_source_search")
        assert "ncu" in p["command"] and "--clock-control none" in p["command"]
        assert p["dram_bytes_per_launch"] > 0 and p["l2_bytes_per_launch"] > p["dram_bytes_per_launch"]
        md = path[:-5] + ".md"
        assert os.path.exists(md), md


def test_roofline_arithmetic():
    B = bench()
    st = {"slots": 1000, "slot_arcs": 5000, "slot_lanes": 1000, "tile_width": 1}
    alg = B.algorithmic_bytes(st, 200)
    assert alg == 8 * 1000 + 8 * 5000 + 8 * 1000 + 1000 / 8 + 12 * 200
    r = B.roofline(st, 200, 0.5, "no_such_workload", 1000.0, "measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["kernel"] == "k_source_search"
    assert abs(r["achieved"] - alg / 0.5e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 1000.0) < 1e-12
    assert r["traffic"] is None and "l2" not in r
    # with the committed profile of the headline workload: its traffic and L2 figures
    prof = B.profile_of("road1070k_join", "k_source_search")
    assert prof is not None
    r = B.roofline(st, 200, 0.5, "road1070k_join", 1000.0, "measured")
    assert r["traffic"] == prof["dram_bytes_per_launch"] and r["l2"]["bytes_per_launch"] == prof["l2_bytes_per_launch"]


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "grid4096_theta1500", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["config"]["workload"] == "grid4096_theta1500"
