"""Host-side logic of bench.py (CPU only): the source hash that ties a committed DRAM-traffic
figure to the kernel it was measured on, and the lookup of that figure."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_only_ignores_comments_and_whitespace():
    a = "int f(int x) {\n    // twice x\n    return 2 * x; /* fast */\n}\n"
    b = "int f(int x) { /* a longer\n comment */ return 2 *   x;\n}"
    c = "int f(int x) {\n    return 3 * x;\n}\n"
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only(a) != bench.code_only(c)


def test_traffic_lookup_follows_the_kernel_hash(tmp_path, monkeypatch):
    src = tmp_path / "k.cuh"
    src.write_text("__global__ void k() {}  // v1\n")
    monkeypatch.setattr(bench, "KERNEL_SRCS", [str(src)])
    table = tmp_path / "traffic.json"
    table.write_text(json.dumps({"stage_kernel|w|fp32": {"bytes_per_launch": 123.0,
                                                          "kernel_sha256": bench.kernel_sha()}}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(table))
    assert bench.traffic_for("stage_kernel|w|fp32") == 123.0
    src.write_text("__global__ void k() {}  // v2: comment only\n")
    assert bench.traffic_for("stage_kernel|w|fp32") == 123.0
    src.write_text("__global__ void k() { int a = 1; }\n")
    assert bench.traffic_for("stage_kernel|w|fp32") is None
    assert bench.traffic_for("stage_kernel|other|fp32") is None



def test_stage_roofline_matches_the_headline_bytes():
    # the 256^2 degree-3 shear layer: 5 fields x 65,536 cells x 16 modes
    nvals, ncell = 5 * 65536 * 16, 65536
    r = bench.stage_roofline(nvals, ncell, True, stage_ms=0.4, peak_gbs=6786.2)
    assert r["algorithmic_bytes_per_launch"] == 88604672.0  # the figure the benchmark line reports
    assert abs(r["achieved"] - 5 * 88604672.0 / 0.4e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 6786.2) < 1e-15 and r["avg_launch_ms"] == 0.08
    assert sum(bench.stage_bytes_per_value(True)) == 84 and sum(bench.stage_bytes_per_value(False)) == 136


def test_working_set_and_l2_flag():
    nvals = 5 * 65536 * 16
    assert bench.step_working_set_bytes(nvals, True) == 36 * nvals  # 189 MB: above the 129 MB L2
    assert bench.step_working_set_bytes(nvals, False) == 40 * nvals  # u^n, u^{n+1}, three deltas
    if bench.l2_bytes(0) is None:  # no device here
        assert bench.l2_resident(1, 0) is None
    else:
        assert bench.l2_resident(1, 0) is True
