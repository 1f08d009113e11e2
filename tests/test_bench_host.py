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

