"""Host-side helpers of bench.py: the roofline arithmetic and the recorded DRAM
traffic, which is reported only for the kernel code it was captured with."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_code_lines_drop_comments_and_blank_lines():
    text = "int a = 1;  // one\n\n   // only a comment\nint b = 2;\n"
    assert list(bench.code_lines(text)) == ["int a = 1;", "int b = 2;"]


def _read_current(f):
    with open(os.path.join(ROOT, "paper_2304_11002_gb300", "csrc", f)) as fh:
        return fh.read()


def test_recorded_traffic_is_reported_only_for_the_code_it_was_captured_with():
    with open(bench.TRAFFIC_FILE) as f:
        entry = json.load(f)["entries"][0]
    nbytes, source = bench.recorded_traffic(entry["stage"], entry["workload"])
    if entry["sources_sha256"] == bench.kernel_sources_sha256():
        assert nbytes == entry["dram_bytes_read"] + entry["dram_bytes_write"], source
        assert "ncu" in source
    else:
        assert nbytes is None and source == "kernel changed since the capture"


def test_comment_edits_keep_and_code_edits_drop_the_capture():
    base = bench.kernel_sources_sha256()
    commented = bench.kernel_sources_sha256(lambda f: _read_current(f) + "\n// a note\n")
    changed = bench.kernel_sources_sha256(lambda f: _read_current(f) + "\nint extra;\n")
    assert commented == base
    assert changed != base


def test_roofline_of_picks_the_binding_pipe_of_the_longest_stage():
    info = [
        {"name": "tree", "flops": 0, "flops64": 0, "bytes": 6.8e12},
        # 1e12 float64 flops and 4e12 float32 flops in 2 s
        {"name": "mixed", "flops": 5e12, "flops64": 1e12, "bytes": 0},
    ]
    r = bench.roofline_of(info, [1000.0, 2000.0], {"hbm_gbs": 6800.0})
    # float64 work at its peak takes longer than the float32 work at its own
    assert r["kernel"] == "mixed" and r["bound"] == "alu" and r["pipe"] == "fp64"
    assert r["achieved"] == pytest.approx(0.5)
    assert r["frac"] == pytest.approx(0.5 / bench.PEAK_FP64_TFLOPS)
    assert r["other_pipe_frac"] == pytest.approx(2.0 / bench.PEAK_FP32_TFLOPS)
    h = bench.roofline_of(info, [3000.0, 2000.0], {"hbm_gbs": 6800.0})
    assert h["bound"] == "hbm" and h["achieved"] == pytest.approx(6800.0 / 3.0)
    assert h["frac"] == pytest.approx(1.0 / 3.0)
