"""The stencil tables of the interaction kernels (csrc/tables.cpp), the leaf halo
geometry (csrc/halo.h) and the float32 record layout (device.cuh), checked on the
host.  tests/tables_check.cpp is compiled
with the host compiler against the library's table builders and run.  It derives
the parity stencils from the opening criterion itself and checks that the x-pair
tables of the paired float32 items, the per-cell boundary pair lists and the leaf
far-field chunk blocks each reproduce their stencil exactly once, and that the
halo pitches give the bank-conflict-free lane patterns the kernels rely on."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2304_11002_gb300", "csrc")


def test_tables_and_halo_geometry(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "tables_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, os.path.join(ROOT, "tests", "tables_check.cpp"),
                    os.path.join(CSRC, "tables.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
    # theta = 0.5: the 1197-entry parity stencil in 617 x-pairs (37 with one cell)
    assert "theta 0.50: 1197 entries, 617 pairs" in r.stdout


def test_float32_record_layout(tmp_path):
    """The x-pair record layout of the mixed far field (device.cuh, compiled as host
    code): a bijection per node, both cells of a pair in one 16-byte word per field
    pair, and a parity-class warp's 32 lanes on 32 consecutive words."""
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "layout_check")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-x", "cu", "-I", CSRC, os.path.join(ROOT, "tests", "layout_check.cu"),
                    "-o", exe], check=True, capture_output=True, timeout=300)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
