"""The stencil tables of the interaction kernels (csrc/tables.cpp) and the leaf halo
geometry (csrc/halo.h), checked on the host: tests/tables_check.cpp is compiled
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
