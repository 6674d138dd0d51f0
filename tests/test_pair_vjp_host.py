"""The adjoint's per-pair reverse mode (m2l_pair_vjp, the core of the M2L
transpose) checked on the host, with no GPU: compiled as a host program and
compared, for every input of the four target/source variants, with central
differences of the forward pair expression evaluated in long double.  With a step
of 1e-6 the truncation error of the differences is about 1e-10 relative, so a
dropped or mis-signed term of the reverse sweep shows up far above the bound."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2304_11002_gb300", "csrc")


def test_pair_vjp_matches_finite_differences(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "pair_vjp_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-x", "cu", "-diag-suppress", "20208", "-I", CSRC,
                    os.path.join(HERE, "pair_vjp_check.cu"), "-o", exe],
                   check=True, capture_output=True, timeout=300)
    r = subprocess.run([exe, "1e-8"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
