"""Oracle parity on the full-size trees of the throughput sweep, the 128^3
differentiation case and the rotating stars, in both precisions.

Every cell is computed on the GPU (the launch configuration the benchmark times:
autotuned strategy, graph replay); a seeded sample of 192 leaf cells is computed by
the oracle once per tree and compared with both the float64 path (relative
tolerance 1e-12) and the mixed path (1e-6).  Norms: phi per cell, g as
max|dg| / max|g| over the sample.  All outputs must be finite.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2304_11002_gb300 import binding
from paper_2304_11002_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL_MIXED = 1e-12, 1e-6
N_SAMPLE = 192

# Host memory of one sampled oracle run, per cell of the tree (all nodes): the
# multipoles in full tensors (40 doubles), the local expansions (43 doubles), the
# near-field sums (4 doubles) and the selection flags, with 10 % margin.
ORACLE_BYTES_PER_CELL = int(1.1 * (8 * (40 + 43 + 4) + 1))


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_11002_gb300 import build
    build.build()


def host_memory_available() -> int:
    """Bytes this process may still allocate: MemAvailable, capped by the cgroup
    limit when there is one."""
    avail = None
    with open("/proc/meminfo") as f:
        for line in f:
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    for path, used_path in (("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory.current"),
                            ("/sys/fs/cgroup/memory/memory.limit_in_bytes",
                             "/sys/fs/cgroup/memory/memory.usage_in_bytes")):
        try:
            lim = open(path).read().strip()
            if lim != "max" and int(lim) < (1 << 60):
                cap = int(lim) - int(open(used_path).read().strip())
                avail = cap if avail is None else min(avail, cap)
            break
        except (OSError, ValueError):
            continue
    return avail or 0


CONFIGS = {
    # throughput sweep: ~1e3 leaf subgrids at q = 0.7 for seeds 0-2, ~1e4 and ~5e4
    "sweep1000_q0.7_s0": lambda: W.sweep(1000, q=0.7, seed=0),
    "sweep1000_q0.7_s1": lambda: W.sweep(1000, q=0.7, seed=1),
    "sweep1000_q0.7_s2": lambda: W.sweep(1000, q=0.7, seed=2),
    "sweep10000_q0.7_s0": lambda: W.sweep(10000, q=0.7, seed=0),
    "sweep50000_q0.7_s0": lambda: W.sweep(50000, q=0.7, seed=0),
    # the 128^3 uniform binary of the differentiation config, forward solve
    "binary128": W.binary128,
    # the rotating star at the paper's level-6 and level-7 tree sizes
    "star6": lambda: W.star(6),
    "star7": lambda: W.star(7),
}


def _gpu(w, precision):
    fmm = binding.OctoFMM(w.tree, w.theta, precision)
    r = torch.from_numpy(np.ascontiguousarray(w.rho.reshape(-1))).cuda()
    phi, g = fmm.forces(r)
    phi2, g2 = fmm.forces(r)  # graph replay after autotuning
    torch.cuda.synchronize()
    binding.octo_fmm_stats(fmm.handle)  # raises on a pending device-side error
    out = phi2.cpu().numpy(), g2.cpu().numpy()
    del fmm, r, phi, g, phi2, g2
    torch.cuda.empty_cache()
    return out


@pytest.mark.parametrize("name", sorted(CONFIGS))
def test_config_both_precisions_against_oracle(name):
    w = CONFIGS[name]()
    n_cells = w.tree.n_nodes * 512
    need = ORACLE_BYTES_PER_CELL * n_cells
    avail = host_memory_available()
    if need > 0.8 * avail:
        pytest.skip(f"{name}: the oracle needs ~{need / 2**30:.0f} GiB of host memory, "
                    f"{avail / 2**30:.0f} GiB available")
    nl = w.tree.n_leaf * 512
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(nl, size=N_SAMPLE, replace=False))
    mask = np.zeros(nl, np.uint8)
    mask[idx] = 1
    po, go, _ = oracle.fmm(w.tree, w.rho, w.theta, leaf_mask=mask)
    po, go = po[idx], go[:, idx]
    gmax = np.max(np.linalg.norm(go, axis=0))
    report = []
    for precision, tol in ((binding.OCTO_FP64, TOL64), (binding.OCTO_MIXED, TOL_MIXED)):
        phi, g = _gpu(w, precision)
        assert np.all(np.isfinite(phi)) and np.all(np.isfinite(g))
        ephi = float(np.max(np.abs(phi[idx] - po) / np.abs(po)))
        eg = float(np.max(np.linalg.norm(g[:, idx] - go, axis=0)) / gmax)
        report.append((precision, ephi, eg))
        assert ephi <= tol and eg <= tol, (name, precision, ephi, eg)
    print(f"{name}: leaf subgrids {w.tree.n_leaf}, " +
          ", ".join(f"{'fp64' if p == 0 else 'mixed'} phi {a:.2e} g {b:.2e}" for p, a, b in report))
