"""Mixed-precision path (float32 far field with compensated sums, float64 near
field, correction accumulation and tree passes) against the float64 oracle:
relative error at most 1e-6 on phi (per cell) and on g (max-normalised)."""
import numpy as np
import pytest

import oracle
from paper_2304_11002_gb300 import binding
from paper_2304_11002_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-6


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_11002_gb300 import build
    build.build()


def _solve(tree, rho, precision):
    fmm = binding.OctoFMM(tree, 0.5, precision)
    r = torch.from_numpy(np.ascontiguousarray(rho.reshape(-1))).cuda()
    phi, g = fmm.forces(r)
    torch.cuda.synchronize()
    return phi.cpu().numpy(), g.cpu().numpy()


def _errs(phi, g, po, go, idx=None):
    if idx is not None:
        phi, g, po, go = phi[idx], g[:, idx], po[idx], go[:, idx]
    ephi = float(np.max(np.abs(phi - po) / np.abs(po)))
    eg = float(np.max(np.linalg.norm(g - go, axis=0)) / np.max(np.linalg.norm(go, axis=0)))
    return ephi, eg


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mixed_uniform16_full(seed):
    w = W.uniform16(seed)
    phi, g = _solve(w.tree, w.rho, binding.OCTO_MIXED)
    po, go, _ = oracle.fmm(w.tree, w.rho)
    ephi, eg = _errs(phi, g, po, go)
    assert ephi <= TOL_MIXED and eg <= TOL_MIXED, (ephi, eg)


def _workload(name):
    """name or (sweep target, q, seed) of the throughput-sweep trees."""
    if name == "adaptive4":
        return W.adaptive_binary(3, 0.08)
    if isinstance(name, tuple):
        return W.sweep(name[0], q=name[1], seed=name[2])
    return W.make(name)


@pytest.mark.parametrize("name", ["adaptive4", "binary64", "adaptive7", (1000, 0.3, 1), (1000, 1.0, 2),
                                  (10000, 0.7, 0), "star5"])
def test_mixed_sampled(name):
    w = _workload(name)
    phi, g = _solve(w.tree, w.rho, binding.OCTO_MIXED)
    n = w.tree.n_leaf * 512
    rng = np.random.default_rng(6)
    idx = np.sort(rng.choice(n, size=min(192, n), replace=False))
    mask = np.zeros(n, np.uint8)
    mask[idx] = 1
    po, go, _ = oracle.fmm(w.tree, w.rho, leaf_mask=mask)
    ephi, eg = _errs(phi, g, po, go, idx)
    assert ephi <= TOL_MIXED and eg <= TOL_MIXED, (ephi, eg)
    assert np.all(np.isfinite(phi)) and np.all(np.isfinite(g))


def test_mixed_is_not_the_fp64_path():
    """The mixed path must differ from the float64 path (at float32 rounding level)."""
    w = W.uniform16(0)
    p64, g64 = _solve(w.tree, w.rho, binding.OCTO_FP64)
    p32, g32 = _solve(w.tree, w.rho, binding.OCTO_MIXED)
    d = np.max(np.abs(p32 - p64) / np.abs(p64))
    assert 1e-12 < d < 1e-6


def test_mixed_physical_units():
    """Cell-width scaling keeps float32 in range for astrophysical units
    (extent 1e11 cm, densities ~1 g/cm^3)."""
    w = W.uniform16(1)
    tree = W.Tree(w.tree.level, w.tree.ijk, w.tree.children, np.array([-5e10, -5e10, -5e10]), 1e11)
    phi, g = _solve(tree, w.rho, binding.OCTO_MIXED)
    po, go, _ = oracle.fmm(tree, w.rho)
    ephi, eg = _errs(phi, g, po, go)
    assert ephi <= TOL_MIXED and eg <= TOL_MIXED, (ephi, eg)
