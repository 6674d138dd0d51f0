"""Edge cases of the solve against the oracle, both precisions: a tree of one leaf
node (the root; every pair is a point-mass pair), the ends of the supported
opening-parameter range (theta = 1 and theta = 0.45; 0.433 <= theta <= 1 keeps the
near field within the 26 neighbouring subgrids), an offset domain whose extent is
not a power of two, a narrow deep refinement (one corner refined down to level 6,
so that pairs cross levels on every level), and densities spanning 20 orders of
magnitude."""
import numpy as np
import pytest

import oracle
from paper_2304_11002_gb300 import binding
from paper_2304_11002_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {binding.OCTO_FP64: 1e-12, binding.OCTO_MIXED: 1e-6}


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_11002_gb300 import build
    build.build()


def _errs(phi, g, po, go):
    ephi = float(np.max(np.abs(phi - po) / np.abs(po)))
    eg = float(np.max(np.linalg.norm(g - go, axis=0)) / np.max(np.linalg.norm(go, axis=0)))
    return ephi, eg


def _check(tree, rho, theta=0.5, precisions=(binding.OCTO_FP64, binding.OCTO_MIXED)):
    po, go, _ = oracle.fmm(tree, rho, theta)
    r = torch.from_numpy(np.ascontiguousarray(rho.reshape(-1))).cuda()
    for precision in precisions:
        fmm = binding.OctoFMM(tree, theta, precision)
        np.testing.assert_array_equal(fmm.counts(), oracle.counts(tree, theta))
        phi, g = fmm.forces(r)
        torch.cuda.synchronize()
        binding.octo_fmm_stats(fmm.handle)
        ephi, eg = _errs(phi.cpu().numpy(), g.cpu().numpy(), po, go)
        assert ephi <= TOL[precision] and eg <= TOL[precision], (precision, ephi, eg)


def test_single_node_tree():
    tree = W.tree_from_refined(set(), 8.0)
    rho = np.random.default_rng(41).lognormal(size=(1, 512))
    _check(tree, rho)


@pytest.mark.parametrize("theta", [1.0, 0.45])
def test_theta_range(theta):
    tree = W.tree_from_refined({(0, 0, 0, 0), (1, 1, 0, 0), (1, 0, 1, 1)}, 16.0)
    rho = np.random.default_rng(42).lognormal(size=(tree.n_leaf, 512))
    _check(tree, rho, theta)


def test_offset_domain_non_power_of_two_extent():
    t = W.tree_from_refined({(0, 0, 0, 0), (1, 1, 1, 0)}, 16.0)
    tree = W.Tree(t.level, t.ijk, t.children, np.array([-1.25, 0.3, 5.0]), 3.7)
    rho = np.random.default_rng(43).lognormal(size=(tree.n_leaf, 512))
    _check(tree, rho)


def test_deep_narrow_refinement():
    """The corner node of every level refined down to level 6 (7 levels), 2:1
    balanced; 192 sampled cells against the oracle."""
    tree = W.tree_from_refined(W.balance_2to1({(l, 0, 0, 0) for l in range(6)}), 1.0)
    rng = np.random.default_rng(44)
    rho = rng.lognormal(size=(tree.n_leaf, 512))
    nl = tree.n_leaf * 512
    idx = np.sort(rng.choice(nl, size=192, replace=False))
    mask = np.zeros(nl, np.uint8)
    mask[idx] = 1
    po, go, _ = oracle.fmm(tree, rho, leaf_mask=mask)
    r = torch.from_numpy(rho.reshape(-1).copy()).cuda()
    for precision in (binding.OCTO_FP64, binding.OCTO_MIXED):
        fmm = binding.OctoFMM(tree, 0.5, precision)
        phi, g = fmm.forces(r)
        torch.cuda.synchronize()
        binding.octo_fmm_stats(fmm.handle)
        ephi, eg = _errs(phi.cpu().numpy()[idx], g.cpu().numpy()[:, idx], po[idx], go[:, idx])
        assert ephi <= TOL[precision] and eg <= TOL[precision], (precision, ephi, eg)


def test_density_spanning_twenty_decades():
    """Stellar-surface contrast: densities from 1e-10 to 1e10 in one tree."""
    tree = W.tree_from_refined({(0, 0, 0, 0), (1, 1, 0, 0)}, 16.0)
    rho = 10.0 ** np.random.default_rng(45).uniform(-10, 10, size=(tree.n_leaf, 512))
    _check(tree, rho, precisions=(binding.OCTO_FP64,))
