"""Whole-solve pins of the oracle: brute-force direct sums, an independent count of
the interaction lists, pair coverage, conservation laws (Section IV-C), exact
homogeneity, mirror symmetry and closed-form potentials."""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2304_11002_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _masses(w):
    return w.rho.reshape(-1) * w.tree.leaf_cell_h() ** 3


def stencil_counts_uniform(max_level: int, theta: float = 0.5):
    """Independent count of ordered same-level M2L and P2P pairs of a complete
    octree, from the definition 'far on this level and parents not far' (with all
    pairs of root cells at level 0), summed per offset d and cell parity p:
    sum_p sum_d [cond(d, p)] prod_axis #{i with parity p_a, i and i+d_a inside}."""
    def far(q2):  # same-level cells at squared integer distance q2
        return theta * theta * (4 * q2) >= 12
    m2l = 0
    for lv in range(max_level + 1):
        n = 8 << lv
        R = 15
        ds = np.arange(-R, R + 1)
        for p in itertools.product((0, 1), repeat=3):
            cnt = []
            for a in range(3):
                i = np.arange(p[a], n, 2)
                cnt.append(np.array([np.sum((i + d >= 0) & (i + d < n)) for d in ds]))
            for dx, dy, dz in itertools.product(range(len(ds)), repeat=3):
                d = np.array([ds[dx], ds[dy], ds[dz]])
                if not far(int(d @ d)):
                    continue
                if lv > 0:
                    pd = (np.array(p) + d) // 2  # parent offset for a cell of parity p
                    if far(int(pd @ pd)):
                        continue
                m2l += int(cnt[0][dx]) * int(cnt[1][dy]) * int(cnt[2][dz])
    n = 8 << max_level
    p2p = 0
    for d in itertools.product(range(-3, 4), repeat=3):
        d = np.array(d)
        q = int(d @ d)
        if q == 0 or far(q):
            continue
        p2p += int(np.prod([n - abs(x) for x in d]))
    return m2l, p2p


def test_counts_match_independent_stencil_count():
    w = W.uniform16(0)
    c = oracle.counts(w.tree)
    m2l, p2p = stencil_counts_uniform(1)
    assert (c[0], c[2]) == (m2l, p2p)
    assert c[1] == 0 and c[3] == 0
    w2 = W.binary32()
    c2 = oracle.counts(w2.tree)
    assert (c2[0], c2[2]) == stencil_counts_uniform(2)


def test_counts_golden():
    """Golden ordered counts of complete trees (tests/golden/counts_uniform.txt)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "counts_uniform.txt")) if l.strip() and l[0] != "#"]
    for name, lv, m2l, p2p in rows:
        assert stencil_counts_uniform(int(lv)) == (int(m2l), int(p2p)), name
    c = oracle.counts(W.uniform16(0).tree)
    assert (c[0], c[2]) == (int(rows[0][2]), int(rows[0][3]))


def _tiny_adaptive():
    refined = {(0, 0, 0, 0), (1, 1, 0, 0)}
    return W.tree_from_refined(refined, 16.0)


@pytest.mark.parametrize("which", ["uniform16", "tiny_adaptive"])
def test_every_leaf_pair_covered_exactly_once(which):
    tree = W.uniform16(0).tree if which == "uniform16" else _tiny_adaptive()
    cov = oracle.coverage(tree)
    n = cov.shape[0]
    assert np.all(np.diag(cov) == 0)
    off = cov[~np.eye(n, dtype=bool)]
    assert off.min() == 1 and off.max() == 1
    if which == "tiny_adaptive":
        c = oracle.counts(tree)
        assert c[1] > 0 and c[3] > 0  # cross-level M2L and P2P both occur


def test_fmm_vs_direct_sum_uniform16():
    """Config 1: FMM (theta 0.5, order 3) against the 4096^2 direct sum."""
    for seed in range(3):
        w = W.uniform16(seed)
        phi, g, _ = oracle.fmm(w.tree, w.rho)
        pd, gd = oracle.direct(w.tree, w.rho)
        ephi = np.max(np.abs(phi - pd)) / np.max(np.abs(pd))
        eg = np.max(np.linalg.norm(g - gd, axis=0)) / np.max(np.linalg.norm(gd, axis=0))
        assert ephi < 1e-4 and eg < 3e-3, (seed, ephi, eg)


def test_fmm_error_falls_with_theta():
    w = W.uniform16(1)
    pd, gd = oracle.direct(w.tree, w.rho)
    errs = []
    for th in (0.5, 0.35, 0.25):
        phi, g, _ = oracle.fmm(w.tree, w.rho, theta=th)
        errs.append(np.max(np.linalg.norm(g - gd, axis=0)) / np.max(np.linalg.norm(gd, axis=0)))
    assert errs[0] > errs[1] > errs[2], errs


def test_fmm_vs_direct_tiny_adaptive():
    tree = _tiny_adaptive()
    rng = np.random.default_rng(7)
    rho = rng.lognormal(size=(tree.n_leaf, 512))
    phi, g, _ = oracle.fmm(tree, rho)
    pd, gd = oracle.direct(tree, rho)
    assert np.max(np.abs(phi - pd)) / np.max(np.abs(pd)) < 1e-4
    assert np.max(np.linalg.norm(g - gd, axis=0)) / np.max(np.linalg.norm(gd, axis=0)) < 3e-3


@pytest.mark.parametrize("which", ["uniform16", "tiny_adaptive"])
def test_linear_and_angular_momentum(which):
    """sum m g = 0 (Newton III) and sum m x cross g = 0 with the correction; without
    it the torque is many orders of magnitude larger (Section IV-C)."""
    if which == "uniform16":
        w = W.uniform16(2)
        tree, rho = w.tree, w.rho
    else:
        tree = _tiny_adaptive()
        rho = np.random.default_rng(8).lognormal(size=(tree.n_leaf, 512))
    m = rho.reshape(-1) * tree.leaf_cell_h() ** 3
    x = tree.leaf_cell_centres()
    phi, g, _ = oracle.fmm(tree, rho)
    F = (m[None, :] * g).T
    assert np.linalg.norm(F.sum(0)) <= 1e-13 * np.abs(F).sum()
    tau = np.cross(x, F)
    assert np.linalg.norm(tau.sum(0)) <= 1e-13 * np.abs(tau).sum()
    _, g0, _ = oracle.fmm(tree, rho, correction=False)
    tau0 = np.cross(x, (m[None, :] * g0).T)
    assert np.linalg.norm(tau0.sum(0)) > 1e4 * np.linalg.norm(tau.sum(0))


def test_homogeneity_bit_exact():
    w = W.uniform16(0)
    phi, g, _ = oracle.fmm(w.tree, w.rho)
    phi2, g2, _ = oracle.fmm(w.tree, 2.0 * w.rho)
    assert np.array_equal(phi2, 2.0 * phi) and np.array_equal(g2, 2.0 * g)


def test_mirror_symmetry():
    """Reflecting the density in x reflects phi and flips g_x (to rounding)."""
    w = W.uniform16(0)
    x = w.tree.leaf_cell_centres()
    key = {tuple(v): i for i, v in enumerate(x)}
    perm = np.array([key[(w.tree.extent - v[0], v[1], v[2])] for v in x])
    rho_m = w.rho.reshape(-1)[perm]
    phi, g, _ = oracle.fmm(w.tree, w.rho)
    phim, gm, _ = oracle.fmm(w.tree, rho_m)
    s = np.max(np.abs(phi))
    assert np.max(np.abs(phim - phi[perm])) <= 1e-13 * s
    gs = np.max(np.abs(g))
    assert np.max(np.abs(gm[0] + g[0][perm])) <= 1e-13 * gs
    assert np.max(np.abs(gm[1:] - g[1:][:, perm])) <= 1e-13 * gs


def _closed_form_error(max_level, profile):
    extent = 8.0 * 2 ** max_level
    tree = W.uniform_tree(max_level, extent)
    x = tree.leaf_cell_centres()
    R = extent / 4.0
    c = np.full(3, extent / 2.0)
    r = np.linalg.norm(x - c, axis=1)
    rho, phi_exact = profile(r, R)
    rho = rho + W.FLOOR
    rng = np.random.default_rng(0)
    inside = np.nonzero(r < 1.5 * R)[0]
    pick = rng.choice(inside, size=48, replace=False)
    mask = np.zeros(x.shape[0], dtype=np.uint8)
    mask[pick] = 1
    phi, g, _ = oracle.fmm(tree, rho.reshape(tree.n_leaf, 512), leaf_mask=mask)
    return np.max(np.abs(phi[pick] - phi_exact[pick])) / np.max(np.abs(phi_exact[pick]))


def _uniform_sphere(r, R):
    M = 4.0 / 3.0 * np.pi * R ** 3
    rho = np.where(r < R, 1.0, 0.0)
    phi = np.where(r < R, -M * (3 * R * R - r * r) / (2 * R ** 3), -M / np.maximum(r, 1e-300))
    return rho, phi


def _polytrope_n1(r, R):
    alpha = R / np.pi
    xi = np.pi * r / R
    s = np.where(xi > 0, np.sin(xi) / np.where(xi > 0, xi, 1.0), 1.0)
    rho = np.where(r < R, s, 0.0)
    M = 4.0 * np.pi ** 2 * alpha ** 3
    phi = np.where(r < R, -4.0 * np.pi * alpha ** 2 * (1.0 + s), -M / np.maximum(r, 1e-300))
    return rho, phi


@pytest.mark.parametrize("profile", [_uniform_sphere, _polytrope_n1])
def test_closed_form_potentials_converge(profile):
    """Uniform sphere and n=1 polytrope (R/h = 4, 8, 16): the point-mass
    discretisation error must fall with resolution."""
    errs = [_closed_form_error(lv, profile) for lv in (1, 2, 3)]
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 0.01, errs
