"""Pins of the oracle's vector-Jacobian product: symbolic fifth derivatives, the
dot-product identity <v, J u> = <J^T v, u> with J u from complex-step
differentiation of the forward oracle, central finite differences, and the
gravitational-energy identity dE/drho_i ~ phi_i dV (exact for the direct sum, to
expansion accuracy for the FMM whose expansions are centred on centres of mass)."""
import itertools

import numpy as np
import pytest
import sympy as sp

import oracle
from paper_2304_11002_gb300 import workloads as W


def _tiny_adaptive():
    return W.tree_from_refined({(0, 0, 0, 0), (1, 1, 0, 0)}, 16.0)


def test_fifth_derivative_tensor_symbolic():
    x, y, z = sp.symbols("x y z", real=True)
    X = (x, y, z)
    f = 1 / sp.sqrt(x * x + y * y + z * z)
    R = np.array([1.7, -0.4, 2.3])
    subs = dict(zip(X, [sp.Float(v, 30) for v in R]))
    D5 = oracle.dtensor5(R)
    seen = {}
    for idx in itertools.product(range(3), repeat=5):
        key = tuple(sorted(idx))
        if key not in seen:
            ex = f
            for i in key:
                ex = sp.diff(ex, X[i])
            seen[key] = float(ex.subs(subs))
        assert abs(D5[idx] - seen[key]) <= 1e-13 * max(abs(seen[key]), 1e-3)


@pytest.fixture(scope="module")
def tiny_case():
    tree = _tiny_adaptive()
    rng = np.random.default_rng(21)
    rho = rng.lognormal(size=(tree.n_leaf, 512))
    return tree, rho


def test_vjp_dot_product_with_complex_step(tiny_case):
    tree, rho = tiny_case
    n = rho.size
    rng = np.random.default_rng(22)
    vphi, vg, u = rng.normal(size=n), rng.normal(size=(3, n)), rng.normal(size=n)
    rb = oracle.fmm_vjp(tree, rho, vphi, vg)
    _, _, dphi, dg = oracle.fmm_jvp(tree, rho, u)
    lhs = vphi @ dphi + np.sum(vg * dg)
    assert abs(lhs - rb @ u) <= 1e-12 * abs(lhs)
    # the correction's own adjoint is exercised too
    rb0 = oracle.fmm_vjp(tree, rho, vphi, vg, correction=False)
    _, _, dphi0, dg0 = oracle.fmm_jvp(tree, rho, u, correction=False)
    lhs0 = vphi @ dphi0 + np.sum(vg * dg0)
    assert abs(lhs0 - rb0 @ u) <= 1e-12 * abs(lhs0)
    assert abs(lhs0 - lhs) > 1e-10 * abs(lhs)


def test_vjp_against_finite_differences():
    """Central differences with h_i = 1e-6 rho_i on a 16^3 case, loss
    l = sum w_i g_x,i with w ~ N(0, 1)."""
    w = W.uniform16(3)
    rho = w.rho.reshape(-1)
    n = rho.size
    rng = np.random.default_rng(23)
    wts = rng.normal(size=n)
    gb = np.zeros((3, n))
    gb[0] = wts
    rb = oracle.fmm_vjp(w.tree, rho, np.zeros(n), gb)
    for i in rng.choice(n, size=4, replace=False):
        hs = 1e-6 * rho[i]
        rp, rm = rho.copy(), rho.copy()
        rp[i] += hs
        rm[i] -= hs
        _, gp, _ = oracle.fmm(w.tree, rp)
        _, gm, _ = oracle.fmm(w.tree, rm)
        fd = (wts @ gp[0] - wts @ gm[0]) / (2 * hs)
        assert abs(rb[i] - fd) <= 1e-6 * np.max(np.abs(rb)), (i, rb[i], fd)


def test_energy_gradient_close_to_potential():
    """E = 1/2 sum rho phi dV: dE/drho = phi dV holds to expansion accuracy."""
    w = W.uniform16(4)
    rho = w.rho.reshape(-1)
    dV = w.tree.leaf_cell_h() ** 3
    phi, g, _ = oracle.fmm(w.tree, rho)
    rb = oracle.fmm_vjp(w.tree, rho, 0.5 * rho * dV, np.zeros((3, rho.size)))
    dE = 0.5 * phi * dV + rb
    err = np.max(np.abs(dE - phi * dV)) / np.max(np.abs(phi * dV))
    assert err < 1e-3, err
