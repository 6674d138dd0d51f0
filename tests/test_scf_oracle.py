"""Pins of the SCF oracle step (oracle/scf_oracle.py) against what the equations fix,
not against a retyped formula:

* a density that already satisfies the algebraic equilibrium H + Phi = C with
  H = (n + 1) K rho^(1/n) (any radial profile) is a fixed point of the step, and
  the step recovers Omega = 0;
* the same star with a rigid-rotation term added to Phi recovers exactly that
  Omega^2 and is again a fixed point;
* on the n = 1 polytrope with its closed-form interior potential the virial
  error 2T + W + 3 Pi (T = 0) is discretisation error only: it falls as the star
  is resolved by more cells.
"""
import math

import numpy as np
import pytest

from oracle import scf_oracle
from paper_2304_11002_gb300 import workloads as W


def _theta(r, R, profile):
    if profile == "parabola":
        return np.clip(1.0 - (r / R) ** 2, 0.0, None)
    xi = np.pi * r / R  # n = 1 Lane-Emden: sin(xi) / xi
    return np.where(r < R, np.where(xi > 0, np.sin(xi) / np.where(xi > 0, xi, 1.0), 1.0), 0.0)


def _stars(tree, centres, R, n, rho_c, K, C, omega2=0.0, axis=(32.5, 32.5), profile="parabola"):
    """rho = rho_c theta_i^n in star i and Phi = C - (n + 1) K rho_c^(1/n) theta_i +
    omega2 w^2 / 2 (w: distance from the z axis through `axis`), theta_i = 0 outside R."""
    x = tree.leaf_cell_centres()
    theta = np.zeros(len(x))
    for c in centres:
        theta += _theta(np.linalg.norm(x - np.asarray(c), axis=1), R, profile)
    w2 = (x[:, 0] - axis[0]) ** 2 + (x[:, 1] - axis[1]) ** 2
    rho = rho_c * theta ** n
    phi = C - (n + 1.0) * K * rho_c ** (1.0 / n) * theta + 0.5 * omega2 * w2
    return rho, phi, x


def _cell_at(x, p):
    return int(np.argmin(np.linalg.norm(x - np.asarray(p), axis=1)))


@pytest.mark.parametrize("n, omega2", [(1.5, 0.0), (1.0, 0.0), (1.5, 3e-4), (3.0, 1e-3)])
def test_equilibrium_binary_is_a_fixed_point(n, omega2):
    """Two equal stars placed symmetrically about x = 32.5, so that the centre of
    mass, and with it the rotation axis, lies at (32.5, 32.5) in x and y."""
    tree = W.uniform_tree(3, 64.0)  # 64^3 cells of width 1
    c1, c2 = np.array([20.5, 32.5, 32.5]), np.array([44.5, 32.5, 32.5])  # cell centres
    R = 10.0
    rho, phi, x = _stars(tree, (c1, c2), R, n, 1.0, 0.7, -5.0, omega2)
    a = _cell_at(x, c1 - [R, 0, 0])  # outer surface of star 1
    b = _cell_at(x, c1 + [R, 0, 0])  # inner surface of star 1
    c = _cell_at(x, c2 - [R, 0, 0])  # inner surface of star 2
    rho_new, st = scf_oracle.scf_step(tree, rho, phi, n, (1.0, 1.0), 0.0, a, b, c, x_split=32.5)
    assert abs(st["omega2"] - omega2) <= 1e-12 * max(omega2, 1.0)
    assert np.max(np.abs(rho_new - rho)) <= 1e-12
    assert st["max_change"] <= 1e-12


def test_virial_error_falls_with_resolution():
    errs = []
    for R in (6.0, 12.0, 24.0):
        tree = W.uniform_tree(3, 64.0)
        c = np.array([32.5, 32.5, 32.5])
        rho_c = 1.0
        K = 2.0 * R * R / np.pi  # n = 1 with G = 1: R = pi sqrt(K / (2 pi))
        M = 4.0 * rho_c * R ** 3 / np.pi
        rho, phi, x = _stars(tree, (c,), R, 1.0, rho_c, K, -M / R, 0.0, profile="lane_emden")
        # outside the star: the potential of a point mass M (H < 0 there)
        r = np.linalg.norm(x - c, axis=1)
        phi = np.where(r < R, phi, -M / np.maximum(r, 1e-9))
        a = _cell_at(x, c + [R, 0, 0])
        b = _cell_at(x, c + [0, 0, R])
        _, st = scf_oracle.scf_step(tree, rho, phi, 1.0, (rho_c, rho_c), 0.0, a, b, a, x_split=60.0)
        assert abs(st["T"]) <= 1e-9 * abs(st["W"])
        errs.append(st["virial_error"])
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 0.02, errs
