"""CPU float64 oracle of one self-consistent-field (SCF) step (test infrastructure).

Only the test suite may import this module; the product path (the CUDA library and
its binding) never does, and the two share no code.

Section IV-C of the paper builds its binary models with an iterative SCF
technique: the hydrostatic equilibrium equation in the rotating frame integrates
to an algebraic relation between the effective potential and the enthalpy.  For
a polytrope P = K rho^(1 + 1/n) the enthalpy is H = (n + 1) K rho^(1/n), and in a
frame rotating rigidly with angular velocity Omega about an axis parallel to z,

    H + Phi - Omega^2 w^2 / 2 = C_i      inside star i,

with w the distance from the rotation axis.  The paper states this much and no
more; the step below is our reading (the two-star version of Hachisu's scheme):

  1. the rotation axis passes through the centre of mass of the current density
     (leaf cells as point masses m = rho h^3);
  2. H = 0 at three given surface cells: A and B on star 1, C on star 2, which
     fixes Omega^2 = 2 (Phi_A - Phi_B) / (w_A^2 - w_B^2),
     C_1 = Phi_A - Omega^2 w_A^2 / 2 and C_2 = Phi_C - Omega^2 w_C^2 / 2;
  3. a cell belongs to star 1 if its x < x_split, else to star 2;
     H = C_i - Phi + Omega^2 w^2 / 2;
  4. each star keeps its maximum density rho_max_i:
     rho_new = rho_max_i (H / H_max_i)^n + rho_floor where H > 0, else rho_floor,
     with H_max_i the largest H over star i's cells;
  5. diagnostics of the state that produced Phi: the largest density change over
     max(rho_max), and the virial terms W = sum m Phi / 2, T = Omega^2 sum m w^2 / 2,
     Pi = sum P h^3 with P = K_i rho^(1 + 1/n), K_i = H_max_i / ((n + 1) rho_max_i^(1/n)),
     virial error |2 T + W + 3 Pi| / |W|.
"""
from __future__ import annotations

import numpy as np

from . import fmm as oracle_fmm

STAT_NAMES = ("omega2", "c1", "c2", "max_change", "W", "T", "Pi", "virial_error")


def scf_step(tree, rho, phi, n, rho_max, rho_floor, cell_a, cell_b, cell_c, x_split):
    """One SCF step.  rho, phi: [n_leaf * 512] in the tree's leaf order.  Returns
    (rho_new, stats) with stats a dict over STAT_NAMES."""
    rho = np.asarray(rho, dtype=np.float64).reshape(-1)
    phi = np.asarray(phi, dtype=np.float64).reshape(-1)
    x = tree.leaf_cell_centres()
    h = tree.leaf_cell_h()
    dV = h ** 3
    m = rho * dV
    # 1. rotation axis through the centre of mass
    M = m.sum()
    xc = (m * x[:, 0]).sum() / M
    yc = (m * x[:, 1]).sum() / M
    w2 = (x[:, 0] - xc) ** 2 + (x[:, 1] - yc) ** 2
    # 2. constants from the three surface cells
    omega2 = 2.0 * (phi[cell_a] - phi[cell_b]) / (w2[cell_a] - w2[cell_b])
    c1 = phi[cell_a] - 0.5 * omega2 * w2[cell_a]
    c2 = phi[cell_c] - 0.5 * omega2 * w2[cell_c]
    # 3. enthalpy
    star1 = x[:, 0] < x_split
    H = np.where(star1, c1, c2) - phi + 0.5 * omega2 * w2
    # 4. new density
    hmax1 = H[star1].max()
    hmax2 = H[~star1].max()
    hmax = np.where(star1, hmax1, hmax2)
    rmax = np.where(star1, rho_max[0], rho_max[1])
    pos = H > 0.0
    rho_new = np.full_like(rho, rho_floor)
    rho_new[pos] = rmax[pos] * (H[pos] / hmax[pos]) ** n + rho_floor
    # 5. diagnostics
    K = hmax / ((n + 1.0) * rmax ** (1.0 / n))
    W = 0.5 * (m * phi).sum()
    T = 0.5 * omega2 * (m * w2).sum()
    Pi = (K * rho ** (1.0 + 1.0 / n) * dV).sum()
    stats = {"omega2": omega2, "c1": c1, "c2": c2,
             "max_change": np.abs(rho_new - rho).max() / max(rho_max[0], rho_max[1]),
             "W": W, "T": T, "Pi": Pi, "virial_error": abs(2.0 * T + W + 3.0 * Pi) / abs(W)}
    return rho_new, stats


def scf_solve(tree, rho0, n, rho_max, rho_floor, cell_a, cell_b, cell_c, x_split, steps, theta=0.5):
    """`steps` SCF steps, each on the potential of the oracle FMM of the current
    density.  Returns (rho, [stats of every step])."""
    rho = np.array(rho0, dtype=np.float64).reshape(-1)
    history = []
    for _ in range(steps):
        phi, _, _ = oracle_fmm(tree, rho, theta)
        rho, st = scf_step(tree, rho, phi, n, rho_max, rho_floor, cell_a, cell_b, cell_c, x_split)
        history.append(st)
    return rho, history
