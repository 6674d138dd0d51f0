"""Pins of the oracle's building blocks against mathematics that does not come
from the oracle itself: symbolic derivatives, brute-force moment sums, polynomial
identities and the Taylor-remainder order of the expansion."""
import itertools

import numpy as np
import pytest
import sympy as sp

import oracle

P2 = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
P3 = [(0, 0, 0), (0, 0, 1), (0, 0, 2), (0, 1, 1), (0, 1, 2), (0, 2, 2), (1, 1, 1), (1, 1, 2), (1, 2, 2), (2, 2, 2)]


def test_derivative_tensors_match_symbolic():
    """D^(n) = grad^n (1/|R|) for n = 0..4 (the expansion kernels of the M2L)."""
    x, y, z = sp.symbols("x y z", real=True)
    X = (x, y, z)
    f = 1 / sp.sqrt(x * x + y * y + z * z)
    rng = np.random.default_rng(1)
    for R in [np.array([1.3, -0.7, 2.1]), rng.normal(size=3) * 5, np.array([3.0, 0.0, 0.0])]:
        subs = dict(zip(X, [sp.Float(v, 30) for v in R]))
        d = oracle.dtensors(R)
        scale = np.linalg.norm(R)
        assert abs(float(f.subs(subs)) - d["D0"]) <= 1e-15 / scale
        for n, key in [(1, "D1"), (2, "D2"), (3, "D3"), (4, "D4")]:
            ref = np.empty((3,) * n)
            for idx in itertools.product(range(3), repeat=n):
                ex = f
                for i in idx:
                    ex = sp.diff(ex, X[i])
                ref[idx] = float(ex.subs(subs))
            tol = 1e-14 * np.max(np.abs(ref))
            np.testing.assert_allclose(d[key], ref, rtol=0, atol=tol)


def _packed_moments(m, x):
    """Brute-force moments of point masses about their centre of mass, packed."""
    M = m.sum()
    X = (m[:, None] * x).sum(0) / M
    s = x - X
    out = np.zeros(20)
    out[0] = M
    out[1:4] = X
    for q, (a, b) in enumerate(P2):
        out[4 + q] = np.sum(m * s[:, a] * s[:, b])
    for q, (a, b, c) in enumerate(P3):
        out[10 + q] = np.sum(m * s[:, a] * s[:, b] * s[:, c])
    return out


def test_m2m_equals_direct_moments_two_levels():
    """Two M2M steps over 8x8 point masses give the moments of all 64 points."""
    rng = np.random.default_rng(2)
    pts = rng.uniform(-1, 1, size=(64, 3)) + np.array([5.0, -2.0, 1.0])
    m = rng.lognormal(size=64)
    groups = []
    for g in range(8):
        kids = []
        for c in range(8):
            i = 8 * g + c
            leaf = np.zeros(20)
            leaf[0] = m[i]
            leaf[1:4] = pts[i]
            kids.append(leaf)
        groups.append(oracle.m2m(np.array(kids)))
    top = oracle.m2m(np.array(groups))
    ref = _packed_moments(m, pts)
    np.testing.assert_allclose(top, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


def _full2(v):
    T = np.zeros((3, 3))
    for q, (a, b) in enumerate(P2):
        T[a, b] = T[b, a] = v[q]
    return T


def _full3(v):
    T = np.zeros((3, 3, 3))
    for q, (a, b, c) in enumerate(P3):
        for p in set(itertools.permutations((a, b, c))):
            T[p] = v[q]
    return T


def _taylor_eval(Lp, t):
    """Cubic polynomial sum_n L^(n) t^n / n! of a packed local expansion."""
    L2, L3 = _full2(Lp[4:10]), _full3(Lp[10:20])
    return Lp[0] + Lp[1:4] @ t + 0.5 * t @ L2 @ t + np.einsum("abc,a,b,c", L3, t, t, t) / 6.0


def test_l2l_reproduces_cubic_exactly():
    """Shifting the expansion centre leaves the cubic polynomial unchanged."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        Lp = rng.normal(size=23)
        delta = rng.normal(size=3)
        Lc = oracle.l2l(Lp, delta)
        np.testing.assert_allclose(Lc[20:], Lp[20:], rtol=0, atol=0)  # dg carried unshifted
        for _ in range(5):
            x = rng.normal(size=3)
            a = _taylor_eval(Lp, x)
            b = _taylor_eval(Lc, x - delta)
            assert abs(a - b) <= 1e-12 * max(1.0, abs(a))


def _cluster(rng, n, size, centre):
    x = centre + rng.uniform(-size, size, size=(n, 3))
    m = rng.lognormal(size=n)
    return m, x


def test_m2l_truncation_order():
    """phi at the target centre from a far cluster: error of the n+k<=3 expansion
    falls like (s/R)^4 (first dropped term k=4); the force with the correction term
    also falls like (s/R)^4 (the correction restores the k=3 force term)."""
    rng = np.random.default_rng(4)
    base = rng.uniform(-1, 1, size=(40, 3))
    m = rng.lognormal(size=40)
    R0 = np.array([10.0, 3.0, -4.0])
    target = np.zeros(20)
    target[0] = 1.0  # a unit monopole at the origin
    errs_phi, errs_g = [], []
    for s in [1.0, 0.5, 0.25]:
        x = R0 + s * base
        src = _packed_moments(m, x)
        out = oracle.m2l_pair(target, src, correction=True)
        d = -x
        r = np.linalg.norm(d, axis=1)
        phi = -np.sum(m / r)
        g = -np.sum(m[:, None] * d / r[:, None] ** 3, axis=0)
        errs_phi.append(abs(out[0] - phi) / abs(phi))
        errs_g.append(np.linalg.norm((-out[1:4] + out[20:23]) - g) / np.linalg.norm(g))
    for e in (errs_phi, errs_g):
        rates = [np.log2(e[i] / e[i + 1]) for i in range(2)]
        assert all(3.6 < r < 4.6 for r in rates), (e, rates)


def test_m2l_pair_newton_and_torque():
    """Mutual forces of one far pair (as applied to both cells): equal and opposite,
    and with the correction the pair exerts no net torque (Section IV-C's angular
    momentum conservation), i.e. the forces derive from a rotation-invariant energy."""
    rng = np.random.default_rng(5)
    mA, xA = _cluster(rng, 30, 0.8, np.array([0.0, 0.0, 0.0]))
    mB, xB = _cluster(rng, 30, 0.8, np.array([6.0, 2.0, -3.0]))
    A, B = _packed_moments(mA, xA), _packed_moments(mB, xB)
    LA = oracle.m2l_pair(A, B, True)
    LB = oracle.m2l_pair(B, A, True)

    def forces(Lp, m, x, X):
        t = x - X
        L2, L3 = _full2(Lp[4:10]), _full3(Lp[10:20])
        grad = Lp[1:4][None, :] + t @ L2 + 0.5 * np.einsum("abc,nb,nc->na", L3, t, t)
        return m[:, None] * (-grad + Lp[20:23][None, :])

    fA = forces(LA, mA, xA, A[1:4])
    fB = forces(LB, mB, xB, B[1:4])
    F = fA.sum(0) + fB.sum(0)
    scale = np.abs(fA).sum()
    assert np.linalg.norm(F) <= 1e-13 * scale
    tau = np.cross(xA, fA).sum(0) + np.cross(xB, fB).sum(0)
    tscale = np.abs(np.cross(xA, fA)).sum()
    assert np.linalg.norm(tau) <= 1e-13 * tscale
    LA0 = oracle.m2l_pair(A, B, False)
    LB0 = oracle.m2l_pair(B, A, False)
    tau0 = np.cross(xA, forces(LA0, mA, xA, A[1:4])).sum(0) + np.cross(xB, forces(LB0, mB, xB, B[1:4])).sum(0)
    assert np.linalg.norm(tau0) > 1e3 * np.linalg.norm(tau)
