"""CPU FP64 oracle of the FMM self-gravity solve (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` leg of ``bench.py`` may import this package.  The product
path (the CUDA library and its binding) never does, and the two share no code.

Array conventions (numpy, float64 unless stated):
  rho, phi      [n_leaf * 512]       leaf order, cells x-fastest inside a leaf
  g             [3, n_leaf * 512]    structure of arrays
  multipoles    [20, n_nodes * 512]  m, X(3), M2 {xx,xy,xz,yy,yz,zz}, M3 {xxx,xxy,xxz,xyy,xyz,xzz,yyy,yyz,yzz,zzz}
  local exp.    [23, n_nodes * 512]  L0, L1(3), L2(6), L3(10), dg(3)
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

from . import build_oracle

_LIB = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def lib():
    global _LIB
    if _LIB is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        tree_args = [ctypes.c_int, _ip, _ip, _ip, _dp, ctypes.c_double]
        L.oracle_upward.argtypes = tree_args + [_dp, _dp]
        L.oracle_fmm.argtypes = tree_args + [_dp, ctypes.c_double, ctypes.c_int, _u8p, _dp, _dp, _dp, _i64p]
        L.oracle_fmm_jvp.argtypes = tree_args + [_dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _u8p,
                                                 _dp, _dp, _dp, _dp]
        L.oracle_direct.argtypes = tree_args + [_dp, _u8p, _dp, _dp]
        L.oracle_counts.argtypes = tree_args + [ctypes.c_double, _i64p]
        L.oracle_coverage.argtypes = tree_args + [ctypes.c_double, _ip]
        L.oracle_dtensors.argtypes = [_dp, _dp]
        L.oracle_m2l_pair.argtypes = [_dp, _dp, ctypes.c_int, _dp]
        L.oracle_m2m.argtypes = [_dp, ctypes.c_int, _dp]
        L.oracle_l2l.argtypes = [_dp, _dp, _dp]
        for f in (L.oracle_upward, L.oracle_fmm, L.oracle_fmm_jvp, L.oracle_direct, L.oracle_counts,
                  L.oracle_coverage):
            f.restype = ctypes.c_int
        for f in (L.oracle_dtensors, L.oracle_m2l_pair, L.oracle_m2m, L.oracle_l2l):
            f.restype = None
        _LIB = L
    return _LIB


def set_threads(n: int = 0) -> int:
    """Thread count of the oracle's OpenMP loops (n <= 0 leaves it); returns the
    count in effect."""
    L = lib()
    L.oracle_set_threads.argtypes = [ctypes.c_int]
    L.oracle_set_threads.restype = ctypes.c_int
    return int(L.oracle_set_threads(int(n)))


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


class _TreeArgs:
    def __init__(self, tree):
        self.level = np.ascontiguousarray(tree.level, dtype=np.int32)
        self.ijk = np.ascontiguousarray(tree.ijk, dtype=np.int32)
        self.children = np.ascontiguousarray(tree.children, dtype=np.int32)
        self.origin = np.ascontiguousarray(tree.origin, dtype=np.float64)
        self.extent = float(tree.extent)
        self.n = int(self.level.shape[0])

    def args(self):
        return [self.n, _p(self.level, _ip), _p(self.ijk, _ip), _p(self.children, _ip), _p(self.origin, _dp),
                self.extent]


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"{what}: oracle returned {rc}")


def _mask(tree, leaf_mask):
    if leaf_mask is None:
        return None
    m = np.ascontiguousarray(np.asarray(leaf_mask).reshape(-1), dtype=np.uint8)
    assert m.size == tree.n_leaf * 512
    return m


def upward(tree, rho) -> np.ndarray:
    ta = _TreeArgs(tree)
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
    out = np.empty((20, ta.n * 512))
    _check(lib().oracle_upward(*ta.args(), _p(rho, _dp), _p(out, _dp)), "upward")
    return out


def fmm(tree, rho, theta: float = 0.5, correction: bool = True, leaf_mask=None,
        want_local: bool = False, work: Optional[np.ndarray] = None) -> Tuple[np.ndarray, np.ndarray, Optional[np.ndarray]]:
    """phi [n_leaf*512], g [3, n_leaf*512] (NaN where not selected), local [23, n_nodes*512] or None.
    `work` (int64 array of size 1, optional) receives the number of ordered interactions evaluated."""
    ta = _TreeArgs(tree)
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
    nl = tree.n_leaf * 512
    phi = np.full(nl, np.nan)
    g = np.full((3, nl), np.nan)
    loc = np.empty((23, ta.n * 512)) if want_local else None
    m = _mask(tree, leaf_mask)
    _check(lib().oracle_fmm(*ta.args(), _p(rho, _dp), float(theta), 1 if correction else 0, _p(m, _u8p),
                            _p(phi, _dp), _p(g, _dp), _p(loc, _dp), _p(work, _i64p)), "fmm")
    return phi, g, loc


def fmm_jvp(tree, rho, u, theta: float = 0.5, correction: bool = True, leaf_mask=None, eps: float = 1e-30):
    """Complex-step directional derivative of (phi, g) along u: returns phi, g, dphi, dg."""
    ta = _TreeArgs(tree)
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    nl = tree.n_leaf * 512
    phi, dphi = np.full(nl, np.nan), np.full(nl, np.nan)
    g, dg = np.full((3, nl), np.nan), np.full((3, nl), np.nan)
    m = _mask(tree, leaf_mask)
    _check(lib().oracle_fmm_jvp(*ta.args(), _p(rho, _dp), _p(u, _dp), float(eps), float(theta),
                                1 if correction else 0, _p(m, _u8p), _p(phi, _dp), _p(g, _dp), _p(dphi, _dp),
                                _p(dg, _dp)), "fmm_jvp")
    return phi, g, dphi, dg


def direct(tree, rho, leaf_mask=None) -> Tuple[np.ndarray, np.ndarray]:
    ta = _TreeArgs(tree)
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
    nl = tree.n_leaf * 512
    phi = np.full(nl, np.nan)
    g = np.full((3, nl), np.nan)
    m = _mask(tree, leaf_mask)
    _check(lib().oracle_direct(*ta.args(), _p(rho, _dp), _p(m, _u8p), _p(phi, _dp), _p(g, _dp)), "direct")
    return phi, g


def counts(tree, theta: float = 0.5) -> np.ndarray:
    """Ordered interaction counts: [M2L same level, M2L cross level, P2P same level, P2P cross level]."""
    ta = _TreeArgs(tree)
    out = np.zeros(4, dtype=np.int64)
    _check(lib().oracle_counts(*ta.args(), float(theta), _p(out, _i64p)), "counts")
    return out


def coverage(tree, theta: float = 0.5) -> np.ndarray:
    ta = _TreeArgs(tree)
    nl = tree.n_leaf * 512
    out = np.zeros((nl, nl), dtype=np.int32)
    _check(lib().oracle_coverage(*ta.args(), float(theta), _p(out, _ip)), "coverage")
    return out


def dtensors(R) -> dict:
    R = np.ascontiguousarray(R, dtype=np.float64)
    out = np.empty(1 + 3 + 9 + 27 + 81)
    lib().oracle_dtensors(_p(R, _dp), _p(out, _dp))
    return {"D0": out[0], "D1": out[1:4], "D2": out[4:13].reshape(3, 3), "D3": out[13:40].reshape(3, 3, 3),
            "D4": out[40:121].reshape(3, 3, 3, 3)}


def m2l_pair(A, B, correction: bool = True) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    out = np.empty(23)
    lib().oracle_m2l_pair(_p(A, _dp), _p(B, _dp), 1 if correction else 0, _p(out, _dp))
    return out


def m2m(children) -> np.ndarray:
    ch = np.ascontiguousarray(children, dtype=np.float64).reshape(-1, 20)
    out = np.empty(20)
    lib().oracle_m2m(_p(ch, _dp), int(ch.shape[0]), _p(out, _dp))
    return out


def l2l(parent, delta) -> np.ndarray:
    P = np.ascontiguousarray(parent, dtype=np.float64)
    d = np.ascontiguousarray(delta, dtype=np.float64)
    out = np.empty(23)
    lib().oracle_l2l(_p(P, _dp), _p(d, _dp), _p(out, _dp))
    return out


def fmm_vjp(tree, rho, phib, gb, theta: float = 0.5, correction: bool = True) -> np.ndarray:
    """drho = (dphi/drho)^T phib + (dg/drho)^T gb (reverse of every step of the solve)."""
    ta = _TreeArgs(tree)
    L = lib()
    if not getattr(L, "_vjp_typed", False):
        L.oracle_fmm_vjp.argtypes = [ctypes.c_int, _ip, _ip, _ip, _dp, ctypes.c_double, _dp, ctypes.c_double,
                                     ctypes.c_int, _dp, _dp, _dp]
        L.oracle_fmm_vjp.restype = ctypes.c_int
        L.oracle_dtensor5.argtypes = [_dp, _dp]
        L.oracle_dtensor5.restype = None
        L._vjp_typed = True
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
    phib = np.ascontiguousarray(phib, dtype=np.float64).reshape(-1)
    gb = np.ascontiguousarray(gb, dtype=np.float64).reshape(3, -1)
    out = np.empty_like(rho)
    _check(L.oracle_fmm_vjp(*ta.args(), _p(rho, _dp), float(theta), 1 if correction else 0, _p(phib, _dp),
                            _p(gb, _dp), _p(out, _dp)), "fmm_vjp")
    return out


def dtensor5(R) -> np.ndarray:
    fmm_vjp  # ensure argtypes are set by a first call path
    L = lib()
    L.oracle_dtensor5.argtypes = [_dp, _dp]
    L.oracle_dtensor5.restype = None
    R = np.ascontiguousarray(R, dtype=np.float64)
    out = np.empty(243)
    L.oracle_dtensor5(_p(R, _dp), _p(out, _dp))
    return out.reshape(3, 3, 3, 3, 3)
