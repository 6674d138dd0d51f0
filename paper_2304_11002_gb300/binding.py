"""Thin ctypes binding of the C ABI in include/octo_fmm.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Device buffers
are passed as torch CUDA tensors (float64, contiguous) and streams as
torch.cuda.Stream (default: the current stream).  All arithmetic runs in the
library's CUDA kernels; there is no CPU path.  Loading fails loudly if the
library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liboctofmm.so")

OCTO_OK = 0
OCTO_FP64 = 0
OCTO_MIXED = 1
STATUS = {0: "OCTO_OK", -1: "OCTO_EINVAL", -2: "OCTO_ETREE", -3: "OCTO_ENOMEM", -4: "OCTO_ECUDA",
          -5: "OCTO_ETIMEOUT", -6: "OCTO_ENONPOS", -7: "OCTO_ESTATE"}

# every symbol include/octo_fmm.h declares
SYMBOLS = ["octo_fmm_create", "octo_fmm_upward", "octo_fmm_interact", "octo_fmm_downward", "octo_fmm_forces",
           "octo_fmm_forces_host", "octo_fmm_backward", "octo_fmm_stats", "octo_fmm_plan_counts",
           "octo_fmm_read_state", "octo_fmm_set_option", "octo_fmm_get_option", "octo_fmm_launches_per_solve",
           "octo_fmm_stage_count",
           "octo_fmm_stage_info", "octo_fmm_stage_times", "octo_fmm_subgrids_noalloc", "octo_fmm_measure_peak",
           "octo_fmm_scf_step", "octo_fmm_scf_solve", "octo_fmm_last_error", "octo_fmm_destroy"]


class OctoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class TreeDesc(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("level", ctypes.POINTER(ctypes.c_int32)),
                ("ijk", ctypes.POINTER(ctypes.c_int32)), ("children", ctypes.POINTER(ctypes.c_int32)),
                ("origin", ctypes.c_double * 3), ("extent", ctypes.c_double)]


class ScfParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_double), ("rho_max", ctypes.c_double * 2), ("rho_floor", ctypes.c_double),
                ("cell_a", ctypes.c_int64), ("cell_b", ctypes.c_int64), ("cell_c", ctypes.c_int64),
                ("x_split", ctypes.c_double)]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} is missing: build it with paper_2304_11002_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, dp = ctypes.c_void_p, ctypes.c_void_p
        L.octo_fmm_create.argtypes = [ctypes.POINTER(TreeDesc), ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(vp)]
        L.octo_fmm_upward.argtypes = [vp, dp, vp]
        L.octo_fmm_interact.argtypes = [vp, vp]
        L.octo_fmm_downward.argtypes = [vp, dp, dp, vp]
        L.octo_fmm_forces.argtypes = [vp, dp, dp, dp, vp]
        L.octo_fmm_forces_host.argtypes = [vp, dp, dp, dp, vp]
        L.octo_fmm_backward.argtypes = [vp, dp, dp, dp, vp]
        L.octo_fmm_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
        L.octo_fmm_plan_counts.argtypes = [ctypes.POINTER(TreeDesc), ctypes.c_double, ctypes.POINTER(ctypes.c_int64)]
        L.octo_fmm_read_state.argtypes = [vp, ctypes.c_int, dp]
        L.octo_fmm_set_option.argtypes = [vp, ctypes.c_int, ctypes.c_int64]
        L.octo_fmm_get_option.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
        L.octo_fmm_launches_per_solve.argtypes = [vp]
        L.octo_fmm_stage_count.argtypes = [vp]
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.octo_fmm_stage_info.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), i64p, i64p, i64p, i64p,
                                          i64p]
        L.octo_fmm_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int]
        L.octo_fmm_subgrids_noalloc.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp, dp, vp]
        L.octo_fmm_measure_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), vp]
        L.octo_fmm_scf_step.argtypes = [vp, ctypes.POINTER(ScfParams), dp, dp, ctypes.POINTER(ctypes.c_double), vp]
        L.octo_fmm_scf_solve.argtypes = [vp, ctypes.POINTER(ScfParams), dp, ctypes.c_int, ctypes.c_double,
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), vp]
        L.octo_fmm_last_error.argtypes = [vp]
        L.octo_fmm_last_error.restype = ctypes.c_char_p
        L.octo_fmm_destroy.argtypes = [vp]
        L.octo_fmm_destroy.restype = None
        for name in SYMBOLS:
            f = getattr(L, name)
            if name not in ("octo_fmm_last_error", "octo_fmm_destroy"):
                f.restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int, h=None):
    if rc != OCTO_OK:
        msg = lib().octo_fmm_last_error(h)
        raise OctoError(rc, msg.decode() if msg else "")


class _Desc:
    """Keeps the numpy arrays of a tree descriptor alive while the C struct is used."""

    def __init__(self, tree):
        self.level = np.ascontiguousarray(tree.level, dtype=np.int32)
        self.ijk = np.ascontiguousarray(tree.ijk, dtype=np.int32)
        self.children = np.ascontiguousarray(tree.children, dtype=np.int32)
        ip = ctypes.POINTER(ctypes.c_int32)
        self.desc = TreeDesc(int(self.level.shape[0]), self.level.ctypes.data_as(ip), self.ijk.ctypes.data_as(ip),
                             self.children.ctypes.data_as(ip), (ctypes.c_double * 3)(*[float(v) for v in tree.origin]),
                             float(tree.extent))


def _buf(t, numel: int, device: Optional[int], name: str) -> int:
    """Device address of a buffer the library reads or writes, after checking what the
    kernels assume of it: a contiguous float64 CUDA tensor of exactly `numel`
    elements on `device` (the handle's device).  A wrong size or dtype would make
    the kernels read or write past the allocation, so it is refused here with a
    ValueError before the library is called."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a torch CUDA tensor, got {type(t).__name__}")
    if not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor, got one on {t.device}")
    if t.dtype != torch.float64:
        raise ValueError(f"{name}: expected float64, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    if t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {t.numel()}")
    if device is not None and t.device.index != device:
        raise ValueError(f"{name}: expected a tensor on cuda:{device} (the handle's device), got {t.device}")
    return t.data_ptr()


def _sizes(h):
    """(leaf cells, CUDA device) of handle h, as the library reports them."""
    return octo_fmm_get_option(h, 20), octo_fmm_get_option(h, 21)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def octo_fmm_plan_counts(tree, theta: float = 0.5) -> np.ndarray:
    d = _Desc(tree)
    out = (ctypes.c_int64 * 4)()
    _check(lib().octo_fmm_plan_counts(ctypes.byref(d.desc), float(theta), out))
    return np.array(out[:], dtype=np.int64)


def octo_fmm_create(tree, theta: float = 0.5, order: int = 3, precision: int = OCTO_FP64) -> ctypes.c_void_p:
    d = _Desc(tree)
    h = ctypes.c_void_p()
    _check(lib().octo_fmm_create(ctypes.byref(d.desc), float(theta), int(order), int(precision), ctypes.byref(h)))
    return h


def octo_fmm_destroy(h) -> None:
    lib().octo_fmm_destroy(h)


def octo_fmm_upward(h, rho, stream=None) -> None:
    n, dev = _sizes(h)
    _check(lib().octo_fmm_upward(h, _buf(rho, n, dev, "rho"), _stream(stream)), h)


def octo_fmm_interact(h, stream=None) -> None:
    _check(lib().octo_fmm_interact(h, _stream(stream)), h)


def octo_fmm_downward(h, phi, g, stream=None) -> None:
    n, dev = _sizes(h)
    _check(lib().octo_fmm_downward(h, _buf(phi, n, dev, "phi"), _buf(g, 3 * n, dev, "g"), _stream(stream)), h)


def octo_fmm_forces(h, rho, phi, g, stream=None) -> None:
    n, dev = _sizes(h)
    _check(lib().octo_fmm_forces(h, _buf(rho, n, dev, "rho"), _buf(phi, n, dev, "phi"), _buf(g, 3 * n, dev, "g"),
                                 _stream(stream)), h)


def octo_fmm_forces_host(h, rho: np.ndarray, phi: np.ndarray, g: np.ndarray, stream=None) -> None:
    n, _ = _sizes(h)
    for name, a, k in (("rho", rho, n), ("phi", phi, n), ("g", g, 3 * n)):
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
            raise ValueError(f"{name}: host buffers must be contiguous float64 numpy arrays")
        if a.size != k:
            raise ValueError(f"{name}: expected {k} elements, got {a.size}")
    _check(lib().octo_fmm_forces_host(h, rho.ctypes.data, phi.ctypes.data, g.ctypes.data, _stream(stream)), h)


def octo_fmm_backward(h, dphi, dg, drho, stream=None) -> None:
    n, dev = _sizes(h)
    _check(lib().octo_fmm_backward(h, _buf(dphi, n, dev, "dphi"), _buf(dg, 3 * n, dev, "dg"),
                                   _buf(drho, n, dev, "drho"), _stream(stream)), h)


def octo_fmm_stats(h) -> np.ndarray:
    out = (ctypes.c_int64 * 4)()
    _check(lib().octo_fmm_stats(h, out), h)
    return np.array(out[:], dtype=np.int64)


def octo_fmm_read_state(h, which: int, n_nodes: int) -> np.ndarray:
    nf = 20 if which == 0 else 23
    out = np.empty((nf, n_nodes * 512), dtype=np.float64)
    _check(lib().octo_fmm_read_state(h, int(which), out.ctypes.data), h)
    return out


def octo_fmm_set_option(h, key: int, value: int) -> None:
    _check(lib().octo_fmm_set_option(h, int(key), int(value)), h)


def octo_fmm_subgrids_noalloc(n_subgrids: int, rho, h: float, phi, g, stream=None) -> None:
    """Allocation-free batch of single-subgrid solves (see include/octo_fmm.h).  The
    buffers must hold n_subgrids * 512 (g: 3 * n_subgrids * 512) float64 values on the
    current CUDA device."""
    import torch
    n = max(int(n_subgrids), 0) * 512
    dev = torch.cuda.current_device()
    _check(lib().octo_fmm_subgrids_noalloc(int(n_subgrids), _buf(rho, n, dev, "rho"), float(h),
                                           _buf(phi, n, dev, "phi"), _buf(g, 3 * n, dev, "g"), _stream(stream)))


def octo_fmm_measure_peak(fp64: bool, stream=None) -> float:
    """Measured float64 (fp64=True) or float32 fused multiply-add rate of the current
    device in flop/s."""
    v = ctypes.c_double()
    _check(lib().octo_fmm_measure_peak(1 if fp64 else 0, ctypes.byref(v), _stream(stream)))
    return float(v.value)


SCF_STATS = ("omega2", "c1", "c2", "max_change", "W", "T", "Pi", "virial_error")


def _scf_params(p: dict) -> ScfParams:
    return ScfParams(float(p["n"]), (ctypes.c_double * 2)(*[float(v) for v in p["rho_max"]]), float(p["rho_floor"]),
                     int(p["cell_a"]), int(p["cell_b"]), int(p["cell_c"]), float(p["x_split"]))


def octo_fmm_scf_step(h, params: dict, rho, phi, stream=None) -> np.ndarray:
    """One SCF step on the device: rho (overwritten) and its potential phi; returns the
    8 statistics named in SCF_STATS."""
    n, dev = _sizes(h)
    prm = _scf_params(params)
    st = (ctypes.c_double * 8)()
    _check(lib().octo_fmm_scf_step(h, ctypes.byref(prm), _buf(rho, n, dev, "rho"), _buf(phi, n, dev, "phi"), st,
                                   _stream(stream)), h)
    return np.array(st[:], dtype=np.float64)


def octo_fmm_scf_solve(h, params: dict, rho, max_iter: int, tol: float, stream=None) -> np.ndarray:
    """The SCF iteration on the device (rho: initial guess in, equilibrium out); returns
    the statistics of every step, [steps, 8]."""
    n, dev = _sizes(h)
    prm = _scf_params(params)
    hist = (ctypes.c_double * (8 * max(int(max_iter), 1)))()
    it = ctypes.c_int(0)
    _check(lib().octo_fmm_scf_solve(h, ctypes.byref(prm), _buf(rho, n, dev, "rho"), int(max_iter), float(tol), hist,
                                    ctypes.byref(it), _stream(stream)), h)
    return np.array(hist[:8 * it.value], dtype=np.float64).reshape(it.value, 8)


def octo_fmm_get_option(h, key: int) -> int:
    v = ctypes.c_int64()
    _check(lib().octo_fmm_get_option(h, int(key), ctypes.byref(v)), h)
    return int(v.value)


def octo_fmm_launches_per_solve(h) -> int:
    return int(lib().octo_fmm_launches_per_solve(h))


def octo_fmm_stage_count(h) -> int:
    return int(lib().octo_fmm_stage_count(h))


def octo_fmm_stage_info(h, i: int) -> dict:
    """name, pairs, cells, flops, flops64 (the float64 part), bytes of stage i."""
    name = ctypes.c_char_p()
    v = [ctypes.c_int64() for _ in range(5)]
    _check(lib().octo_fmm_stage_info(h, int(i), ctypes.byref(name), *[ctypes.byref(x) for x in v]), h)
    return {"name": name.value.decode(), "pairs": int(v[0].value), "cells": int(v[1].value),
            "flops": int(v[2].value), "flops64": int(v[3].value), "bytes": int(v[4].value)}


def octo_fmm_stage_times(h) -> np.ndarray:
    n = octo_fmm_stage_count(h)
    buf = (ctypes.c_float * max(n, 1))()
    rc = lib().octo_fmm_stage_times(h, buf, n)
    if rc < 0:
        _check(rc, h)
    return np.array(buf[:n], dtype=np.float64)


class OctoFMM:
    """Owning wrapper: one solver handle for one tree on the current CUDA device."""

    def __init__(self, tree, theta: float = 0.5, precision: int = OCTO_FP64, order: int = 3):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("OctoFMM needs a CUDA device")
        self.tree = tree
        self.n_leaf_cells = tree.n_leaf * 512
        self.handle = octo_fmm_create(tree, theta, order, precision)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            octo_fmm_destroy(h)
            self.handle = None

    def forces(self, rho, phi=None, g=None, stream=None):
        import torch
        if phi is None:
            phi = torch.empty(self.n_leaf_cells, dtype=torch.float64, device=rho.device)
        if g is None:
            g = torch.empty((3, self.n_leaf_cells), dtype=torch.float64, device=rho.device)
        octo_fmm_forces(self.handle, rho, phi, g, stream)
        return phi, g

    def counts(self) -> np.ndarray:
        return octo_fmm_stats(self.handle)
