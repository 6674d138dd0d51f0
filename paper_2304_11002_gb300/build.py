"""Builds the solver's shared library in-tree: paper_2304_11002_gb300/_lib/liboctofmm.so.

nvcc for sm_103a only (GB300), one translation unit per file compiled in
parallel, linked against the shared CUDA runtime.  Host code is portable C++17
(the library is rebuilt on each machine that runs it: x86_64 here, aarch64 on
Grace hosts).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_lib", "obj")
LIB = os.path.join(HERE, "_lib", "liboctofmm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["capi.cu", "kernels_fp64.cu", "kernels_adjoint.cu", "kernels_boundary.cu", "noalloc.cu",
              "kernels_interact.cu", "kernels_interact_b64.cu", "peak.cu", "scf.cu"]
CXX_SOURCES = ["plan.cpp", "tables.cpp"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return [os.path.join(CSRC, f) for f in CU_SOURCES + CXX_SOURCES]


def _deps():
    out = _sources()
    for f in os.listdir(CSRC):
        if f.endswith((".h", ".cuh")):
            out.append(os.path.join(CSRC, f))
    out.append(os.path.join(INC, "octo_fmm.h"))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    common = ["-O3", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC", "-I", INC]
    jobs = []
    for f in CU_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        cmd = [nv, *ARCH, "-lineinfo", *common, "-c", os.path.join(CSRC, f), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((cmd, obj))
    for f in CXX_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        jobs.append((["g++", "-O2", "-std=c++17", "-fPIC", "-I", INC, "-c", os.path.join(CSRC, f), "-o", obj], obj))

    def run(job):
        cmd, _ = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or ptxas_info or r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}")
        return r

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        list(ex.map(run, jobs))
    tmp = LIB + ".tmp"
    link = [nv, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *[o for _, o in jobs],
            "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link failed")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
