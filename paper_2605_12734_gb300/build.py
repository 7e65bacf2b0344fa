"""Build libod.so (the CUDA library behind include/od.h) in place.

Every translation unit is compiled for sm_103a only
(``-gencode arch=compute_103a,code=sm_103a``); the tile kernels are compiled
with ``-fmad=false`` (and use explicit round-to-nearest adds and division)
so no multiply-add contraction can change the Jacobi update's bits.  The
units compile in parallel; nothing here needs a GPU.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libod.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden", "-I", INCLUDE, "-I", CSRC]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-fvisibility=hidden", "-I", INCLUDE, "-I", CSRC]

SOURCES = ["od_kernels.cu", "od_api.cu", "od_plan.cpp", "od_noalloc.cu", "od_serve.cu", "od_launch.cu",
           "od_comm.cu"]
# the tile kernels, compiled once per arithmetic mode (-DOD_AMODE=m)
TILE_SOURCE = "od_tiles.cu"
AMODES = range(16)
# the 2D 5-point kernels (-DOD_STENCIL=1): modes 4..6 coincide there (three adds)
AMODES_2D = (0, 1, 2, 3, 4, 7, 8, 9, 10, 11, 12, 13, 14, 15)
HEADERS = ["od_internal.h", "od_kernels.h", "od_plan.h", "od_tile.cuh", "od_arith.cuh", "od_ctx.h"]


def _nvcc() -> str:
    cand = [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]
    for c in cand:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libod")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile (if needed) and return the path of libod.so."""
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "od.h")]
    srcs = [os.path.join(CSRC, s) for s in SOURCES + [TILE_SOURCE]]
    if not force and not ptxas_info and not _stale(LIB, srcs + hdrs + [__file__]):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    # tuning overrides for experiments, e.g. OD_NVCC_EXTRA="-DOD_MIN_THREADS_PER_SM=1280"
    EXTRA = os.environ.get("OD_NVCC_EXTRA", "").split()
    procs, objs = [], []
    units = [(os.path.join(CSRC, s), [], os.path.basename(s)) for s in SOURCES]
    units += [(os.path.join(CSRC, TILE_SOURCE), [f"-DOD_AMODE={m}"], f"od_tiles_am{m}")
              for m in AMODES]
    units += [(os.path.join(CSRC, TILE_SOURCE), [f"-DOD_AMODE={m}", "-DOD_STENCIL=1"], f"od_tiles2d_am{m}")
              for m in AMODES_2D]
    for src, defs, stem in units:
        obj = os.path.join(BUILD, stem + ".o")
        objs.append(obj)
        if src.endswith(".cu"):
            cmd = [nvcc, *ARCH, *NVCC_FLAGS, *defs, *EXTRA, "-c", src, "-o", obj]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
        else:
            cxx = os.environ.get("CXX", "g++")
            cmd = [cxx, *CXX_FLAGS, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    errors = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(" ".join(cmd) + "\n" + out)
        elif out and (verbose or ptxas_info):
            print(out, file=sys.stderr)
    if errors:
        raise RuntimeError("libod build failed:\n" + "\n".join(errors))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", tmp]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
