"""CPU oracle for the overdecomposed 3D 7-point FP64 Jacobi sweep.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_2605_12734_gb300``) never imports it, and it never imports the product.

The arithmetic lives in ``jacobi_oracle.c`` (plain C, ``-O2 -ffp-contract=off``,
no fast-math, OpenMP only to split z-planes of the monolithic sweep).  This
module builds that file into ``liboracle.so`` next to it and wraps it with
ctypes and NumPy arrays.  Every function follows the paper's Jacobi proxy
(Sec. V, "jacobi2d": Jacobi iteration on a block-decomposed grid with halo
exchange, fixed iteration count, no convergence check) in 3D with the readings
listed in the C file's header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jacobi_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_I64 = ctypes.c_int64
_DP = ctypes.POINTER(ctypes.c_double)
_I64P = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile jacobi_oracle.c into liboracle.so (in place).  gcc only."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    lib.oracle_splitmix64.restype = ctypes.c_uint64
    lib.oracle_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    lib.oracle_uniform.restype = ctypes.c_double
    lib.oracle_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    lib.oracle_init_padded.restype = None
    lib.oracle_init_padded.argtypes = [_I64, _I64, _I64, ctypes.c_uint64, ctypes.c_int, _DP]
    lib.oracle_sweep.restype = ctypes.c_int
    lib.oracle_sweep.argtypes = [_I64, _I64, _I64, _DP, ctypes.c_int, ctypes.c_int]
    lib.oracle_interior.restype = None
    lib.oracle_interior.argtypes = [_I64, _I64, _I64, _DP, _DP]
    lib.oracle_split.restype = ctypes.c_int
    lib.oracle_split.argtypes = [_I64, ctypes.c_int, _I64P]
    lib.oracle_sweep_decomposed.restype = ctypes.c_int
    lib.oracle_sweep_decomposed.argtypes = [_I64, _I64, _I64, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, _I64P, _I64P, _I64P, _DP, ctypes.c_int]
    lib.oracle_point.restype = ctypes.c_int
    lib.oracle_point.argtypes = [_I64, _I64, _I64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                 _I64, _I64, _I64, _DP]
    lib.oracle_max_threads.restype = ctypes.c_int
    lib.oracle_max_threads.argtypes = []
    lib.oracle2d_init_padded.restype = None
    lib.oracle2d_init_padded.argtypes = [_I64, _I64, ctypes.c_uint64, ctypes.c_int, _DP]
    lib.oracle2d_sweep.restype = ctypes.c_int
    lib.oracle2d_sweep.argtypes = [_I64, _I64, _DP, ctypes.c_int, ctypes.c_int]
    lib.oracle2d_sweep_decomposed.restype = ctypes.c_int
    lib.oracle2d_sweep_decomposed.argtypes = [_I64, _I64, ctypes.c_int, ctypes.c_int, _I64P, _I64P, _DP,
                                              ctypes.c_int]
    lib.oracle2d_point.restype = ctypes.c_int
    lib.oracle2d_point.argtypes = [_I64, _I64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _I64, _I64, _DP]
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


def _ip(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_I64P)


def splitmix64(seed: int, index: int) -> int:
    """Output number index+1 of a SplitMix64 stream seeded with ``seed``."""
    return int(_load().oracle_splitmix64(seed & (2**64 - 1), index))


def uniform(seed: int, index: int) -> float:
    return float(_load().oracle_uniform(seed & (2**64 - 1), index))


def init_padded(nx: int, ny: int, nz: int, seed: int, init_mode: int) -> np.ndarray:
    """Padded global initial field, shape (nz+2, ny+2, nx+2)."""
    P = np.empty((nz + 2, ny + 2, nx + 2), dtype=np.float64)
    _load().oracle_init_padded(nx, ny, nz, seed & (2**64 - 1), init_mode, _dp(P))
    return P


def interior(P: np.ndarray) -> np.ndarray:
    """Interior of a padded array as a flat x-fastest vector (nx*ny*nz)."""
    nz, ny, nx = (d - 2 for d in P.shape)
    out = np.empty(nx * ny * nz, dtype=np.float64)
    _load().oracle_interior(nx, ny, nz, _dp(np.ascontiguousarray(P)), _dp(out))
    return out


def sweep(P: np.ndarray, iters: int, threads: int = 1) -> np.ndarray:
    """Monolithic Jacobi sweep of a padded array; returns a new padded array."""
    Q = np.array(P, dtype=np.float64, copy=True, order="C")
    nz, ny, nx = (d - 2 for d in Q.shape)
    rc = _load().oracle_sweep(nx, ny, nz, _dp(Q), iters, threads)
    if rc != 0:
        raise MemoryError("oracle_sweep failed")
    return Q


def split(n: int, p: int) -> np.ndarray:
    """Balanced split edges (p+1 values) of n cells into p blocks."""
    e = np.empty(p + 1, dtype=np.int64)
    if _load().oracle_split(n, p, _ip(e)) != 0:
        raise ValueError(f"cannot split {n} cells into {p} blocks")
    return e


def sweep_decomposed(P: np.ndarray, ex, ey, ez, iters: int) -> np.ndarray:
    """Block-decomposed sweep with explicit halo copies; returns padded array."""
    Q = np.array(P, dtype=np.float64, copy=True, order="C")
    nz, ny, nx = (d - 2 for d in Q.shape)
    ex = np.ascontiguousarray(ex, dtype=np.int64)
    ey = np.ascontiguousarray(ey, dtype=np.int64)
    ez = np.ascontiguousarray(ez, dtype=np.int64)
    if ex[0] != 0 or ex[-1] != nx or ey[0] != 0 or ey[-1] != ny or ez[0] != 0 or ez[-1] != nz:
        raise ValueError("cut lists must run from 0 to the interior extent")
    rc = _load().oracle_sweep_decomposed(nx, ny, nz, len(ex) - 1, len(ey) - 1, len(ez) - 1,
                                         _ip(ex), _ip(ey), _ip(ez), _dp(Q), iters)
    if rc != 0:
        raise ValueError(f"oracle_sweep_decomposed failed ({rc})")
    return Q


def point(nx: int, ny: int, nz: int, seed: int, init_mode: int, iters: int,
          x: int, y: int, z: int) -> float:
    """u^iters at interior cell (x, y, z) of the seeded field, via its cone."""
    out = ctypes.c_double()
    rc = _load().oracle_point(nx, ny, nz, seed & (2**64 - 1), init_mode, iters, x, y, z,
                              ctypes.byref(out))
    if rc != 0:
        raise ValueError("oracle_point failed")
    return out.value


def solve(nx: int, ny: int, nz: int, seed: int, init_mode: int, iters: int,
          threads: int = 1) -> np.ndarray:
    """Interior (x fastest) of u^iters for the seeded field: the reference answer
    every decomposition and execution path must reproduce bit for bit."""
    return interior(sweep(init_padded(nx, ny, nz, seed, init_mode), iters, threads))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


# ------------------------------------------------------------------ 2D (5-point)

def init_padded_2d(nx: int, ny: int, seed: int, init_mode: int) -> np.ndarray:
    """Padded 2D initial field, shape (ny+2, nx+2)."""
    P = np.empty((ny + 2, nx + 2), dtype=np.float64)
    _load().oracle2d_init_padded(nx, ny, seed & (2**64 - 1), init_mode, _dp(P))
    return P


def sweep_2d(P: np.ndarray, iters: int, threads: int = 1) -> np.ndarray:
    Q = np.array(P, dtype=np.float64, copy=True, order="C")
    ny, nx = (d - 2 for d in Q.shape)
    if _load().oracle2d_sweep(nx, ny, _dp(Q), iters, threads) != 0:
        raise MemoryError("oracle2d_sweep failed")
    return Q


def sweep_decomposed_2d(P: np.ndarray, ex, ey, iters: int) -> np.ndarray:
    Q = np.array(P, dtype=np.float64, copy=True, order="C")
    ny, nx = (d - 2 for d in Q.shape)
    ex = np.ascontiguousarray(ex, dtype=np.int64)
    ey = np.ascontiguousarray(ey, dtype=np.int64)
    if ex[0] != 0 or ex[-1] != nx or ey[0] != 0 or ey[-1] != ny:
        raise ValueError("cut lists must run from 0 to the interior extent")
    rc = _load().oracle2d_sweep_decomposed(nx, ny, len(ex) - 1, len(ey) - 1, _ip(ex), _ip(ey), _dp(Q), iters)
    if rc != 0:
        raise ValueError(f"oracle2d_sweep_decomposed failed ({rc})")
    return Q


def point_2d(nx: int, ny: int, seed: int, init_mode: int, iters: int, x: int, y: int) -> float:
    out = ctypes.c_double()
    if _load().oracle2d_point(nx, ny, seed & (2**64 - 1), init_mode, iters, x, y, ctypes.byref(out)) != 0:
        raise ValueError("oracle2d_point failed")
    return out.value


def solve_2d(nx: int, ny: int, seed: int, init_mode: int, iters: int, threads: int = 1) -> np.ndarray:
    """Interior (x fastest) of the 2D field after `iters` Jacobi steps."""
    Q = sweep_2d(init_padded_2d(nx, ny, seed, init_mode), iters, threads)
    return np.ascontiguousarray(Q[1:-1, 1:-1]).ravel()
