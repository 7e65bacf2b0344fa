"""ctypes binding of libod (include/od.h).  Argument marshalling only: every
step of the solver runs in the CUDA library; there is no Python or CPU
fallback.  Loading fails loudly when libod.so has not been built."""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libod.so")

OD_OK, OD_EINVAL, OD_ENOMEM, OD_ECUDA, OD_ETIMEOUT, OD_EBUDGET, OD_ESTATE, OD_ENOTFOUND = range(8)
STATUS_NAMES = {0: "OD_OK", 1: "OD_EINVAL", 2: "OD_ENOMEM", 3: "OD_ECUDA", 4: "OD_ETIMEOUT",
                5: "OD_EBUDGET", 6: "OD_ESTATE", 7: "OD_ENOTFOUND"}
OD_PATH_PER_CHARE, OD_PATH_FUSED, OD_PATH_GRAPH, OD_PATH_PERSISTENT, OD_PATH_FUSED_GRAPH = range(5)
OD_STENCIL_3D7, OD_STENCIL_2D5 = 0, 1
PATHS = {"per_chare": OD_PATH_PER_CHARE, "fused": OD_PATH_FUSED, "graph": OD_PATH_GRAPH,
         "persistent": OD_PATH_PERSISTENT, "fused_graph": OD_PATH_FUSED_GRAPH}

_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_vp = ctypes.c_void_p


class od_config(ctypes.Structure):
    _fields_ = [
        ("nx", _i64), ("ny", _i64), ("nz", _i64),
        ("px", _i32), ("py", _i32), ("pz", _i32),
        ("cuts_x", ctypes.POINTER(_i32)), ("cuts_y", ctypes.POINTER(_i32)), ("cuts_z", ctypes.POINTER(_i32)),
        ("ncuts_x", _i32), ("ncuts_y", _i32), ("ncuts_z", _i32),
        ("seed", _u64),
        ("init_mode", _i32), ("path", _i32), ("autotune", _i32),
        ("tile_y", _i32), ("tile_z", _i32), ("threads", _i32), ("cells_per_thread", _i32),
        ("stages", _i32), ("arith", _i32), ("order", _i32), ("stream_pool", _i32), ("device", _i32),
        ("stream", _vp), ("arena", _vp), ("arena_bytes", _u64), ("spin_limit_ns", _u64),
        ("stencil", _i32), ("pe_threads", _i32),
        ("gnx", _i64), ("gny", _i64), ("gnz", _i64), ("gx0", _i64), ("gy0", _i64), ("gz0", _i64),
    ]


class od_plan_info(ctypes.Structure):
    _fields_ = [
        ("nchares", _i64), ("ntiles", _i64), ("cells", _i64),
        ("face_cells_internal", _i64), ("face_cells_dirichlet", _i64),
        ("arena_bytes", _u64), ("bytes_per_step", ctypes.c_double),
        ("tile_y", _i32), ("tile_z", _i32), ("threads", _i32), ("cells_per_thread", _i32),
        ("stages", _i32), ("arith", _i32), ("smem_bytes", _i32),
    ]


class od_stats(ctypes.Structure):
    _fields_ = [
        ("steps_done", _i64), ("kernel_launches", _i64), ("api_calls", _i64), ("graph_launches", _i64),
        ("path", _i32), ("persistent_grid", _i32), ("tuned", _i32), ("tune_ms_per_step", ctypes.c_double),
        ("plan", od_plan_info),
    ]


class od_server_config(ctypes.Structure):
    _fields_ = [
        ("hbm_budget_bytes", _u64), ("max_active", _i32), ("max_jobs_per_launch", _i32), ("device", _i32),
        ("threads", _i32), ("cells_per_thread", _i32), ("stages", _i32), ("arith", _i32), ("pool", _vp),
        ("batch_steps", _i32), ("job_streams", _i32),
    ]


class od_job_info(ctypes.Structure):
    _fields_ = [
        ("state", _i32), ("iters", _i32), ("cells", _i64), ("arena_bytes", _u64),
        ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
    ]


class od_server_stats_t(ctypes.Structure):
    _fields_ = [
        ("queued", _i64), ("running", _i64), ("done", _i64), ("failed", _i64), ("launches", _i64),
        ("updates_done", ctypes.c_double), ("pool_used", _u64), ("pool_peak", _u64), ("seconds", ctypes.c_double),
        ("admit_seconds", ctypes.c_double), ("busy_seconds", ctypes.c_double),
    ]


OD_JOB_QUEUED, OD_JOB_RUNNING, OD_JOB_DONE, OD_JOB_FAILED = range(4)


class ODError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

# name -> (restype, argtypes); the exported C ABI, in header order
SIGNATURES = {
    "od_config_default": (None, [ctypes.POINTER(od_config)]),
    "od_plan": (_i32, [ctypes.POINTER(od_config), ctypes.POINTER(od_plan_info)]),
    "od_decompose": (_i32, [ctypes.POINTER(od_config), ctypes.POINTER(_i64), ctypes.POINTER(_i32), _i64]),
    "od_plan_tiles": (_i32, [ctypes.POINTER(od_config), _vp, _i64, _vp, _vp, _i64, ctypes.POINTER(_i64),
                             ctypes.POINTER(_i64)]),
    "od_create": (_i32, [ctypes.POINTER(_vp), ctypes.POINTER(od_config)]),
    "od_step": (_i32, [_vp, _i32]),
    "od_set_path": (_i32, [_vp, _i32]),
    "od_sync": (_i32, [_vp]),
    "od_read": (_i32, [_vp, _vp, _i32]),
    "od_write": (_i32, [_vp, _vp, _i32]),
    "od_stats_get": (_i32, [_vp, ctypes.POINTER(od_stats)]),
    "od_debug_stall_tile": (_i32, [_vp, _i64]),
    "od_arith_host": (_i32, [_i32, _vp, _vp, _vp, _i64]),
    "od_arith_device": (_i32, [_i32, _vp, _vp, _vp, _i64]),
    "od_server_config_default": (None, [ctypes.POINTER(od_server_config)]),
    "od_server_create": (_i32, [ctypes.POINTER(_vp), ctypes.POINTER(od_server_config)]),
    "od_server_submit": (_i32, [_vp, ctypes.POINTER(od_config), _i32, ctypes.POINTER(_u64)]),
    "od_server_wait": (_i32, [_vp, _u64, ctypes.c_double, ctypes.POINTER(_i32)]),
    "od_server_next_completion": (_i32, [_vp, ctypes.c_double, ctypes.POINTER(_u64)]),
    "od_server_job_info": (_i32, [_vp, _u64, ctypes.POINTER(od_job_info)]),
    "od_server_fetch": (_i32, [_vp, _u64, _vp, _i32]),
    "od_server_release": (_i32, [_vp, _u64]),
    "od_server_stats": (_i32, [_vp, ctypes.POINTER(od_server_stats_t)]),
    "od_server_destroy": (_i32, [_vp]),
    "od_submit": (_i32, [_vp, ctypes.POINTER(od_config), _i32, ctypes.POINTER(_u64)]),
    "od_poll": (_i32, [_vp, _u64, ctypes.POINTER(_i32)]),
    "od_fetch": (_i32, [_vp, _u64, _vp, _i32]),
    "od_jacobi_noalloc": (_i32, [_vp, _vp, _i64, _i64, _i64, _i32, _vp]),
    "od_bench_launch_latency": (_i32, [_i32, _i32, _i32, ctypes.POINTER(ctypes.c_double)]),
    "od_bench_release": (_i32, [_i32, _i64, _i32, _i32, _vp, ctypes.POINTER(ctypes.c_double)]),
    "od_bench_launch_rate": (_i32, [_i32, _i32, _i32, _i32, ctypes.POINTER(ctypes.c_double)]),
    "od_face_copy": (_i32, [_vp, _i32, _i32, _vp, _i32]),
    "od_read_cells": (_i32, [_vp, _vp, _i64, _vp]),
    "od_write_async": (_i32, [_vp, _vp]),
    "od_read_async": (_i32, [_vp, _vp]),
    "od_comm_create": (_i32, [ctypes.POINTER(_vp), _i32, _u64, _i32]),
    "od_comm_handles": (_i32, [_vp, _vp, _u64]),
    "od_comm_open": (_i32, [ctypes.POINTER(_vp), _i32, _vp, _u64]),
    "od_comm_buffer": (_i32, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_u64), ctypes.POINTER(_i32)]),
    "od_comm_record": (_i32, [_vp, _i32, _vp]),
    "od_comm_wait": (_i32, [_vp, _i32, _vp]),
    "od_comm_destroy": (_i32, [_vp]),
    "od_destroy": (_i32, [_vp]),
    "od_last_error": (ctypes.c_char_p, []),
    "od_version": (ctypes.c_char_p, []),
}


def lib() -> ctypes.CDLL:
    """Load libod.so (built in-tree by paper_2605_12734_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libod.so is not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'` first")
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(status: int, where: str) -> None:
    if status != OD_OK:
        raise ODError(status, where, lib().od_last_error().decode(errors="replace"))
