"""paper_2605_12734_gb300 -- overdecomposed 3D 7-point FP64 Jacobi on one GB300.

The solver is the C-ABI library libod.so (include/od.h, CUDA for sm_103a);
this package is its thin Python binding (same entry points, argument
marshalling only) plus the seeded workload generators in ``inputs``.
PyTorch, when present, only provides device memory (the chare arena, device
result tensors) and streams.

    from paper_2605_12734_gb300 import Jacobi3D
    s = Jacobi3D(512, 512, 512, split=(16, 16, 16), path="persistent", seed=2)
    s.step(100)
    u = s.read()          # numpy (nx*ny*nz,) x-fastest, bit-identical to the
                          # undecomposed sweep
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import ODError, PATHS, check, lib, od_config, od_plan_info, od_stats

STENCILS = {"3d7": 0, "2d5": 1}

__all__ = ["Jacobi3D", "Jacobi2D", "Server", "STENCILS", "ODError", "PATHS", "make_config", "plan", "decompose", "lib", "arith_host",
           "arith_device", "jacobi_noalloc", "plan_2d", "decompose_2d", "bench_launch_latency", "bench_release",
           "bench_launch_rate", "Comm"]


def _cuts_array(cuts):
    if cuts is None:
        return None, 0
    arr = (ctypes.c_int32 * len(cuts))(*[int(v) for v in cuts])
    return arr, len(cuts) - 1


def make_config(nx: int, ny: int, nz: int, *, split=(1, 1, 1), cuts=None, seed: int = 1,
                init_mode: int = 1, path: str | int = "fused", autotune: bool = False,
                tile_y: int = 0, tile_z: int = 0, threads: int = 0, cells_per_thread: int = 0,
                stages: int = 0, arith: int = -1, order: int = 0, stream_pool: int = 0, device: int = 0,
                stream: int | None = None, arena: int | None = None, arena_bytes: int = 0,
                spin_limit_ns: int = 0, stencil: str | int = "3d7", gdims=None, goff=None,
                pe_threads: int = 0):
    """Build an od_config (returns (config, keepalive) -- keep both alive while
    the config is used, the cut arrays are referenced by pointer).  For the
    2D stencil ("2d5") nz is 1 and split / cuts may give two axes."""
    cfg = od_config()
    lib().od_config_default(ctypes.byref(cfg))
    cfg.nx, cfg.ny, cfg.nz = int(nx), int(ny), int(nz)
    split = tuple(split) + (1,) * (3 - len(split))
    if cuts is not None:
        cuts = tuple(cuts) + (None,) * (3 - len(cuts))
    cfg.px, cfg.py, cfg.pz = (int(v) for v in split)
    cfg.stencil = STENCILS[stencil] if isinstance(stencil, str) else int(stencil)
    cfg.pe_threads = int(pe_threads)
    if gdims is not None:  # a shard: this context is a sub-box of the global grid gdims at offset goff
        g = tuple(int(v) for v in gdims) + (1,) * (3 - len(gdims))
        o = tuple(int(v) for v in (goff or ())) + (0,) * (3 - len(goff or ()))
        cfg.gnx, cfg.gny, cfg.gnz = g
        cfg.gx0, cfg.gy0, cfg.gz0 = o
    keep = []
    if cuts is not None:
        for axis, cl in zip("xyz", cuts):
            arr, n = _cuts_array(cl)
            keep.append(arr)
            if arr is not None:
                setattr(cfg, f"cuts_{axis}", ctypes.cast(arr, ctypes.POINTER(ctypes.c_int32)))
                setattr(cfg, f"ncuts_{axis}", n)
    cfg.seed = int(seed) & (2**64 - 1)
    cfg.init_mode = int(init_mode)
    cfg.path = PATHS[path] if isinstance(path, str) else int(path)
    cfg.autotune = int(bool(autotune))
    cfg.tile_y, cfg.tile_z, cfg.threads = int(tile_y), int(tile_z), int(threads)
    cfg.cells_per_thread, cfg.stages, cfg.order = int(cells_per_thread), int(stages), int(order)
    cfg.arith = int(arith)
    cfg.stream_pool, cfg.device = int(stream_pool), int(device)
    cfg.stream = stream
    cfg.arena = arena
    cfg.arena_bytes = int(arena_bytes)
    cfg.spin_limit_ns = int(spin_limit_ns)
    return cfg, keep


def plan(nx, ny, nz, **kw) -> dict:
    """Host-only decomposition summary (no GPU needed)."""
    cfg, keep = make_config(nx, ny, nz, **kw)
    info = od_plan_info()
    check(lib().od_plan(ctypes.byref(cfg), ctypes.byref(info)), "od_plan")
    return {f: getattr(info, f) for f, _ in od_plan_info._fields_}


def decompose(nx, ny, nz, **kw):
    """Chare boxes (n,6: x0,bx,y0,by,z0,bz) and neighbours (n,6), host-only."""
    cfg, keep = make_config(nx, ny, nz, **kw)
    n = plan(nx, ny, nz, **kw)["nchares"]
    box = np.zeros((n, 6), dtype=np.int64)
    nbr = np.zeros((n, 6), dtype=np.int32)
    check(lib().od_decompose(ctypes.byref(cfg), box.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                             nbr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n), "od_decompose")
    return box, nbr


def plan_tiles(nx, ny, nz, **kw):
    """The persistent schedule, host-only: tiles (n, 7: chare, x0, nx, y0, ny,
    z0, nz) and the dependency CSR (dep_ptr, dep_idx)."""
    cfg, keep = make_config(nx, ny, nz, **kw)
    nt, nd = ctypes.c_int64(), ctypes.c_int64()
    check(lib().od_plan_tiles(ctypes.byref(cfg), None, 0, None, None, 0, ctypes.byref(nt), ctypes.byref(nd)),
          "od_plan_tiles")
    tiles = np.zeros((nt.value, 8), dtype=np.int64)
    ptr = np.zeros(nt.value + 1, dtype=np.int32)
    idx = np.zeros(max(nd.value, 1), dtype=np.int32)
    check(lib().od_plan_tiles(ctypes.byref(cfg), tiles.ctypes.data, nt.value, ptr.ctypes.data, idx.ctypes.data,
                              nd.value, ctypes.byref(nt), ctypes.byref(nd)), "od_plan_tiles")
    return tiles[:, :7], ptr, idx[:nd.value]


def _operands(op: int) -> int:
    """Operands per element of a self-test op (see od_arith_host)."""
    if 10 <= op < 20 or 30 <= op < 40:
        return 6
    if 20 <= op < 30 or op >= 40:
        return 4
    return 1


def arith_host(op: int, a: np.ndarray, b: np.ndarray | None = None) -> np.ndarray:
    """Run the kernels' exact integer-pipe arithmetic on the host: op 0
    a/6, op 1 a+b, op 10+m the 3D Jacobi update in arithmetic mode m over six
    operands per element, op 20+m the 2D update over four; op 30+f / 40+f the
    3D / 2D update in the anchored window with f adds on the FP64 pipe, b[0]
    holding the anchor exponent (float64 arrays)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = a if b is None else np.ascontiguousarray(b, dtype=np.float64)
    n = a.size // _operands(op)
    out = np.empty(n, dtype=np.float64)
    check(lib().od_arith_host(int(op), a.ctypes.data, b.ctypes.data, out.ctypes.data, n), "od_arith_host")
    return out


def arith_device(op: int, a, b=None):
    """Same on the device (torch CUDA float64 tensors); ops 2/3 use the FP64
    pipe's IEEE division / add."""
    import torch
    b = a if b is None else b
    n = a.numel() // _operands(op)
    out = torch.empty(n, dtype=torch.float64, device=a.device)
    check(lib().od_arith_device(int(op), a.data_ptr(), b.data_ptr(), out.data_ptr(), n), "od_arith_device")
    return out


def jacobi_noalloc(u_in, u_out, nx: int, ny: int, nz: int, iters: int, stream: int | None = None) -> None:
    """Iterate a caller-owned padded field (device tensors of (nx+2)(ny+2)(nz+2)
    float64) without any device allocation; see od_jacobi_noalloc in od.h."""
    check(lib().od_jacobi_noalloc(u_in.data_ptr(), u_out.data_ptr(), int(nx), int(ny), int(nz), int(iters),
                                  stream), "od_jacobi_noalloc")


def bench_launch_latency(wait: str | int = "sync", reps: int = 2000, device: int = 0) -> float:
    """Mean microseconds per launch-and-wait round trip of an empty kernel
    (wait: "sync" | "event" | "callback"); see od_bench_launch_latency."""
    w = {"sync": 0, "event": 1, "callback": 2}[wait] if isinstance(wait, str) else int(wait)
    us = ctypes.c_double()
    check(lib().od_bench_launch_latency(int(device), w, int(reps), ctypes.byref(us)), "od_bench_launch_latency")
    return us.value


def bench_release(total_threads: int, nkernels: int, work: int = 256, out=None, device: int = 0) -> float:
    """Microseconds from the release of `nkernels` pre-enqueued kernels (one
    stream each, held by cuStreamWaitValue32 on a host flag) to the end of the
    last; out: optional CUDA uint32/int32 tensor of total_threads results."""
    us = ctypes.c_double()
    ptr = None if out is None else out.data_ptr()
    check(lib().od_bench_release(int(device), int(total_threads), int(nkernels), int(work), ptr, ctypes.byref(us)),
          "od_bench_release")
    return us.value


def bench_launch_rate(host_threads: int, chares: int, kernels: int = 2000, device: int = 0) -> float:
    """Kernels per second fired by `host_threads` threads driving `chares`
    chares each (next kernel once the previous one completed)."""
    r = ctypes.c_double()
    check(lib().od_bench_launch_rate(int(device), int(host_threads), int(chares), int(kernels), ctypes.byref(r)),
          "od_bench_launch_rate")
    return r.value


class Jacobi3D:
    """One overdecomposed solve resident on a GPU (wraps an od_ctx)."""

    def __init__(self, nx: int, ny: int, nz: int, *, torch_arena: bool = True, **kw):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self._arena_tensor = None
        if torch_arena and kw.get("arena") is None:
            try:
                import torch
                if torch.cuda.is_available():
                    need = plan(nx, ny, nz, **kw)["arena_bytes"]
                    if kw.get("autotune"):  # other tilings need larger tables
                        need = need + need // 16 + (64 << 20)
                    dev = kw.get("device", 0)
                    self._arena_tensor = torch.empty(need + 256, dtype=torch.uint8, device=f"cuda:{dev}")
                    base = self._arena_tensor.data_ptr()
                    kw["arena"] = (base + 255) // 256 * 256
                    kw["arena_bytes"] = need
            except ImportError:
                pass
        self._cfg, self._keep = make_config(nx, ny, nz, **kw)
        h = ctypes.c_void_p()
        check(lib().od_create(ctypes.byref(h), ctypes.byref(self._cfg)), "od_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def step(self, iters: int) -> None:
        check(lib().od_step(self._h, int(iters)), "od_step")

    def set_path(self, path: str | int) -> None:
        check(lib().od_set_path(self._h, PATHS[path] if isinstance(path, str) else int(path)), "od_set_path")

    def sync(self) -> None:
        check(lib().od_sync(self._h), "od_sync")

    def read(self, out=None):
        """Current field, interior x-fastest.  out: None (new numpy array), a
        numpy float64 array, or a CUDA torch float64 tensor (device copy)."""
        if out is None:
            out = np.empty(self.cells, dtype=np.float64)
        if isinstance(out, np.ndarray):
            assert out.dtype == np.float64 and out.size == self.cells and out.flags["C_CONTIGUOUS"]
            check(lib().od_read(self._h, out.ctypes.data, 0), "od_read")
            return out
        assert out.is_cuda and out.numel() == self.cells and out.is_contiguous()
        check(lib().od_read(self._h, out.data_ptr(), 1), "od_read")
        return out

    def read_cells(self, cells) -> np.ndarray:
        """Values of the current field at the given global interior indices
        (x fastest), without reading the whole grid."""
        idx = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.empty(idx.size, dtype=np.float64)
        check(lib().od_read_cells(self._h, idx.ctypes.data, idx.size, out.ctypes.data), "od_read_cells")
        return out

    def write(self, src) -> None:
        if isinstance(src, np.ndarray):
            src = np.ascontiguousarray(src, dtype=np.float64)
            assert src.size == self.cells
            check(lib().od_write(self._h, src.ctypes.data, 0), "od_write")
        else:
            assert src.is_cuda and src.numel() == self.cells and src.is_contiguous()
            check(lib().od_write(self._h, src.data_ptr(), 1), "od_write")

    @staticmethod
    def _host_ptr(buf, n):
        if isinstance(buf, np.ndarray):
            assert buf.dtype == np.float64 and buf.size == n and buf.flags["C_CONTIGUOUS"]
            return buf.ctypes.data
        assert not buf.is_cuda and buf.is_pinned() and buf.numel() == n and buf.is_contiguous()
        return buf.data_ptr()

    def write_async(self, src) -> None:
        """Enqueue the import of a pinned host field (a pinned torch tensor or
        a numpy view of one); src must stay untouched until sync()."""
        check(lib().od_write_async(self._h, self._host_ptr(src, self.cells)), "od_write_async")

    def read_async(self, out) -> None:
        """Enqueue the export of the current field into pinned host memory;
        out is valid after sync()."""
        check(lib().od_read_async(self._h, self._host_ptr(out, self.cells)), "od_read_async")

    def face_copy(self, face: int, direction: int, buf) -> None:
        """Export (direction 0) the boundary layer on domain face `face` into
        buf, or import (1) buf into its ghost layer; buf: a device pointer
        (int), a CUDA float64 tensor, or a numpy float64 array (host)."""
        if isinstance(buf, np.ndarray):
            assert buf.dtype == np.float64 and buf.flags["C_CONTIGUOUS"]
            ptr, dev = buf.ctypes.data, 0
        elif isinstance(buf, int):
            ptr, dev = buf, 1
        else:
            assert buf.is_cuda and buf.dtype.itemsize == 8 and buf.is_contiguous()
            ptr, dev = buf.data_ptr(), 1
        check(lib().od_face_copy(self._h, int(face), int(direction), ptr, dev), "od_face_copy")

    def stats(self) -> dict:
        st = od_stats()
        check(lib().od_stats_get(self._h, ctypes.byref(st)), "od_stats_get")
        d = {f: getattr(st, f) for f, _ in od_stats._fields_ if f != "plan"}
        d["plan"] = {f: getattr(st.plan, f) for f, _ in od_plan_info._fields_}
        return d

    def stall_tile(self, tile: int) -> None:
        check(lib().od_debug_stall_tile(self._h, int(tile)), "od_debug_stall_tile")

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().od_destroy(self._h)
            self._h = ctypes.c_void_p()
        self._arena_tensor = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Jacobi2D(Jacobi3D):
    """The 2D 5-point Jacobi (the paper's own application) on an nx x ny grid
    split into px x py chares; read/write move nx*ny doubles, x fastest."""

    def __init__(self, nx: int, ny: int, *, torch_arena: bool = True, **kw):
        kw["stencil"] = "2d5"
        super().__init__(nx, ny, 1, torch_arena=torch_arena, **kw)


def plan_2d(nx, ny, **kw) -> dict:
    return plan(nx, ny, 1, stencil="2d5", **kw)


def decompose_2d(nx, ny, **kw):
    """2D chare boxes (n,4: x0,bx,y0,by) and neighbours (n,4: x-,x+,y-,y+)."""
    box, nbr = decompose(nx, ny, 1, stencil="2d5", **kw)
    return box[:, :4].copy(), nbr[:, :4].copy()


class Comm:
    """A communication endpoint (od_comm_*): a device buffer and a pool of
    interprocess events, created here or mapped from a peer's handles."""

    def __init__(self, handle):
        self._h = handle
        buf, nbytes, nev = ctypes.c_void_p(), ctypes.c_uint64(), ctypes.c_int32()
        check(lib().od_comm_buffer(self._h, ctypes.byref(buf), ctypes.byref(nbytes), ctypes.byref(nev)),
              "od_comm_buffer")
        self.ptr, self.nbytes, self.nevents = buf.value, nbytes.value, nev.value

    @classmethod
    def create(cls, nbytes: int, nevents: int, device: int = 0) -> "Comm":
        h = ctypes.c_void_p()
        check(lib().od_comm_create(ctypes.byref(h), int(device), int(nbytes), int(nevents)), "od_comm_create")
        return cls(h)

    @classmethod
    def open(cls, handles: bytes, device: int = 0) -> "Comm":
        h = ctypes.c_void_p()
        blob = ctypes.create_string_buffer(bytes(handles), len(handles))
        check(lib().od_comm_open(ctypes.byref(h), int(device), blob, len(handles)), "od_comm_open")
        return cls(h)

    def handles(self) -> bytes:
        n = 16 + 64 * (1 + self.nevents)
        blob = ctypes.create_string_buffer(n)
        check(lib().od_comm_handles(self._h, blob, n), "od_comm_handles")
        return blob.raw

    def record(self, event: int, stream: int) -> None:
        check(lib().od_comm_record(self._h, int(event), stream), "od_comm_record")

    def wait(self, event: int, stream: int) -> None:
        check(lib().od_comm_wait(self._h, int(event), stream), "od_comm_wait")

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().od_comm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop (od_server): admits independent solves under an HBM budget
    and keeps them resident until released.  By default each admitted job's
    whole run is one persistent launch on one of 16 streams (job_streams), the
    jobs' kernels sharing the SMs; job_streams=0 advances all running 3D jobs
    together in batched launches of batch_steps steps.  next_completion()
    hands out jobs as they end, so a client can release them at once."""

    def __init__(self, hbm_budget_bytes: int, *, max_active: int = 0, device: int = 0, threads: int = 0,
                 cells_per_thread: int = 0, stages: int = 0, arith: int = -1, max_jobs_per_launch: int = 0,
                 batch_steps: int = 0, job_streams: int | None = None):
        cfg = _native.od_server_config()
        lib().od_server_config_default(ctypes.byref(cfg))
        cfg.batch_steps = int(batch_steps)
        if job_streams is not None:  # else the library's default (one persistent launch per job)
            cfg.job_streams = int(job_streams)
        cfg.hbm_budget_bytes = int(hbm_budget_bytes)
        cfg.max_active, cfg.device = int(max_active), int(device)
        cfg.threads, cfg.cells_per_thread, cfg.stages, cfg.arith = int(threads), int(cells_per_thread), \
            int(stages), int(arith)
        if max_jobs_per_launch:
            cfg.max_jobs_per_launch = int(max_jobs_per_launch)
        h = ctypes.c_void_p()
        check(lib().od_server_create(ctypes.byref(h), ctypes.byref(cfg)), "od_server_create")
        self._h = h
        self._sizes = {}

    def submit(self, nx, ny, nz, iters, **kw) -> int:
        cfg, keep = make_config(nx, ny, nz, **kw)
        jid = ctypes.c_uint64()
        check(lib().od_server_submit(self._h, ctypes.byref(cfg), int(iters), ctypes.byref(jid)), "od_server_submit")
        self._sizes[jid.value] = int(nx) * int(ny) * int(nz)
        return jid.value

    def poll(self, job: int) -> bool:
        """True once the job is done or failed (od_poll, no waiting)."""
        done = ctypes.c_int32()
        check(lib().od_poll(self._h, int(job), ctypes.byref(done)), "od_poll")
        return bool(done.value)

    def wait(self, job: int, timeout_s: float = 60.0) -> int:
        st = ctypes.c_int32()
        check(lib().od_server_wait(self._h, job, float(timeout_s), ctypes.byref(st)), "od_server_wait")
        return st.value

    def next_completion(self, timeout_s: float = 1.0) -> int | None:
        """The next job that ended (done or failed), in the order they ended;
        None if none ended within timeout_s (od_server_next_completion)."""
        jid = ctypes.c_uint64()
        check(lib().od_server_next_completion(self._h, float(timeout_s), ctypes.byref(jid)),
              "od_server_next_completion")
        return jid.value or None

    def info(self, job: int) -> dict:
        i = _native.od_job_info()
        check(lib().od_server_job_info(self._h, job, ctypes.byref(i)), "od_server_job_info")
        return {f: getattr(i, f) for f, _ in _native.od_job_info._fields_}

    def fetch(self, job: int, out=None):
        if out is None:
            out = np.empty(self._sizes[job], dtype=np.float64)
        if isinstance(out, np.ndarray):
            check(lib().od_server_fetch(self._h, job, out.ctypes.data, 0), "od_server_fetch")
        else:
            check(lib().od_server_fetch(self._h, job, out.data_ptr(), 1), "od_server_fetch")
        return out

    def release(self, job: int) -> None:
        check(lib().od_server_release(self._h, job), "od_server_release")
        self._sizes.pop(job, None)

    def stats(self) -> dict:
        st = _native.od_server_stats_t()
        check(lib().od_server_stats(self._h, ctypes.byref(st)), "od_server_stats")
        return {f: getattr(st, f) for f, _ in _native.od_server_stats_t._fields_}

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().od_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
