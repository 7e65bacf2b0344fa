"""od_jacobi_noalloc: the entry point for callers that cannot allocate device
memory where they call (a framework owning all device memory through its own
pool, or a latency-critical loop where cudaMalloc would synchronise the
device).  Its double buffer is a static device array shared by every call.

It is checked through the C ABI against the CPU oracle's undecomposed sweep
and against the existing entry points (od_create / od_step / od_read on a
decomposed grid), bit for bit -- the tolerance every parity test here uses --
on calls in a row with different sizes and iteration counts, including 0 (the
input comes back) and 1 (the scratch is never seeded; the one step writes
u_out), so no call can lean on what an earlier one left in the shared
scratch.  This file is collected last so that a run stopping at its first
failure has run every other test already."""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_12734_gb300 import build
    build.build()
    import paper_2605_12734_gb300 as pkg
    return pkg, torch


def reference_interior(pkg, nx, ny, nz, seed, mode, iters, split):
    with pkg.Jacobi3D(nx, ny, nz, split=split, seed=seed, init_mode=mode, path="fused") as s:
        s.step(iters)
        return s.read()


def run_noalloc(pkg, torch, nx, ny, nz, seed, mode, iters):
    u_in = torch.from_numpy(oracle.init_padded(nx, ny, nz, seed, mode).ravel()).to("cuda:0")
    u_out = torch.full_like(u_in, float("nan"))
    L = pkg.lib()
    st = L.od_jacobi_noalloc(ctypes.c_void_p(u_in.data_ptr()), ctypes.c_void_p(u_out.data_ptr()),
                             nx, ny, nz, iters, None)
    assert st == 0, L.od_last_error()
    torch.cuda.synchronize()
    out = u_out.cpu().numpy().reshape(nz + 2, ny + 2, nx + 2)
    src = u_in.cpu().numpy().reshape(nz + 2, ny + 2, nx + 2)
    return out, src


def test_noalloc_matches_oracle_and_existing_entry_points_in_a_row(env):
    pkg, torch = env
    # odd and even counts, one step (the scratch is not used) and none
    cases = [(40, 36, 30, 12, 1, 7, (2, 3, 2)), (24, 20, 18, 5, 0, 4, (3, 2, 2)),
             (17, 9, 13, 3, 1, 1, (2, 1, 3)), (8, 8, 8, 2, 1, 0, (2, 2, 2)), (33, 5, 7, 9, 1, 2, (1, 1, 1))]
    for (nx, ny, nz, seed, mode, iters, split) in cases:
        want = oracle.solve(nx, ny, nz, seed, mode, iters)
        fused = reference_interior(pkg, nx, ny, nz, seed, mode, iters, split)
        assert np.array_equal(fused.view(np.uint64), want.view(np.uint64)), (nx, ny, nz, iters)
        out, src = run_noalloc(pkg, torch, nx, ny, nz, seed, mode, iters)
        got = np.ascontiguousarray(out[1:-1, 1:-1, 1:-1]).ravel()
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), (nx, ny, nz, iters)
        # the Dirichlet shell is carried over unchanged
        shell = np.ones(out.shape, dtype=bool)
        shell[1:-1, 1:-1, 1:-1] = False
        assert np.array_equal(out[shell].view(np.uint64), src[shell].view(np.uint64))


def test_noalloc_rejects_oversized_and_overlapping(env):
    pkg, torch = env
    L = pkg.lib()
    buf = torch.empty(64, dtype=torch.float64, device="cuda:0")
    # a padded grid larger than the static scratch is refused before any work
    st = L.od_jacobi_noalloc(ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr() + 8 * 32),
                             400, 400, 400, 1, None)
    assert st == 1 and b"static scratch" in L.od_last_error()
    st = L.od_jacobi_noalloc(ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr() + 8),
                             1, 1, 1, 1, None)
    assert st == 1 and b"overlap" in L.od_last_error()
