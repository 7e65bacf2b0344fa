"""GPU parity: every execution path of libod against the CPU oracle, bit for
bit (the method promises the undecomposed answer for any decomposition).

Small cases run the oracle's full sweep.  The full-size workloads (512^3 at
ODF 1 and 4096 for 100 iterations, the uneven 768x512x512 grid of 300 chares
for 200, 1024^3 at ODF 4096 for 50) run in the launch configuration the
benchmark times and are compared with the oracle's multithreaded sweep on
every cell."""
import numpy as np
import pytest

import oracle
from paper_2605_12734_gb300 import inputs

pytestmark = pytest.mark.gpu

PATHS = ["per_chare", "fused", "graph", "persistent", "fused_graph"]


@pytest.fixture(scope="module")
def od():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_12734_gb300 import build
    build.build()
    import paper_2605_12734_gb300 as pkg
    return pkg


def bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


def assert_bitexact(got, want, what=""):
    g, w = bits(got), bits(want)
    if not np.array_equal(g, w):
        bad = np.flatnonzero(g != w)
        i = int(bad[0])
        raise AssertionError(f"{what}: {bad.size} cells differ; first at {i}: "
                             f"got {got[i]!r} want {want[i]!r}")


CASES = {
    # name: (nx, ny, nz, decomposition kwargs, seed, init_mode, iters)
    "cfg1_64_2x2x2": (64, 64, 64, dict(split=(2, 2, 2)), 1, 0, 10),
    "odf1_ragged": (40, 36, 33, dict(split=(1, 1, 1)), 5, 1, 7),
    "uneven_cuts": (70, 45, 38, dict(cuts=([0, 13, 40, 70], [0, 24, 45], [0, 5, 6, 38])), 8, 1, 9),
    "one_wide": (6, 5, 7, dict(cuts=([0, 1, 2, 3, 4, 5, 6], [0, 1, 5], [0, 3, 4, 7])), 11, 1, 6),
    "small_tiles": (64, 48, 40, dict(split=(2, 3, 2), tile_y=5, tile_z=7), 3, 1, 8),
    "balanced_odd": (50, 31, 29, dict(split=(3, 3, 2)), 21, 0, 11),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("path", PATHS)
def test_path_matches_oracle(od, path, case):
    nx, ny, nz, dec, seed, mode, iters = CASES[case]
    want = oracle.solve(nx, ny, nz, seed, mode, iters)
    with od.Jacobi3D(nx, ny, nz, seed=seed, init_mode=mode, path=path, **dec) as s:
        first = iters // 3
        s.step(first)            # two calls: the step count carries over
        s.step(iters - first)
        got = s.read()
        st = s.stats()
    assert st["steps_done"] == iters
    assert st["kernel_launches"] >= 1
    assert_bitexact(got, want, f"{path}/{case}")


@pytest.mark.parametrize("path", PATHS)
def test_zero_iterations_is_initial_field(od, path):
    nx, ny, nz = 33, 20, 17
    want = oracle.solve(nx, ny, nz, 4, 1, 0)
    with od.Jacobi3D(nx, ny, nz, split=(2, 2, 3), seed=4, init_mode=1, path=path) as s:
        s.step(0)
        assert_bitexact(s.read(), want, "iters=0")


def test_switching_paths_mid_run(od):
    nx, ny, nz = 48, 40, 36
    want = oracle.solve(nx, ny, nz, 9, 1, 13)
    with od.Jacobi3D(nx, ny, nz, split=(2, 2, 3), seed=9, init_mode=1, path="fused") as s:
        for path, n in [("fused", 3), ("per_chare", 2), ("persistent", 4), ("graph", 3), ("fused", 1)]:
            s.set_path(path)
            s.step(n)
        assert_bitexact(s.read(), want, "mixed paths")


@pytest.mark.parametrize("arith", [10, 12, 14])
def test_switching_paths_uneven_cuts(od, arith):
    # the fused 3D paths read the neighbours' faces straight from their arrays
    # and leave the ghost layers behind; a per-chare or graph step after them
    # must find its ghost layers refreshed (1-wide blocks and uneven faces)
    nx, ny, nz = 37, 29, 26
    cuts = ([0, 1, 13, 30, 37], [0, 9, 10, 29], [0, 7, 25, 26])
    want = oracle.solve(nx, ny, nz, 31, 1, 30)
    with od.Jacobi3D(nx, ny, nz, cuts=cuts, seed=31, init_mode=1, path="persistent", arith=arith) as s:
        for path, n in [("persistent", 2), ("per_chare", 1), ("fused", 3), ("graph", 2), ("persistent", 1),
                        ("fused_graph", 11), ("graph", 1), ("fused", 2), ("per_chare", 3), ("fused_graph", 2),
                        ("persistent", 2)]:
            s.set_path(path)
            s.step(n)
        assert_bitexact(s.read(), want, f"mixed paths, uneven cuts, arith {arith}")


def test_checkpoint_restore(od):
    nx, ny, nz = 40, 36, 30
    want = oracle.solve(nx, ny, nz, 12, 1, 10)
    with od.Jacobi3D(nx, ny, nz, split=(2, 3, 2), seed=12, init_mode=1, path="fused") as a:
        a.step(4)
        ckpt = a.read()
    # a fresh context (same seed: same Dirichlet shell) resumes from the checkpoint
    with od.Jacobi3D(nx, ny, nz, split=(3, 2, 1), seed=12, init_mode=1, path="persistent") as b:
        b.write(ckpt)
        b.step(6)
        assert_bitexact(b.read(), want, "restored")


def test_device_read_and_write(od):
    import torch
    nx, ny, nz = 32, 32, 32
    want = oracle.solve(nx, ny, nz, 2, 1, 5)
    with od.Jacobi3D(nx, ny, nz, split=(2, 2, 2), seed=2, init_mode=1, path="fused") as s:
        s.step(5)
        t = torch.empty(nx * ny * nz, dtype=torch.float64, device="cuda:0")
        s.read(t)
        assert_bitexact(t.cpu().numpy(), want, "device read")
        # writing the field back leaves it unchanged
        s.write(t)
        assert_bitexact(s.read(), want, "device write")


def _imported_field(kind, n, rng):
    """Interior values for an imported field: magnitudes far from the seeded
    shell's [0, 1), signs, zeros and subnormals -- cells whose operands span
    more binades than the exact arithmetic's window, or leave its domain."""
    u = rng.random(n)
    if kind == "large":        # 1e6 times the shell's values: the anchor moves up with the field
        return u * 1e6
    if kind == "signed":       # negative operands leave the window's domain
        return u * 2.0 - 1.0
    if kind == "tiny":         # zeros, subnormals and values far below the shell's
        v = u * 1e-300
        v[::7] = 0.0
        v[3::11] = 5e-324
        return v
    # mixed binades: 2^k for k in [-40, 40] times U[1, 2)
    return (1.0 + u) * np.exp2(rng.integers(-40, 41, n).astype(np.float64))


@pytest.mark.parametrize("path", ["persistent", "fused", "per_chare"])
@pytest.mark.parametrize("kind", ["large", "signed", "tiny", "binades"])
def test_imported_fields_of_any_range(od, path, kind):
    # od_write raises the field's largest value, which anchors the exact
    # arithmetic's window; cells whose operands leave the window take the
    # IEEE form.  Either way every cell equals the oracle's sweep of the same
    # padded field (the imported interior inside the seeded shell).
    nx, ny, nz, seed, iters = 40, 34, 29, 21, 9
    rng = np.random.default_rng({"large": 41, "signed": 42, "tiny": 43, "binades": 44}[kind])
    interior = _imported_field(kind, nx * ny * nz, rng)
    P = oracle.init_padded(nx, ny, nz, seed, 1)
    P[1:-1, 1:-1, 1:-1] = interior.reshape(nz, ny, nx)
    want = oracle.interior(oracle.sweep(P, iters))
    with od.Jacobi3D(nx, ny, nz, split=(3, 2, 2), seed=seed, init_mode=1, path=path) as s:
        s.write(interior)
        s.step(iters)
        assert_bitexact(s.read(), want, f"imported {kind} field, {path}")


@pytest.mark.parametrize("pe", [2, 3, 8])
def test_per_chare_with_several_submitting_threads(od, pe):
    # the per-chare path submitted by several host threads (the paper's PEs)
    nx, ny, nz = 70, 45, 38
    cuts = ([0, 13, 40, 70], [0, 24, 45], [0, 5, 6, 38])
    want = oracle.solve(nx, ny, nz, 8, 1, 9)
    with od.Jacobi3D(nx, ny, nz, cuts=cuts, seed=8, init_mode=1, path="per_chare", pe_threads=pe,
                     stream_pool=6) as s:
        s.step(4)
        s.step(5)
        assert_bitexact(s.read(), want, f"pe_threads={pe}")
        assert s.stats()["steps_done"] == 9


def test_pinned_host_read_and_write(od):
    # pinned host buffers are read and written in place by the I/O kernels
    import torch
    nx, ny, nz = 40, 33, 29
    want = oracle.solve(nx, ny, nz, 3, 1, 6)
    with od.Jacobi3D(nx, ny, nz, split=(2, 3, 1), seed=3, init_mode=1, path="fused") as s:
        s.step(6)
        h = torch.zeros(nx * ny * nz, dtype=torch.float64, pin_memory=True)
        s.read(h.numpy())
        assert_bitexact(h.numpy(), want, "pinned read")
        s.write(h.numpy())
        s.step(2)
        assert_bitexact(s.read(), oracle.solve(nx, ny, nz, 3, 1, 8), "pinned write, then two steps")
        view = torch.zeros(nx * ny * nz + 5, dtype=torch.float64, pin_memory=True)[3:3 + nx * ny * nz]
        s.read(view.numpy())  # a pointer inside a pinned allocation
        assert_bitexact(view.numpy(), oracle.solve(nx, ny, nz, 3, 1, 8), "pinned read at an offset")


def test_async_host_transfers_pipelined(od):
    # two contexts as a pipeline: job j's import and iterations are enqueued
    # before job j-1's export, so copies of one overlap the other's steps
    import torch
    nx, ny, nz = 50, 41, 37
    n = nx * ny * nz
    fields = [oracle.solve(nx, ny, nz, 7, 1, t) for t in (0, 3)]
    want = [oracle.solve(nx, ny, nz, 7, 1, t + 5) for t in (0, 3)]
    hin = [torch.from_numpy(f.copy()).pin_memory() for f in fields]
    hout = torch.zeros(n, dtype=torch.float64, pin_memory=True)
    strm = (torch.cuda.Stream(), torch.cuda.Stream())
    # the Dirichlet shell comes from the seed; the interior from each import
    with od.Jacobi3D(nx, ny, nz, split=(2, 2, 2), seed=7, init_mode=1, path="persistent",
                     stream=strm[0].cuda_stream) as a, \
            od.Jacobi3D(nx, ny, nz, split=(3, 1, 2), seed=7, init_mode=1, path="fused",
                        stream=strm[1].cuda_stream) as b:
        ctx = (a, b)
        ctx[0].write_async(hin[0])
        ctx[0].step(5)
        for j in range(1, 6):
            cur, prev = ctx[j % 2], ctx[(j - 1) % 2]
            cur.write_async(hin[j % 2])
            prev.read_async(hout)
            ev = torch.cuda.Event()
            ev.record(strm[(j - 1) % 2])  # after prev's gather, before its copy
            strm[j % 2].wait_event(ev)
            cur.step(5)
            prev.sync()
            assert_bitexact(hout.numpy(), want[(j - 1) % 2], f"job {j - 1}")
        ctx[1].read_async(hout.numpy())  # a numpy view of pinned memory works too
        ctx[1].sync()
        assert_bitexact(hout.numpy(), want[1], "job 5")


def test_async_export_then_import_share_the_staging_buffer(od):
    # the import's copy into the staging buffer waits for the export's copy out
    import torch
    nx, ny, nz = 33, 30, 28
    n = nx * ny * nz
    out = torch.zeros(n, dtype=torch.float64, pin_memory=True)
    new = torch.from_numpy(oracle.solve(nx, ny, nz, 5, 1, 2)).pin_memory()
    with od.Jacobi3D(nx, ny, nz, split=(2, 2, 1), seed=5, init_mode=1, path="fused") as s:
        s.step(4)
        s.read_async(out)
        s.write_async(new)
        s.step(3)
        s.sync()
        assert_bitexact(out.numpy(), oracle.solve(nx, ny, nz, 5, 1, 4), "export before the import")
        assert_bitexact(s.read(), oracle.solve(nx, ny, nz, 5, 1, 5), "import, then three steps")


def test_async_host_transfers_need_pinned_memory(od):
    with od.Jacobi3D(16, 16, 16, split=(2, 2, 2), seed=1, init_mode=1, path="fused") as s:
        pageable = np.zeros(16 ** 3)
        for call in (s.write_async, s.read_async):
            with pytest.raises(od.ODError) as ei:
                call(pageable)
            assert ei.value.status == od._native.OD_EINVAL
        s.step(1)
        s.sync()


@pytest.mark.parametrize("shape", [
    dict(threads=128, cells_per_thread=2), dict(threads=128, cells_per_thread=8),
    dict(threads=256, cells_per_thread=1), dict(threads=256, cells_per_thread=8),
    dict(threads=512, cells_per_thread=1), dict(threads=512, cells_per_thread=2, stages=3),
    dict(threads=256, cells_per_thread=4, stages=8),
    dict(threads=256, cells_per_thread=4, tile_y=3, tile_z=1),
    # deeper rings with tiles of odd, one and two planes
    dict(stages=5), dict(stages=5, tile_z=7), dict(stages=6, tile_z=2), dict(stages=6, tile_z=1),
    dict(stages=5, tile_z=3, tile_y=5, arith=7),
 ] + [dict(arith=m) for m in range(16)] + [dict(arith=m, threads=256, cells_per_thread=2) for m in (12, 14)])
@pytest.mark.parametrize("path", ["fused", "persistent"])
def test_launch_shapes(od, path, shape):
    nx, ny, nz = 96, 40, 44
    want = oracle.solve(nx, ny, nz, 17, 1, 6)
    with od.Jacobi3D(nx, ny, nz, split=(1, 2, 2), seed=17, init_mode=1, path=path, **shape) as s:
        s.step(6)
        assert_bitexact(s.read(), want, f"{path} {shape}")


@pytest.mark.parametrize("order", [1, 2, 3])
def test_persistent_task_orders(od, order):
    # 1: reversed on odd steps, 2: Morton order of the chares, 3: both
    nx, ny, nz = 64, 64, 64
    want = oracle.solve(nx, ny, nz, 6, 1, 9)
    with od.Jacobi3D(nx, ny, nz, cuts=([0, 10, 30, 33, 64], [0, 20, 40, 64], [0, 31, 64]), seed=6, init_mode=1,
                     path="persistent", order=order) as s:
        s.step(9)
        assert_bitexact(s.read(), want, f"order={order}")


def test_stalled_tile_times_out_without_hanging(od):
    # A tile that never publishes its step counter: the tiles that read it hit
    # the (short) wait limit; the kernel returns, the error surfaces on sync,
    # and the GPU context stays usable.
    with od.Jacobi3D(32, 32, 32, split=(2, 2, 2), seed=1, path="persistent",
                     spin_limit_ns=200_000_000) as s:
        s.stall_tile(0)
        s.step(3)
        with pytest.raises(od.ODError) as ei:
            s.sync()
        assert ei.value.status == od._native.OD_ETIMEOUT
        with pytest.raises(od.ODError) as ei:
            s.step(1)
        assert ei.value.status == od._native.OD_ESTATE
    want = oracle.solve(32, 32, 32, 1, 1, 2)
    with od.Jacobi3D(32, 32, 32, split=(2, 2, 2), seed=1, path="persistent") as s:
        s.step(2)
        assert_bitexact(s.read(), want, "after a timeout")


# ------------------------------------------------------------------ full size
#
# The benchmark's workloads at their own sizes, every cell compared with the
# oracle's undecomposed sweep (OpenMP over z-planes: a few seconds each on the
# GPU host's cores).  The launch configuration is the benchmark's: the
# library's default shape and arithmetic for the persistent path.


def check_full(od, w, path, iters, **kw):
    dec = {"cuts": w.cuts} if w.cuts else {"split": w.split}
    with od.Jacobi3D(w.nx, w.ny, w.nz, seed=w.seed, init_mode=w.init_mode, path=path, **dec, **kw) as s:
        s.step(iters)
        got = s.read()
    want = oracle.solve(w.nx, w.ny, w.nz, w.seed, w.init_mode, iters, threads=oracle.max_threads())
    assert_bitexact(got, want, f"{w.name} {path} {iters} iterations")


@pytest.mark.parametrize("odf", [1, 4096])
@pytest.mark.parametrize("path", ["fused", "persistent"])
def test_full_512_every_cell(od, path, odf):
    w = inputs.odf_sweep_512(odf)
    check_full(od, w, path, w.iters)


def test_full_uneven_768_every_cell(od):
    w = inputs.uneven_768()
    check_full(od, w, "persistent", w.iters)


def test_full_1024_odf4096_every_cell(od):
    w = inputs.ceiling_1024()
    check_full(od, w, "persistent", w.iters)
