"""GPU parity of the 2D 5-point Jacobi (the paper's Jacobi2D application,
Sec. V) against the CPU oracle, bit for bit, on every execution path.

Small grids run the oracle's full 2D sweep; they span several tiles (row
segments and row chunks), ragged segments, blocks one cell wide or one row
high, and 1 x 1 blocks.  The paper's 32768 x 32768 domain is checked at
several ODFs on sampled cells the oracle computes on their dependency cone,
plus the discrete maximum principle on every cell."""
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
    # name: (nx, ny, decomposition kwargs, seed, init_mode, iters)
    "64_2x2": (64, 64, dict(split=(2, 2)), 1, 0, 10),
    "ragged_odd": (301, 77, dict(split=(3, 2)), 5, 1, 9),
    "uneven_cuts": (100, 40, dict(cuts=([0, 3, 50, 51, 100], [0, 1, 2, 40])), 8, 1, 7),
    "one_by_one": (9, 7, dict(split=(9, 7)), 11, 1, 6),
    "segments": (3001, 20, dict(split=(1, 2)), 3, 1, 8),
    "small_tiles": (301, 77, dict(split=(2, 3), tile_y=64, tile_z=5), 13, 1, 8),
    "single_cell": (1, 1, dict(split=(1, 1)), 2, 1, 4),
    "zero_interior": (130, 90, dict(split=(4, 3)), 21, 0, 11),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("path", PATHS)
def test_2d_path_matches_oracle(od, path, case):
    nx, ny, dec, seed, mode, iters = CASES[case]
    want = oracle.solve_2d(nx, ny, seed, mode, iters)
    with od.Jacobi2D(nx, ny, seed=seed, init_mode=mode, path=path, **dec) as s:
        first = iters // 3
        s.step(first)
        s.step(iters - first)
        got = s.read()
        st = s.stats()
    assert st["steps_done"] == iters
    assert got.size == nx * ny
    assert_bitexact(got, want, f"{path}/{case}")


@pytest.mark.parametrize("path", PATHS)
def test_2d_zero_iterations_is_initial_field(od, path):
    want = oracle.solve_2d(57, 33, 4, 1, 0)
    with od.Jacobi2D(57, 33, split=(3, 2), seed=4, init_mode=1, path=path) as s:
        s.step(0)
        assert_bitexact(s.read(), want, "iters=0")


@pytest.mark.parametrize("shape", [
    dict(threads=128, cells_per_thread=2), dict(threads=128, cells_per_thread=8),
    dict(threads=256, cells_per_thread=1), dict(threads=256, cells_per_thread=8),
    dict(threads=512, cells_per_thread=1), dict(threads=512, cells_per_thread=2, stages=3),
    dict(threads=256, cells_per_thread=4, stages=8),
    dict(threads=128, cells_per_thread=4, tile_y=6, tile_z=1),
] + [dict(arith=m) for m in range(16)])
@pytest.mark.parametrize("path", ["fused", "persistent"])
def test_2d_launch_shapes(od, path, shape):
    nx, ny = 777, 45
    want = oracle.solve_2d(nx, ny, 17, 1, 6)
    with od.Jacobi2D(nx, ny, split=(2, 3), seed=17, init_mode=1, path=path, **shape) as s:
        s.step(6)
        assert_bitexact(s.read(), want, f"{path} {shape}")


def test_2d_switching_paths_and_checkpoint(od):
    nx, ny = 200, 150
    want = oracle.solve_2d(nx, ny, 6, 1, 12)
    with od.Jacobi2D(nx, ny, split=(4, 3), seed=6, init_mode=1, path="per_chare") as s:
        for path in ["per_chare", "fused", "graph", "persistent"]:
            s.set_path(path)
            s.step(3)
        assert_bitexact(s.read(), want, "switching")
    # restore u^5 into a fresh context and continue
    u5 = oracle.solve_2d(nx, ny, 6, 1, 5)
    with od.Jacobi2D(nx, ny, split=(2, 5), seed=6, init_mode=1, path="persistent") as s:
        s.write(u5)
        s.step(7)
        assert_bitexact(s.read(), want, "restore")


@pytest.mark.parametrize("path", ["persistent", "per_chare"])
@pytest.mark.parametrize("kind", ["large", "signed", "binades"])
def test_2d_imported_fields_of_any_range(od, path, kind):
    # the 2D sweep's anchored window follows the imported field's largest
    # value; cells outside it take the IEEE form; every cell is the oracle's
    nx, ny, seed, iters = 300, 170, 23, 11
    rng = np.random.default_rng({"large": 51, "signed": 52, "binades": 53}[kind])
    u = rng.random(nx * ny)
    if kind == "large":
        interior = u * 3e7
    elif kind == "signed":
        interior = u * 2.0 - 1.0
    else:
        interior = (1.0 + u) * np.exp2(rng.integers(-30, 31, nx * ny).astype(np.float64))
    P = oracle.init_padded_2d(nx, ny, seed, 1)
    P[1:-1, 1:-1] = interior.reshape(ny, nx)
    want = np.ascontiguousarray(oracle.sweep_2d(P, iters)[1:-1, 1:-1]).ravel()
    with od.Jacobi2D(nx, ny, split=(4, 3), seed=seed, init_mode=1, path=path) as s:
        s.write(interior)
        s.step(iters)
        assert_bitexact(s.read(), want, f"imported {kind} 2D field, {path}")


def test_2d_device_read_and_write(od):
    import torch
    nx, ny = 96, 80
    want = oracle.solve_2d(nx, ny, 2, 1, 5)
    with od.Jacobi2D(nx, ny, split=(2, 2), seed=2, init_mode=1, path="fused") as s:
        s.step(5)
        t = torch.empty(nx * ny, dtype=torch.float64, device="cuda:0")
        s.read(t)
        assert_bitexact(t.cpu().numpy(), want, "device read")
        s.write(t)
        assert_bitexact(s.read(), want, "device write")


def test_2d_async_host_transfers(od):
    import torch
    nx, ny = 300, 170
    u3 = torch.from_numpy(oracle.solve_2d(nx, ny, 8, 1, 3)).pin_memory()
    out = torch.zeros(nx * ny, dtype=torch.float64, pin_memory=True)
    with od.Jacobi2D(nx, ny, split=(3, 2), seed=8, init_mode=1, path="persistent") as s:
        s.write_async(u3)
        s.step(4)
        s.read_async(out)
        s.sync()
        assert_bitexact(out.numpy(), oracle.solve_2d(nx, ny, 8, 1, 7), "import u^3, four steps, export")
        assert bits(s.read_cells([0, nx * ny - 1]))[1] == bits(out.numpy()[-1:])[0]


def test_2d_autotune(od, tmp_path, monkeypatch):
    monkeypatch.setenv("OD_TUNE_CACHE", str(tmp_path / "tune.txt"))
    nx, ny = 1024, 512
    want = oracle.solve_2d(nx, ny, 3, 1, 5)
    with od.Jacobi2D(nx, ny, split=(4, 4), seed=3, init_mode=1, path="persistent", autotune=True) as s:
        s.step(5)
        assert_bitexact(s.read(), want, "autotuned")
        assert s.stats()["tuned"] == 1


def test_2d_server_batched_rejects(od):
    # a batched launch shares the 3D kernel: 2D jobs are refused there
    with od.Server(1 << 30, job_streams=0) as srv:
        with pytest.raises(od.ODError) as ei:
            srv.submit(64, 64, 1, 5, stencil="2d5")
        assert ei.value.status == od._native.OD_EINVAL


def test_2d_jobs_served_beside_3d(od):
    # per-job launches (the default) run each job's own kernel: 2D jobs of the
    # paper's application, uneven splits included, beside 3D jobs, each equal
    # to the oracle
    jobs2d = [((512, 384), (4, 3), 9, 31), ((1000, 130), (8, 2), 25, 32), ((96, 64), (1, 1), 4, 33)]
    jobs3d = [((64, 64, 64), (2, 2, 2), 12, 34), ((100, 100, 100), (6, 6, 6), 7, 35)]
    with od.Server(2 << 30) as srv:
        ids2 = [srv.submit(nx, ny, 1, it, split=sp, seed=seed, stencil="2d5") for (nx, ny), sp, it, seed in jobs2d]
        ids3 = [srv.submit(*dims, it, split=sp, seed=seed) for dims, sp, it, seed in jobs3d]
        got2, got3 = [], []
        for jid in ids2 + ids3:
            assert srv.wait(jid, 120.0) == od._native.OD_JOB_DONE, srv.info(jid)
        for jid, ((nx, ny), _, _, _) in zip(ids2, jobs2d):
            got2.append(srv.fetch(jid, np.empty(nx * ny)))
            srv.release(jid)
        for jid in ids3:
            got3.append(srv.fetch(jid))
            srv.release(jid)
    for res, ((nx, ny), sp, it, seed) in zip(got2, jobs2d):
        assert_bitexact(res, oracle.solve_2d(nx, ny, seed, 1, it), f"2D {nx}x{ny} {sp}")
    for res, (dims, sp, it, seed) in zip(got3, jobs3d):
        assert_bitexact(res, oracle.solve(*dims, seed, 1, it), f"3D {dims} {sp}")


# ------------------------------------------------------------------ full size

def check_sampled_2d(od, w, path, iters, n_random=6, **kw):
    box, _ = od.decompose_2d(w.nx, w.ny, split=w.split[:2])
    with od.Jacobi2D(w.nx, w.ny, seed=w.seed, init_mode=w.init_mode, path=path, split=w.split[:2], **kw) as s:
        s.step(iters)
        u = s.read()
    assert float(u.min()) >= 0.0 and float(u.max()) < 1.0
    rng = np.random.default_rng(w.seed)
    pts = {(0, 0), (w.nx - 1, w.ny - 1), (w.nx // 2, w.ny // 2), (0, w.ny - 1), (w.nx - 1, 0)}
    for (x0, bx, y0, by) in box[rng.choice(len(box), size=min(len(box), 6), replace=False)]:
        pts.add((int(x0), int(y0)))
        pts.add((int(x0 + bx - 1), int(y0 + by - 1)))
        pts.add((int(x0 + bx // 2), int(y0)))
    for _ in range(n_random):
        pts.add((int(rng.integers(w.nx)), int(rng.integers(w.ny))))
    for (x, y) in sorted(pts):
        want = oracle.point_2d(w.nx, w.ny, w.seed, w.init_mode, iters, x, y)
        got = u[x + w.nx * y]
        assert bits(np.array([got]))[0] == bits(np.array([want]))[0], (path, x, y, got, want)


@pytest.mark.parametrize("odf", [1, 64, 4096])
def test_2d_full_32768_sampled(od, odf):
    w = inputs.jacobi2d_32768(odf)
    check_sampled_2d(od, w, "persistent", w.iters)


def test_2d_full_32768_fused_sampled(od):
    w = inputs.jacobi2d_32768(256, iters=20)
    check_sampled_2d(od, w, "fused", w.iters)
