"""The largest grids one device holds, and reading selected cells.

od_read_cells is first checked against a full read on small 3D and 2D grids
(every parity, several decompositions, shards).  Then the two largest
workloads: a 2048^3 3D grid (two fp64 fields of 8.6e9 cells, about 140 GB
with ghosts) and the paper's Jacobi2D strong-scaling domain, 131072 x 98304
(Sec. V; about 206 GB), each after a few iterations on sampled cells the
oracle computes on their dependency cone: chare corners and faces, the domain
corners and random cells, plus the discrete maximum principle on a random
million cells.  No full-grid copy leaves the device."""
import numpy as np
import pytest

import oracle
from paper_2605_12734_gb300 import inputs

pytestmark = pytest.mark.gpu


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
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def free_bytes():
    # a closed context's arena goes back to torch's caching allocator; hand it to the device
    import torch
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info(0)
    return free


@pytest.mark.parametrize("iters", [0, 3, 4])
def test_read_cells_matches_read_3d(od, iters):
    nx, ny, nz = 45, 38, 29
    with od.Jacobi3D(nx, ny, nz, split=(3, 2, 2), seed=9, init_mode=1, path="fused") as s:
        s.step(iters)
        full = s.read()
        idx = np.random.default_rng(iters).integers(0, full.size, 5000)
        idx = np.concatenate([idx, [0, full.size - 1, nx - 1, nx * ny - 1]])
        assert np.array_equal(bits(s.read_cells(idx)), bits(full[idx]))
        assert s.read_cells(np.zeros(0, dtype=np.int64)).size == 0


def test_read_cells_matches_read_2d(od):
    nx, ny = 301, 77
    with od.Jacobi2D(nx, ny, split=(3, 2), seed=5, init_mode=1, path="persistent") as s:
        s.step(5)
        full = s.read()
        idx = np.arange(full.size)
        assert np.array_equal(bits(s.read_cells(idx)), bits(full))


def test_read_cells_in_a_shard(od):
    # cells are indexed in the shard's own interior
    with od.Jacobi3D(20, 16, 12, split=(2, 2, 1), seed=4, init_mode=1, path="fused",
                     gdims=(40, 16, 12), goff=(20, 0, 0)) as s:
        s.step(2)
        full = s.read()
        idx = np.arange(0, full.size, 7)
        assert np.array_equal(bits(s.read_cells(idx)), bits(full[idx]))


def test_read_cells_rejects_outside_indices(od):
    with od.Jacobi3D(16, 16, 16, split=(2, 2, 2), seed=1, init_mode=1, path="fused") as s:
        for bad in ([-1], [16 ** 3], [0, 5, 16 ** 3 + 9]):
            with pytest.raises(od.ODError) as ei:
                s.read_cells(np.array(bad, dtype=np.int64))
            assert ei.value.status == od._native.OD_EINVAL
        s.step(1)  # the context stays usable
        assert s.read_cells([0]).size == 1


def sample_points(rng, box, dims, n_random):
    """Domain corners and centre, corners and face midpoints of a few chares,
    random cells."""
    pts = set()
    for corner in np.ndindex(*(2,) * len(dims)):
        pts.add(tuple((d - 1) * c for d, c in zip(dims, corner)))
    pts.add(tuple(d // 2 for d in dims))
    nd = len(dims)
    for row in box[rng.choice(len(box), size=min(len(box), 6), replace=False)]:
        o = [int(row[2 * a]) for a in range(nd)]
        e = [int(row[2 * a + 1]) for a in range(nd)]
        pts.add(tuple(o))
        pts.add(tuple(a + b - 1 for a, b in zip(o, e)))
        pts.add(tuple(a + b // 2 if q else a for q, (a, b) in enumerate(zip(o, e))))
    for _ in range(n_random):
        pts.add(tuple(int(rng.integers(d)) for d in dims))
    return sorted(pts)


def linear(p, dims):
    g, stride = 0, 1
    for c, d in zip(p, dims):
        g += c * stride
        stride *= d
    return g


def check_max_principle(s, ncell, rng):
    # every iterate of the 7- (5-) point average of a field in [0, 1) stays in [0, 1)
    v = s.read_cells(rng.integers(0, ncell, 1 << 20))
    assert float(v.min()) >= 0.0 and float(v.max()) < 1.0


@pytest.mark.parametrize("split,path", [((16, 16, 16), "persistent"), ((8, 8, 8), "persistent"),
                                        ((16, 16, 16), "fused")])
def test_3d_2048_cubed_sampled(od, split, path):
    n, iters, seed = 2048, 3, 12
    need = 2 * (n // split[0] + 2) ** 3 * 8 * split[0] * split[1] * split[2]
    if free_bytes() < need + (4 << 30):
        pytest.skip(f"needs {need / 1e9:.0f} GB free on the device")
    box, _ = od.decompose(n, n, n, split=split)
    rng = np.random.default_rng(seed)
    pts = sample_points(rng, box, (n, n, n), 24)
    with od.Jacobi3D(n, n, n, split=split, seed=seed, init_mode=inputs.INIT_UNIFORM, path=path) as s:
        s.step(iters)
        got = s.read_cells([linear(p, (n, n, n)) for p in pts])
        check_max_principle(s, n ** 3, rng)
    for p, g in zip(pts, got):
        want = oracle.point(n, n, n, seed, inputs.INIT_UNIFORM, iters, *p)
        assert bits([g])[0] == bits([want])[0], (path, split, p, g, want)


@pytest.mark.parametrize("split", [(64, 64), (8, 8)])
def test_2d_strong_scaling_domain_sampled(od, split):
    nx, ny, iters, seed = 131072, 98304, 3, 14
    need = 2 * (nx // split[0] + 2) * (ny // split[1] + 2) * 8 * split[0] * split[1]
    if free_bytes() < need + (4 << 30):
        pytest.skip(f"needs {need / 1e9:.0f} GB free on the device")
    box, _ = od.decompose_2d(nx, ny, split=split)
    rng = np.random.default_rng(seed)
    pts = sample_points(rng, box, (nx, ny), 24)
    with od.Jacobi2D(nx, ny, split=split, seed=seed, init_mode=inputs.INIT_UNIFORM, path="persistent") as s:
        s.step(iters)
        got = s.read_cells([linear(p, (nx, ny)) for p in pts])
        check_max_principle(s, nx * ny, rng)
    for p, g in zip(pts, got):
        want = oracle.point_2d(nx, ny, seed, inputs.INIT_UNIFORM, iters, *p)
        assert bits([g])[0] == bits([want])[0], (split, p, g, want)
