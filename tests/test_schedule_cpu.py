"""The persistent path's schedule, checked on the host for many
decompositions: the tiles partition every chare exactly, and each tile's
dependency list is exactly the set of tiles that a 7-point update links it
to -- the tiles whose cells it reads, and those that read its cells (a tile
reads the cells next to its own along each axis, across chare faces too).
With that, waiting for the listed tiles' previous step covers both the
read-after-write and the write-after-read hazards of the two parity buffers.
The expected sets are computed here from the tile boxes by dilation, not by
the library's own rule."""
import numpy as np
import pytest

from paper_2605_12734_gb300 import build as od_build


@pytest.fixture(scope="module")
def od():
    od_build.build()
    import paper_2605_12734_gb300 as pkg
    return pkg


def random_cuts(rng, n, parts):
    inner = sorted(rng.choice(np.arange(1, n), size=parts - 1, replace=False).tolist())
    return [0] + inner + [n]


def labels(tiles, dims):
    """Grid (z, y, x) of tile indices; every cell must belong to exactly one tile."""
    nx, ny, nz = dims
    lab = np.full((nz, ny, nx), -1, dtype=np.int64)
    for t, (_, x0, bx, y0, by, z0, bz) in enumerate(tiles):
        blk = lab[z0:z0 + bz, y0:y0 + by, x0:x0 + bx]
        assert (blk == -1).all(), "tiles overlap"
        blk[...] = t
    assert (lab >= 0).all(), "a cell belongs to no tile"
    return lab


def expected_deps(lab, ntiles):
    """b in deps(a) iff some cell of b is a cell of a or a face neighbour of one."""
    deps = [set([t]) for t in range(ntiles)]
    for axis in range(3):
        a = np.moveaxis(lab, axis, 0)
        lo, hi = a[:-1].ravel(), a[1:].ravel()
        for u, v in set(zip(lo.tolist(), hi.tolist())):
            deps[u].add(v)
            deps[v].add(u)
    return deps


def check(od, dims, internal=None, **kw):
    """dims: the configuration's grid; internal: the tiles' coordinate space
    (the same for 3D; (nx, 1, ny) for a 2D grid)."""
    internal = internal or dims
    tiles, ptr, idx = od.plan_tiles(*dims, **kw)
    lab = labels(tiles, internal)
    want = expected_deps(lab, len(tiles))
    box, _ = od.decompose(*dims, **kw)
    if internal != dims:  # 2D: chare boxes come back as (x0, bx, y0, by, 0, 1); tiles see (x, 1, y)
        box = box[:, [0, 1, 4, 5, 2, 3]]
    for t, row in enumerate(tiles):
        c, x0, bx, y0, by, z0, bz = row
        cb = box[c]
        assert cb[0] <= x0 and x0 + bx <= cb[0] + cb[1], "tile outside its chare (x)"
        assert cb[2] <= y0 and y0 + by <= cb[2] + cb[3], "tile outside its chare (y)"
        assert cb[4] <= z0 and z0 + bz <= cb[4] + cb[5], "tile outside its chare (z)"
        got = set(idx[ptr[t]:ptr[t + 1]].tolist())
        assert got == want[t], (t, sorted(got ^ want[t]))


@pytest.mark.parametrize("seed", range(12))
def test_schedule_uneven_3d(od, seed):
    rng = np.random.default_rng(seed)
    dims = tuple(int(v) for v in rng.integers(6, 40, 3))
    parts = [int(rng.integers(1, min(5, d) + 1)) for d in dims]
    cuts = tuple(random_cuts(rng, d, p) for d, p in zip(dims, parts))
    kw = dict(cuts=cuts, tile_y=int(rng.integers(0, 6)), tile_z=int(rng.integers(0, 9)))
    check(od, dims, **kw)


@pytest.mark.parametrize("kw", [dict(split=(2, 2, 2)), dict(split=(4, 4, 4), tile_y=3, tile_z=5),
                                dict(split=(1, 3, 2), threads=128, cells_per_thread=2),
                                dict(cuts=([0, 1, 2, 30], [0, 29, 30], [0, 1, 30]))])
def test_schedule_regular_3d(od, kw):
    check(od, (30, 30, 30), **kw)


@pytest.mark.parametrize("seed", range(6))
def test_schedule_2d(od, seed):
    # a 2D grid appears as (nx, 1, ny); its tiles are row segments
    rng = np.random.default_rng(100 + seed)
    nx, ny = int(rng.integers(20, 3000)), int(rng.integers(4, 60))
    kw = dict(split=(int(rng.integers(1, 4)), int(rng.integers(1, 4))), stencil="2d5",
              tile_y=int(rng.choice([0, 64, 200])), tile_z=int(rng.integers(0, 9)))
    tiles, _, _ = od.plan_tiles(nx, ny, 1, **kw)
    box, _ = od.decompose(nx, ny, 1, **kw)
    assert ((tiles[:, 1] - box[tiles[:, 0], 0]) % 2 == 0).all(), "a segment must start at an even column"
    check(od, (nx, ny, 1), internal=(nx, 1, ny), **kw)
