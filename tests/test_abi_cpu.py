"""Host-side tests of the C ABI: the library loads without a GPU, exports
every entry point include/od.h declares, and its planner (decomposition,
tiles, dependency lists, arena layout) is right.  No compute call is made."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2605_12734_gb300 import build as od_build
from paper_2605_12734_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def od():
    od_build.build()
    import paper_2605_12734_gb300 as pkg
    pkg.lib()
    return pkg


def header_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:OD_API\s+)?(?:const\s+)?[a-z_0-9]+\s*\**\s*(od_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(od):
    names = header_functions()
    assert "od_create" in names and "od_step" in names and "od_read" in names and "od_destroy" in names
    L = ctypes.CDLL(od._native.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding wraps all of them
    assert set(names) <= set(od._native.SIGNATURES), set(names) - set(od._native.SIGNATURES)


def test_version_and_defaults(od):
    assert b"sm_103a" in od.lib().od_version()
    cfg = od._native.od_config()
    od.lib().od_config_default(ctypes.byref(cfg))
    assert (cfg.nx, cfg.px, cfg.path) == (64, 1, od._native.OD_PATH_FUSED)


@pytest.mark.parametrize("n,p", [(64, 2), (100, 6), (512, 16), (7, 7), (513, 8), (1, 1)])
def test_balanced_split_matches_oracle(od, n, p):
    box, nbr = od.decompose(n, 1, 1, split=(p, 1, 1))
    edges = list(box[:, 0]) + [int(box[-1, 0] + box[-1, 1])]
    assert edges == list(oracle.split(n, p))


def test_decompose_uneven_cuts_and_neighbours(od):
    w = inputs.uneven_768()
    box, nbr = od.decompose(w.nx, w.ny, w.nz, cuts=w.cuts)
    px, py, pz = (len(c) - 1 for c in w.cuts)
    assert len(box) == px * py * pz == w.nchares == 300
    for c in range(len(box)):
        cx, cy, cz = c % px, (c // px) % py, c // (px * py)
        assert box[c, 0] == w.cuts[0][cx] and box[c, 1] == w.cuts[0][cx + 1] - w.cuts[0][cx]
        assert box[c, 2] == w.cuts[1][cy] and box[c, 4] == w.cuts[2][cz]
        assert 24 <= box[c, 1] <= 160 and 24 <= box[c, 3] <= 160 and 24 <= box[c, 5] <= 160
        want = [c - 1 if cx > 0 else -1, c + 1 if cx < px - 1 else -1,
                c - px if cy > 0 else -1, c + px if cy < py - 1 else -1,
                c - px * py if cz > 0 else -1, c + px * py if cz < pz - 1 else -1]
        assert list(nbr[c]) == want
    # the boxes tile the grid exactly
    assert int(np.sum(box[:, 1] * box[:, 3] * box[:, 5])) == w.cells


def test_auto_cta_shape(od):
    def shape(*dims, **kw):
        i = od.plan(*dims, **kw)
        return i["threads"], i["cells_per_thread"]
    assert shape(512, 512, 512, split=(16, 16, 16)) == (128, 4)
    assert shape(512, 512, 512, split=(1, 1, 1)) == (256, 4)
    assert shape(1024, 8, 8, split=(1, 1, 1)) == (256, 8)
    assert shape(2048, 8, 8, split=(1, 1, 1)) == (256, 8)


@pytest.mark.parametrize("odf", [1, 8, 64, 512, 4096])
def test_plan_model_bytes(od, odf):
    p = round(odf ** (1 / 3))
    info = od.plan(512, 512, 512, split=(p, p, p))
    assert info["nchares"] == odf
    assert info["cells"] == 512 ** 3
    b = 512 // p
    # every chare has 6 faces of b*b ghost cells; internal ones are fed by a
    # neighbour, the rest lie on the Dirichlet shell
    assert info["face_cells_internal"] + info["face_cells_dirichlet"] == odf * 6 * b * b
    assert info["face_cells_dirichlet"] == 6 * 512 * 512
    assert info["bytes_per_step"] == 16 * 512**3 + 16 * info["face_cells_internal"] + 8 * 6 * 512**2
    assert info["arena_bytes"] > 2 * 8 * 512**3


@pytest.mark.parametrize("bad", [
    dict(split=(3, 1, 1), dims=(2, 4, 4)),          # more blocks than cells
    dict(split=(1, 1, 1), dims=(0, 4, 4)),          # empty grid
    dict(split=(1, 1, 1), dims=(4, 4, 4), threads=96),
    dict(split=(1, 1, 1), dims=(4, 4, 4), cells_per_thread=3),
    dict(split=(1, 1, 1), dims=(4, 4, 4), threads=512, cells_per_thread=4),
    dict(split=(1, 1, 1), dims=(4, 4, 4), arith=9),
    dict(split=(1, 1, 1), dims=(4, 4, 4), stages=9),
    dict(split=(1, 1, 1), dims=(4, 4, 4), stages=2),
    dict(split=(1, 1, 1), dims=(8192, 4, 4)),       # row wider than any CTA can hold
    dict(split=(1, 1, 1), dims=(600, 4, 4), threads=128, cells_per_thread=4),  # 600 > 512
    dict(cuts=([0, 3, 2, 8], None, None), dims=(8, 4, 4)),  # not ascending
    dict(cuts=([1, 8], None, None), dims=(8, 4, 4)),        # does not start at 0
])
def test_invalid_configs_rejected(od, bad):
    dims = bad.pop("dims")
    with pytest.raises(od.ODError) as ei:
        od.plan(*dims, **bad)
    assert ei.value.status == od._native.OD_EINVAL
    assert od.lib().od_last_error()


# ----------------------------------------------------------------- tiles/deps
# A Python re-derivation of the tile partition from the plan is not possible
# through the ABI (tiles are internal), so these properties are checked through
# a debug view: od_plan's counts plus the decomposition.

@pytest.mark.parametrize("kw", [
    dict(dims=(64, 64, 64), split=(2, 2, 2)),
    dict(dims=(37, 29, 23), split=(3, 2, 2), tile_y=5, tile_z=4),
    dict(dims=(512, 512, 512), split=(1, 1, 1)),
    dict(dims=(120, 7, 9), split=(1, 1, 1), threads=128, cells_per_thread=2),
])
def test_tile_counts(od, kw):
    dims = kw.pop("dims")
    info = od.plan(*dims, **kw)
    box, _ = od.decompose(*dims, **kw)
    thr, cpt = info["threads"], info["cells_per_thread"]
    ty = kw.get("tile_y", 0)
    tz = kw.get("tile_z", 0) or 32
    total = 0
    for (x0, bx, y0, by, z0, bz) in box:
        cap = max(1, min(by, (thr * cpt) // bx, ty if ty else 1 << 30))
        total += -(-by // cap) * -(-bz // min(tz, bz))
    assert info["ntiles"] == total
    assert info["smem_bytes"] <= 232448
