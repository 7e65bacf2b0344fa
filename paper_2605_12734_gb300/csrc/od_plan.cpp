// od_plan.cpp -- decomposition, tiling, dependency lists and arena layout.
//
// Decompose (A1 of the hot path): the paper's runtime pre-fills a location
// table so that a sender knows where each destination chare lives (Sec. IV);
// here every chare lives on the same GPU, so the "location table" is a static
// neighbour table plus the device addresses of each neighbour's ghost layers,
// built once here and copied to the device by od_create.
#include "od_plan.h"

#include <algorithm>
#include <cstdio>
#include <cstring>

namespace od {

namespace {

constexpr size_t kAlign = 256;
constexpr int32_t kMaxSmem = 232448;  // 227 KB opt-in per CTA on sm_100/sm_103
constexpr int32_t kSmemHeader = 256;  // mbarriers + neighbour push table
constexpr int32_t kDefaultArith = 12;  // two FP64 adds, the rest in the anchored integer window

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
int32_t round_up(int32_t v, int32_t a) { return (v + a - 1) / a * a; }

bool edges_from(int64_t n, int32_t p, const int32_t *cuts, int32_t ncuts, const char *axis,
                std::vector<int64_t> *e, std::string *err) {
    e->clear();
    if (cuts) {
        if (ncuts < 1) {
            *err = std::string("cut list on axis ") + axis + " needs at least one block";
            return false;
        }
        for (int32_t b = 0; b <= ncuts; ++b) e->push_back(cuts[b]);
        if ((*e)[0] != 0 || (*e)[ncuts] != n) {
            *err = std::string("cut list on axis ") + axis + " must start at 0 and end at n";
            return false;
        }
        for (int32_t b = 0; b < ncuts; ++b)
            if ((*e)[b + 1] <= (*e)[b]) {
                *err = std::string("cut list on axis ") + axis + " must be strictly ascending";
                return false;
            }
        return true;
    }
    if (p < 1 || p > n) {
        char buf[160];
        snprintf(buf, sizeof buf, "cannot split %lld cells on axis %s into %d blocks",
                 (long long)n, axis, p);
        *err = buf;
        return false;
    }
    // balanced split: the first n mod p blocks are one cell longer
    int64_t q = n / p, r = n % p, at = 0;
    e->push_back(0);
    for (int32_t b = 0; b < p; ++b) {
        at += q + (b < r ? 1 : 0);
        e->push_back(at);
    }
    return true;
}

struct Box {
    int64_t lo[3], hi[3];
};

Box tile_box(const HostChare &c, const TileDev &t) {
    Box b;
    b.lo[0] = c.x0 + t.i0;    b.hi[0] = b.lo[0] + t.ni;
    b.lo[1] = c.y0 + t.j0;    b.hi[1] = b.lo[1] + t.nj;
    b.lo[2] = c.z0 + t.k0;    b.hi[2] = b.lo[2] + t.nk;
    return b;
}

// Tiles whose cells a 7-point update of `a` reads, or that read `a`'s cells:
// the same tile, or boxes that touch along one axis and overlap on the other
// two.
bool adjacent_or_same(const Box &a, const Box &b) {
    int overlap = 0, touch = 0;
    for (int d = 0; d < 3; ++d) {
        if (a.lo[d] < b.hi[d] && b.lo[d] < a.hi[d]) ++overlap;
        else if (a.hi[d] == b.lo[d] || b.hi[d] == a.lo[d]) ++touch;
    }
    return overlap == 3 || (overlap == 2 && touch == 1);
}

// split n into parts of at most `cap`, balanced
void balanced_parts(int32_t n, int32_t cap, std::vector<int32_t> *starts, std::vector<int32_t> *lens) {
    int32_t parts = (n + cap - 1) / cap;
    int32_t q = n / parts, r = n % parts, at = 0;
    starts->clear();
    lens->clear();
    for (int32_t b = 0; b < parts; ++b) {
        int32_t l = q + (b < r ? 1 : 0);
        starts->push_back(at);
        lens->push_back(l);
        at += l;
    }
}

}  // namespace

int32_t stage_doubles_for(int32_t nj, int32_t pitch) {
    return round_up((nj + 2) * pitch, 16);     // keep slots 128-byte aligned
}

od_status build_plan(const od_config *cfg, Plan *P, std::string *err) { return build_plan(cfg, P, err, true); }

od_status build_plan(const od_config *cfg, Plan *P, std::string *err, bool fill_gpu) {
    Plan &p = *P;
    p = Plan();
    if (!cfg) { *err = "null config"; return OD_EINVAL; }
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1 || cfg->nx > (1 << 30) || cfg->ny > (1 << 30) ||
        cfg->nz > (1 << 30)) {
        *err = "grid extents must be in [1, 2^30]";
        return OD_EINVAL;
    }
    if (cfg->init_mode != OD_INIT_ZERO_INTERIOR && cfg->init_mode != OD_INIT_UNIFORM) {
        *err = "init_mode must be 0 or 1";
        return OD_EINVAL;
    }
    if (cfg->path < OD_PATH_PER_CHARE || cfg->path > OD_PATH_FUSED_GRAPH) {
        *err = "unknown path";
        return OD_EINVAL;
    }
    if (cfg->pe_threads < 0 || cfg->pe_threads > 64) {
        *err = "pe_threads must be in [0, 64]";
        return OD_EINVAL;
    }
    if (cfg->order < 0 || cfg->order > 3) {
        *err = "order must be 0..3 (bit 0: reverse on odd steps, bit 1: Morton order of the chares)";
        return OD_EINVAL;
    }
    p.threads = cfg->threads ? cfg->threads : 128;
    p.cpt = cfg->cells_per_thread ? cfg->cells_per_thread : 4;
    const bool auto_shape = cfg->threads == 0 && cfg->cells_per_thread == 0;
    p.stages = cfg->stages ? cfg->stages : 4;
    p.tile_y = cfg->tile_y;
    p.tile_z = cfg->tile_z;
    // default: the anchored window -- in 3D two FP64 adds and the rest in
    // the window (202 G updates/s at 512^3 in 4096 chares against 167 for
    // the earlier tail form), in 2D one FP64 add (279 against 252 for one
    // per-cell window add at 32768^2)
    p.amode = cfg->arith >= 0 ? cfg->arith : kDefaultArith;
    if (p.amode > 15) {
        *err = "arith must be in [0, 15] (or -1 for the default)";
        return OD_EINVAL;
    }
    if (p.threads != 128 && p.threads != 256 && p.threads != 512) {
        *err = "threads must be 128, 256 or 512";
        return OD_EINVAL;
    }
    if (!((p.threads == 128 && (p.cpt == 2 || p.cpt == 4 || p.cpt == 8)) ||
          (p.threads == 256 && (p.cpt == 1 || p.cpt == 2 || p.cpt == 4 || p.cpt == 8)) ||
          (p.threads == 512 && (p.cpt == 1 || p.cpt == 2)))) {
        *err = "supported (threads, cells_per_thread): 128 x {2,4,8}, 256 x {1,2,4,8}, 512 x {1,2}";
        return OD_EINVAL;
    }
    if (p.stages < 3 || p.stages > 8) {
        *err = "stages must be in [3, 8]";
        return OD_EINVAL;
    }
    if (p.tile_y < 0 || p.tile_z < 0) {
        *err = "tile sizes must be >= 0";
        return OD_EINVAL;
    }
    if (cfg->stencil != OD_STENCIL_3D7 && cfg->stencil != OD_STENCIL_2D5) {
        *err = "unknown stencil";
        return OD_EINVAL;
    }
    p.stencil = cfg->stencil;
    if (p.stencil == OD_STENCIL_2D5) {
        // A 2D nx x ny grid is laid out as the 3D grid (nx, 1, ny): the 2D rows
        // are the planes the kernels stream, and the (unused) y-ghost rows of
        // every plane keep the 3D layout and I/O kernels valid unchanged.
        if (cfg->nz != 1 || (cfg->cuts_z && cfg->ncuts_z != 1) || (!cfg->cuts_z && cfg->pz > 1)) {
            *err = "the 2D stencil needs nz = 1 and a single block along z";
            return OD_EINVAL;
        }
        p.nx = cfg->nx; p.ny = 1; p.nz = cfg->ny;
        if (!edges_from(cfg->nx, cfg->px, cfg->cuts_x, cfg->ncuts_x, "x", &p.ex, err) ||
            !edges_from(cfg->ny, cfg->py, cfg->cuts_y, cfg->ncuts_y, "y", &p.ez, err))
            return OD_EINVAL;
        p.ey = {0, 1};
    } else {
        p.nx = cfg->nx; p.ny = cfg->ny; p.nz = cfg->nz;
        if (!edges_from(cfg->nx, cfg->px, cfg->cuts_x, cfg->ncuts_x, "x", &p.ex, err) ||
            !edges_from(cfg->ny, cfg->py, cfg->cuts_y, cfg->ncuts_y, "y", &p.ey, err) ||
            !edges_from(cfg->nz, cfg->pz, cfg->cuts_z, cfg->ncuts_z, "z", &p.ez, err))
            return OD_EINVAL;
    }
    // shard of a global grid (all zero: the context is the whole grid)
    const bool shard = cfg->gnx || cfg->gny || cfg->gnz || cfg->gx0 || cfg->gy0 || cfg->gz0;
    if (!shard) {
        p.gnx = p.nx; p.gny = p.ny; p.gnz = p.nz;
    } else if (p.stencil == OD_STENCIL_2D5) {
        if ((cfg->gnz != 0 && cfg->gnz != 1) || cfg->gz0 != 0) {
            *err = "2D shard: gnz must be 1 (or 0) and gz0 0";
            return OD_EINVAL;
        }
        p.gnx = cfg->gnx; p.gny = 1; p.gnz = cfg->gny;
        p.gx0 = cfg->gx0; p.gy0 = 0; p.gz0 = cfg->gy0;
    } else {
        p.gnx = cfg->gnx; p.gny = cfg->gny; p.gnz = cfg->gnz;
        p.gx0 = cfg->gx0; p.gy0 = cfg->gy0; p.gz0 = cfg->gz0;
    }
    if (p.gx0 < 0 || p.gy0 < 0 || p.gz0 < 0 || p.gx0 + p.nx > p.gnx || p.gy0 + p.ny > p.gny ||
        p.gz0 + p.nz > p.gnz) {
        *err = "shard box must lie inside the global grid (gx0 + nx <= gnx, ...)";
        return OD_EINVAL;
    }
    p.px = (int32_t)p.ex.size() - 1;
    p.py = (int32_t)p.ey.size() - 1;
    p.pz = (int32_t)p.ez.size() - 1;
    int64_t nch = (int64_t)p.px * p.py * p.pz;
    if (nch > (1ll << 24)) {
        *err = "more than 2^24 chares";
        return OD_EINVAL;
    }
    if (auto_shape && p.stencil == OD_STENCIL_2D5) {
        // 2D tiles are row segments of up to threads x cpt cells: 128 x 4, or
        // 128 x 2 when every chare row fits in 256 cells
        int64_t wmax = 0;
        for (int64_t e = 1; e < (int64_t)p.ex.size(); ++e) wmax = std::max(wmax, p.ex[e] - p.ex[e - 1]);
        p.threads = 128;
        p.cpt = wmax <= 256 ? 2 : 4;
    } else if (auto_shape) {
        // Score each CTA shape that holds a row of the widest chare by
        //   lanes used (tile cells / CTA cells, over the whole grid)
        //   x (1 - 0.2 / rows per tile)       (the two y-halo rows loaded per plane)
        //   x min(1, tiles / half the resident CTAs)   (too few tiles leave SMs
        //        idle; a GB300 holds about 1280 threads per SM of these
        //        kernels, 152 SMs, and runs well from half of that)
        // and keep 128 x 4 unless another shape scores 10 % higher (measured,
        // fused path: 384^3 in 8 chares 256 x 4 120 vs 103 G updates/s; 150^3
        // in 27 and 200^3 in 64 128 x 2, 70 vs 52 and 97 vs 85; 32^3 and 64^3
        // chares of large grids 128 x 4).
        int64_t wmax = 0;
        for (int64_t e = 1; e < (int64_t)p.ex.size(); ++e) wmax = std::max(wmax, p.ex[e] - p.ex[e - 1]);
        const int32_t shapes[4][2] = {{128, 4}, {128, 2}, {256, 4}, {256, 8}};
        const int32_t tz = p.tile_z > 0 ? p.tile_z : 32;
        double best = -1.0, base = -1.0;
        int pick = -1;
        for (int i = 0; i < 4; ++i) {
            const int64_t cap = (int64_t)shapes[i][0] * shapes[i][1];
            if (cap < wmax || (i == 3 && wmax <= 1024)) continue;  // 256 x 8 only for rows past 1024
            double used = 0.0, cells = 0.0, rows = 0.0, tiles = 0.0;
            for (int64_t a = 1; a < (int64_t)p.ex.size(); ++a)
                for (int64_t b = 1; b < (int64_t)p.ey.size(); ++b)
                    for (int64_t c = 1; c < (int64_t)p.ez.size(); ++c) {
                        const int64_t bx = p.ex[a] - p.ex[a - 1], by = p.ey[b] - p.ey[b - 1],
                                      bz = p.ez[c] - p.ez[c - 1];
                        int64_t nj = std::min<int64_t>(by, cap / bx);
                        if (p.tile_y > 0) nj = std::min<int64_t>(nj, p.tile_y);
                        nj = std::max<int64_t>(nj, 1);
                        const int64_t slabs = (by + nj - 1) / nj, chunks = (bz + std::min<int64_t>(tz, bz) - 1) /
                                                                               std::min<int64_t>(tz, bz);
                        const double v = (double)bx * by * bz;
                        used += v;
                        cells += (double)cap * slabs * bz;  // lanes offered: one CTA plane per slab and plane
                        rows += v * ((double)by / slabs);
                        tiles += (double)slabs * chunks;
                    }
            const double resident = 0.5 * 152.0 * (1280 / shapes[i][0]);
            const double score = used / cells * (1.0 - 0.2 / (rows / used)) *
                                 (fill_gpu ? std::min(1.0, tiles / resident) : 1.0);
            if (i == 0) base = score;
            if (score > best) {
                best = score;
                pick = i;
            }
        }
        if (pick < 0) pick = 3;  // rows past 1024 cells: only 256 x 8 holds them (checked below)
        if (pick != 0 && base >= 0.0 && best < 1.1 * base) pick = 0;
        p.threads = shapes[pick][0];
        p.cpt = shapes[pick][1];
    }
    for (int64_t e = 1; e < (int64_t)p.ex.size() && p.stencil == OD_STENCIL_3D7; ++e)
        if (p.ex[e] - p.ex[e - 1] > (int64_t)p.threads * p.cpt) {
            char buf[200];
            snprintf(buf, sizeof buf,
                     "block row of %lld cells exceeds threads*cells_per_thread = %d; "
                     "use more chares along x or a larger CTA",
                     (long long)(p.ex[e] - p.ex[e - 1]), p.threads * p.cpt);
            *err = buf;
            return OD_EINVAL;
        }

    // chares, x fastest
    p.ch.resize((size_t)nch);
    for (int32_t cz = 0; cz < p.pz; ++cz)
        for (int32_t cy = 0; cy < p.py; ++cy)
            for (int32_t cx = 0; cx < p.px; ++cx) {
                int64_t c = cx + (int64_t)p.px * (cy + (int64_t)p.py * cz);
                HostChare &h = p.ch[(size_t)c];
                h.cx = cx; h.cy = cy; h.cz = cz;
                h.x0 = p.ex[cx]; h.bx = (int32_t)(p.ex[cx + 1] - p.ex[cx]);
                h.y0 = p.ey[cy]; h.by = (int32_t)(p.ey[cy + 1] - p.ey[cy]);
                h.z0 = p.ez[cz]; h.bz = (int32_t)(p.ez[cz + 1] - p.ez[cz]);
                h.pitch = round_up(h.bx + 2, 2);
                h.rows = p.stencil == OD_STENCIL_2D5 ? 1 : h.by + 2;
                h.row0 = p.stencil == OD_STENCIL_2D5 ? 0 : 1;
                h.nbr[OD_FACE_XLO] = cx > 0 ? (int32_t)(c - 1) : -1;
                h.nbr[OD_FACE_XHI] = cx < p.px - 1 ? (int32_t)(c + 1) : -1;
                h.nbr[OD_FACE_YLO] = cy > 0 ? (int32_t)(c - p.px) : -1;
                h.nbr[OD_FACE_YHI] = cy < p.py - 1 ? (int32_t)(c + p.px) : -1;
                h.nbr[OD_FACE_ZLO] = cz > 0 ? (int32_t)(c - (int64_t)p.px * p.py) : -1;
                h.nbr[OD_FACE_ZHI] = cz < p.pz - 1 ? (int32_t)(c + (int64_t)p.px * p.py) : -1;
                const int64_t bx = h.bx, by = h.by, bz = h.bz;
                int64_t fs[6] = {by * bz, by * bz, bx * bz, bx * bz, bx * by, bx * by};
                if (p.stencil == OD_STENCIL_2D5) fs[OD_FACE_YLO] = fs[OD_FACE_YHI] = 0;  // no y faces in 2D
                if (fs[0] + fs[1] + fs[2] + fs[3] + fs[4] + fs[5] > 0x7fffffffll) {
                    *err = "a block's faces exceed 2^31 cells; use more blocks";
                    return OD_EINVAL;
                }
                h.foff[0] = 0;
                for (int f = 0; f < 6; ++f) h.foff[f + 1] = h.foff[f] + (int32_t)fs[f];
                for (int f = 0; f < 6; ++f) {
                    if (h.nbr[f] >= 0) p.face_internal += fs[f];
                    else p.face_dirichlet += fs[f];
                }
            }
    p.cells = p.nx * p.ny * p.nz;
    p.bytes_per_step = 16.0 * (double)p.cells + 16.0 * (double)p.face_internal +
                       8.0 * (double)p.face_dirichlet;

    // tiles: full rows, balanced row slabs and plane chunks
    std::vector<int32_t> js, jl, ks, kl;
    int32_t max_stage = 0;
    for (size_t c = 0; c < p.ch.size() && p.stencil == OD_STENCIL_2D5; ++c) {
        // 2D: tiles of one row segment (x range) x a run of rows (planes); the
        // segment start is even so its bulk copy stays 16-byte aligned
        HostChare &h = p.ch[c];
        int32_t cap = p.threads * p.cpt;
        if (p.tile_y > 0) cap = std::min(cap, p.tile_y);  // tile_y caps the segment for 2D
        const int32_t nseg = (h.bx + cap - 1) / cap;
        const int32_t w = round_up((h.bx + nseg - 1) / nseg, 2);
        int32_t tz = p.tile_z > 0 ? p.tile_z : 32;
        tz = std::min(tz, h.bz);
        balanced_parts(h.bz, tz, &ks, &kl);
        h.tile_begin = (int32_t)p.tiles.size();
        h.ti.clear();
        for (int32_t i0 = 0; i0 < h.bx; i0 += w) h.ti.push_back(i0);
        h.tj.assign(1, 0);
        h.tk = ks;
        for (size_t a = 0; a < ks.size(); ++a)
            for (int32_t i0 = 0; i0 < h.bx; i0 += w) {
                TileDev t;
                memset(&t, 0, sizeof t);
                t.c = (int32_t)c;
                t.j0 = 0; t.nj = 1;
                t.k0 = ks[a]; t.nk = kl[a];
                t.i0 = i0; t.ni = std::min(w, h.bx - i0);
                p.tiles.push_back(t);
                max_stage = std::max(max_stage, round_up(t.ni + 4, 16));
                p.max_nj = std::max(p.max_nj, t.ni);
                p.max_nk = std::max(p.max_nk, t.nk);
                if (p.tiles.size() > (size_t)0x7fffffff) {
                    *err = "too many tiles";
                    return OD_EINVAL;
                }
            }
        h.tile_end = (int32_t)p.tiles.size();
    }
    for (size_t c = 0; c < p.ch.size() && p.stencil == OD_STENCIL_3D7; ++c) {
        HostChare &h = p.ch[c];
        int32_t nj_cap = (p.threads * p.cpt) / h.bx;
        if (p.tile_y > 0) nj_cap = std::min(nj_cap, p.tile_y);
        nj_cap = std::max(1, std::min(nj_cap, h.by));
        int32_t tz = p.tile_z > 0 ? p.tile_z : 32;
        tz = std::min(tz, h.bz);
        balanced_parts(h.by, nj_cap, &js, &jl);
        balanced_parts(h.bz, tz, &ks, &kl);
        h.tile_begin = (int32_t)p.tiles.size();
        h.ti.assign(1, 0);
        h.tj = js;
        h.tk = ks;
        for (size_t a = 0; a < ks.size(); ++a)
            for (size_t b = 0; b < js.size(); ++b) {
                TileDev t;
                memset(&t, 0, sizeof t);
                t.c = (int32_t)c;
                t.j0 = js[b]; t.nj = jl[b];
                t.k0 = ks[a]; t.nk = kl[a];
                t.i0 = 0; t.ni = h.bx;
                p.tiles.push_back(t);
                max_stage = std::max(max_stage, stage_doubles_for(t.nj, h.pitch));
                p.max_nj = std::max(p.max_nj, t.nj);
                p.max_nk = std::max(p.max_nk, t.nk);
                if (p.tiles.size() > (size_t)0x7fffffff) {
                    *err = "too many tiles";
                    return OD_EINVAL;
                }
            }
        h.tile_end = (int32_t)p.tiles.size();
    }
    p.stage_doubles = max_stage;
    // the tile kernels pack a cell's ring offset into 16 bits and its tile row
    // into 11 bits
    if (p.stage_doubles >= 65536 || (p.stencil == OD_STENCIL_3D7 && p.max_nj > 2048)) {
        *err = "tile too large for the kernels' cell encoding; lower tile_y";
        return OD_EINVAL;
    }
    int64_t smem = kSmemHeader + (int64_t)p.stages * p.stage_doubles * 8;
    if (smem > kMaxSmem) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "tile needs %lld bytes of shared memory (> %d); lower tile_y, "
                 "cells_per_thread or stages",
                 (long long)smem, kMaxSmem);
        *err = buf;
        return OD_EINVAL;
    }
    p.smem_bytes = (int32_t)smem;

    // dependency lists (tiles of the chare itself and its six neighbours):
    // per axis only the candidate's tiles within one cell of the tile's range
    // can touch it, found by bisection over the chare's tile starts
    p.dep_ptr.assign(p.tiles.size() + 1, 0);
    p.dep_idx.clear();
    for (size_t ti = 0; ti < p.tiles.size(); ++ti) {
        const TileDev &t = p.tiles[ti];
        const HostChare &h = p.ch[(size_t)t.c];
        Box a = tile_box(h, t);
        int32_t cand[7] = {t.c, h.nbr[0], h.nbr[1], h.nbr[2], h.nbr[3], h.nbr[4], h.nbr[5]};
        for (int q = 0; q < 7; ++q) {
            if (cand[q] < 0) continue;
            const HostChare &g = p.ch[(size_t)cand[q]];
            const std::vector<int32_t> *st[3] = {&g.ti, &g.tj, &g.tk};
            const int64_t org[3] = {g.x0, g.y0, g.z0};
            size_t lo[3], hi[3];
            for (int d = 0; d < 3; ++d) {
                // tiles whose start is <= a.hi (chare-local), from the last one starting <= a.lo - 1
                const std::vector<int32_t> &v = *st[d];
                const int64_t l = a.lo[d] - 1 - org[d], r = a.hi[d] - org[d];
                size_t first = (size_t)(std::upper_bound(v.begin(), v.end(), l) - v.begin());
                lo[d] = first > 0 ? first - 1 : 0;
                hi[d] = (size_t)(std::upper_bound(v.begin(), v.end(), r) - v.begin());
            }
            for (size_t e = lo[2]; e < hi[2]; ++e)
                for (size_t b = lo[1]; b < hi[1]; ++b)
                    for (size_t i = lo[0]; i < hi[0]; ++i) {
                        const int32_t u = g.tile_begin + (int32_t)((e * g.tj.size() + b) * g.ti.size() + i);
                        if (adjacent_or_same(a, tile_box(g, p.tiles[(size_t)u]))) p.dep_idx.push_back(u);
                    }
        }
        p.dep_ptr[ti + 1] = (int32_t)p.dep_idx.size();
    }
    p.order.resize(p.tiles.size());
    for (size_t ti = 0; ti < p.tiles.size(); ++ti) p.order[ti] = (int32_t)ti;
    if (cfg->order & 2) {
        // Z-order (Morton) over the chare grid: chares that are close in all
        // three axes run close in time, so a face written by one is more
        // likely still in L2 when its neighbour reads it; a chare's own tiles
        // keep their order
        auto spread = [](uint64_t v) {  // bits of a 21-bit value to every third bit
            v &= 0x1fffffull;
            v = (v | v << 32) & 0x1f00000000ffffull;
            v = (v | v << 16) & 0x1f0000ff0000ffull;
            v = (v | v << 8) & 0x100f00f00f00f00full;
            v = (v | v << 4) & 0x10c30c30c30c30c3ull;
            v = (v | v << 2) & 0x1249249249249249ull;
            return v;
        };
        std::vector<uint64_t> key(p.tiles.size());
        for (size_t ti = 0; ti < p.tiles.size(); ++ti) {
            const HostChare &h = p.ch[(size_t)p.tiles[ti].c];
            key[ti] = spread((uint64_t)h.cx) | spread((uint64_t)h.cy) << 1 | spread((uint64_t)h.cz) << 2;
        }
        std::stable_sort(p.order.begin(), p.order.end(),
                         [&](int32_t a, int32_t b) { return key[(size_t)a] < key[(size_t)b]; });
    }

    // arena layout
    size_t at = 0;
    auto take = [&](size_t bytes) {
        size_t o = at;
        at = align_up(at + bytes, kAlign);
        return o;
    };
    p.off_err = take(sizeof(ErrDev));
    p.off_queue = take(64);
    p.off_epoch = take(p.tiles.size() * sizeof(int32_t));
    p.off_chares = take(p.ch.size() * sizeof(ChareDev));
    p.off_tiles = take(p.tiles.size() * sizeof(TileDev));
    p.off_dep_ptr = take(p.dep_ptr.size() * sizeof(int32_t));
    p.off_dep_idx = take(std::max<size_t>(1, p.dep_idx.size()) * sizeof(int32_t));
    p.off_order = take(p.order.size() * sizeof(int32_t));
    for (auto &h : p.ch) {
        size_t a_bytes = (size_t)(h.bz + 2) * (size_t)h.rows * (size_t)h.pitch * 8;
        size_t f_bytes = (size_t)h.foff[6] * 8;
        for (int s = 0; s < 2; ++s) h.offA[s] = take(a_bytes);
        h.offSend = take(f_bytes);
        h.offRecv[0] = take(f_bytes);
        h.offRecv[1] = take(f_bytes);
    }
    p.arena_bytes = at;
    return OD_OK;
}

void plan_info(const Plan &p, od_plan_info *o) {
    memset(o, 0, sizeof *o);
    o->nchares = (int64_t)p.ch.size();
    o->ntiles = (int64_t)p.tiles.size();
    o->cells = p.cells;
    o->face_cells_internal = p.face_internal;
    o->face_cells_dirichlet = p.face_dirichlet;
    o->arena_bytes = p.arena_bytes;
    o->bytes_per_step = p.bytes_per_step;
    o->tile_y = p.max_nj;
    o->tile_z = p.max_nk;
    o->arith = p.amode;
    o->threads = p.threads;
    o->cells_per_thread = p.cpt;
    o->stages = p.stages;
    o->smem_bytes = p.smem_bytes;
}

}  // namespace od
