"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no stencil arithmetic and imports neither the CUDA library
nor the oracle: it only draws the *descriptions* of workloads (block edges,
request streams) that both sides then consume.  The initial field itself is
not drawn here: it is a counter-based SplitMix64 function of the global cell
index that each side implements on its own (device init kernel, C oracle).

Workloads (3D 7-point FP64 Jacobi, the paper's Jacobi proxy of Sec. V in 3D):

* ``PARITY_64``    64^3 split 2x2x2 into 8 blocks of 32^3; interior 0, shell
                   U[0,1); 10 iterations; compared bit for bit.
* ``ODF_SWEEP_512`` 512^3, 100 iterations, cubic blocks 512^3 .. 32^3
                   (1, 8, 64, 512, 4096 blocks); every cell U[0,1).
* ``UNEVEN_768``   768x512x512 cut at seeded random positions, block edges in
                   [24, 160] (about 300 blocks of uneven volume); 200 iterations.
* serving stream   Poisson arrivals of independent cubic jobs, edge log-uniform
                   in [64, 384], blocks per job in {8, 27, 64, 216}, iterations
                   uniform in [10, 200].
* ``CEILING_1024`` 1024^3 in 4096 blocks of 64^3, 50 iterations.

2D 5-point FP64 Jacobi (the paper's Jacobi2D application, Sec. V):

* ``JACOBI2D_32768`` the paper's per-GPU base domain 32768 x 32768, 100
                   iterations, every cell U[0,1), split into px x py blocks
                   with px*py = ODF (px = 2^ceil(log2(ODF)/2), py = ODF/px).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# init_mode values understood by both sides
INIT_ZERO_INTERIOR = 0   # interior 0, Dirichlet shell U[0,1)
INIT_UNIFORM = 1         # every cell (interior and shell) U[0,1)


def uneven_edges(n: int, seed: int, lo: int = 24, hi: int = 160) -> list[int]:
    """Block edges along one axis for an uneven (AMR-like) decomposition.

    Draws block lengths one by one from their own PCG64 stream: while the
    remaining length R exceeds ``hi`` the next length is uniform on the
    integers [lo, min(hi, R - lo)], so that what remains stays >= lo; the last
    block takes the remainder, which then lies in [lo, hi].  Returns the
    ascending cut positions 0 = e_0 < e_1 < ... < e_p = n.
    """
    if n < lo:
        raise ValueError("axis shorter than the minimum block")
    if hi < 2 * lo:
        raise ValueError("need hi >= 2*lo so the remainder rule always works")
    rng = np.random.Generator(np.random.PCG64(seed))
    edges = [0]
    rem = n
    while rem > hi:
        e = int(rng.integers(lo, min(hi, rem - lo) + 1))
        edges.append(edges[-1] + e)
        rem -= e
    edges.append(n)
    return edges


@dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    iters: int
    seed: int
    init_mode: int
    split: tuple[int, int, int] | None = None           # uniform px, py, pz
    cuts: tuple[list[int], list[int], list[int]] | None = None  # explicit edges
    stencil: str = "3d7"                                 # "3d7" or "2d5" (nz = 1)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nchares(self) -> int:
        if self.cuts is not None:
            return (len(self.cuts[0]) - 1) * (len(self.cuts[1]) - 1) * (len(self.cuts[2]) - 1)
        px, py, pz = self.split
        return px * py * pz


def parity_64() -> Workload:
    return Workload("jacobi3d-64^3-2x2x2", 64, 64, 64, 10, 1, INIT_ZERO_INTERIOR, split=(2, 2, 2))


def odf_sweep_512(odf: int, iters: int = 100) -> Workload:
    p = round(odf ** (1.0 / 3.0))
    if p ** 3 != odf:
        raise ValueError("ODF must be a perfect cube (1, 8, 64, 512, 4096)")
    return Workload(f"jacobi3d-512^3-odf{odf}", 512, 512, 512, iters, 2, INIT_UNIFORM,
                    split=(p, p, p))


# Axis streams 25/26/27 give 10 x 5 x 6 = 300 blocks: the "about 300" of the
# uneven workload (the expected count with mean edge 92 is ~260).
UNEVEN_AXIS_SEEDS = (25, 26, 27)


def uneven_768(iters: int = 200) -> Workload:
    sx, sy, sz = UNEVEN_AXIS_SEEDS
    cx = uneven_edges(768, sx)
    cy = uneven_edges(512, sy)
    cz = uneven_edges(512, sz)
    return Workload("jacobi3d-768x512x512-uneven", 768, 512, 512, iters, 3, INIT_UNIFORM,
                    cuts=(cx, cy, cz))


def ceiling_1024(iters: int = 50) -> Workload:
    return Workload("jacobi3d-1024^3-odf4096", 1024, 1024, 1024, iters, 7, INIT_UNIFORM,
                    split=(16, 16, 16))


def jacobi2d_32768(odf: int, iters: int = 100, edge: int = 32768) -> Workload:
    """The paper's Jacobi2D base domain on one GPU, in ODF blocks."""
    if odf < 1 or odf & (odf - 1):
        raise ValueError("ODF must be a power of two")
    lg = odf.bit_length() - 1
    px = 1 << ((lg + 1) // 2)
    py = odf // px
    return Workload(f"jacobi2d-{edge}^2-odf{odf}", edge, edge, 1, iters, 9, INIT_UNIFORM,
                    split=(px, py, 1), stencil="2d5")


@dataclass(frozen=True)
class Job:
    job_id: int
    arrival_s: float
    edge: int
    p: int          # blocks per axis (ODF = p^3)
    iters: int
    seed: int

    @property
    def cells(self) -> int:
        return self.edge ** 3

    @property
    def updates(self) -> int:
        return self.cells * self.iters


def serving_stream(n_jobs: int, rate_per_s: float, seed: int = 6,
                   edge_lo: int = 64, edge_hi: int = 384,
                   odfs: tuple[int, ...] = (8, 27, 64, 216),
                   iters_lo: int = 10, iters_hi: int = 200) -> list[Job]:
    """Poisson request stream of independent Jacobi solves.

    Inter-arrival gaps are exponential with mean 1/rate; each job's cubic
    edge is round(exp(U[ln lo, ln hi])); blocks per job uniform over ``odfs``
    (cubes, split per axis as evenly as possible); iterations uniform on the
    integers [iters_lo, iters_hi]; each job gets its own field seed.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    jobs = []
    t = 0.0
    for i in range(n_jobs):
        t += float(rng.exponential(1.0 / rate_per_s))
        edge = int(round(math.exp(rng.uniform(math.log(edge_lo), math.log(edge_hi)))))
        odf = int(odfs[int(rng.integers(0, len(odfs)))])
        p = round(odf ** (1.0 / 3.0))
        iters = int(rng.integers(iters_lo, iters_hi + 1))
        jseed = int(rng.integers(1, 2**62))
        jobs.append(Job(i, t, edge, p, iters, jseed))
    return jobs
