"""Pins for the CPU oracle: facts the mathematics or published definitions fix.

Each test checks the oracle against something other than its own formula:
published generator outputs, closed forms, exact invariants, a hand-computed
value, an eigenmode decay rate, brute force by an independent NumPy sweep, and
the decomposition invariance the method promises (an overdecomposed run must
give exactly the undecomposed answer).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2605_12734_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore")


# ---------------------------------------------------------------- generator

def test_splitmix64_published_sequence():
    # First five outputs of SplitMix64 seeded with 1234567, as published with
    # the generator's reference description (Steele, Lea & Flood 2014 /
    # Vigna's splitmix64.c); widely reproduced as a test vector.
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [oracle.splitmix64(1234567, i) for i in range(5)] == want


def test_uniform_is_top53_bits_and_in_unit_interval():
    for seed in (0, 1, 2**63 + 5):
        for i in range(200):
            u = oracle.uniform(seed, i)
            assert 0.0 <= u < 1.0
            assert u == (oracle.splitmix64(seed, i) >> 11) * 2.0**-53
    us = np.array([oracle.uniform(7, i) for i in range(20000)])
    assert abs(us.mean() - 0.5) < 0.01
    assert abs(us.var() - 1.0 / 12.0) < 0.005


def test_init_modes_shell_and_interior():
    P0 = oracle.init_padded(5, 4, 3, seed=11, init_mode=0)
    P1 = oracle.init_padded(5, 4, 3, seed=11, init_mode=1)
    inner = (slice(1, -1),) * 3
    assert np.all(P0[inner] == 0.0)
    assert np.all(P1[inner] > 0.0) or np.count_nonzero(P1[inner]) == P1[inner].size - 1
    shell = np.ones_like(P0, dtype=bool)
    shell[inner] = False
    assert np.array_equal(P0[shell], P1[shell])
    # cell value = uniform(seed, padded linear index)
    nz, ny, nx = P1.shape
    for (z, y, x) in [(0, 0, 0), (1, 2, 3), (4, 5, 6), (2, 3, 1)]:
        assert P1[z, y, x] == oracle.uniform(11, x + nx * (y + ny * z))


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("c", [0.75, 0.3125, 12345 * 2.0**-20, 1.0, 0.0])
@pytest.mark.parametrize("dims", [(6, 5, 4), (9, 3, 7)])
def test_constant_field_is_fixed_point_bitexact(c, dims):
    nx, ny, nz = dims
    P = np.full((nz + 2, ny + 2, nx + 2), c)
    Q = oracle.sweep(P, 7)
    assert np.array_equal(Q, P)


def test_constant_field_arbitrary_value_within_one_ulp():
    rng = np.random.default_rng(0)
    for c in rng.uniform(0, 1, 50):
        P = np.full((5, 5, 5), c)
        Q = oracle.sweep(P, 1)
        assert np.all(np.abs(Q - c) <= np.spacing(c))


@pytest.mark.parametrize("coef", [(3.0, 1.0, 2.0, -1.0), (0.5, 0.25, -0.75, 1.5), (-7.0, 4.0, 0.0, 3.0)])
def test_affine_field_is_fixed_point_bitexact(coef):
    # u = a + b x + c y + d z is discrete-harmonic: the six neighbours sum to
    # 6u exactly (small dyadic values), so one step returns u.  Unlike a
    # constant field this breaks for a wrong offset or a swapped axis.
    a, b, c, d = coef
    nx, ny, nz = 7, 5, 6
    z, y, x = np.meshgrid(np.arange(nz + 2), np.arange(ny + 2), np.arange(nx + 2), indexing="ij")
    P = a + b * x + c * y + d * z
    Q = oracle.sweep(P, 5)
    assert np.array_equal(Q, P)
    ex, ey, ez = [0, 3, 7], [0, 1, 5], [0, 2, 4, 6]
    Qd = oracle.sweep_decomposed(P, ex, ey, ez, 5)
    assert np.array_equal(Qd, P)


def test_two_cubed_closed_form():
    # 2x2x2 interior at 0 inside a shell of 1: every cell has three shell
    # neighbours and three interior neighbours, all equal by symmetry, so
    # u <- (3 + 3u)/6 and u_n = 1 - 2^-n exactly while 1 - 2^-n fits.
    P = np.ones((4, 4, 4))
    P[1:3, 1:3, 1:3] = 0.0
    for n in [0, 1, 2, 3, 10, 30, 50, 51]:
        Q = oracle.sweep(P, n)
        assert np.all(Q[1:3, 1:3, 1:3] == 1.0 - 2.0**-n), n


def test_single_cell_hand_value():
    # One unknown with six dyadic shell neighbours:
    # (0.5 + 0.25 + 1 + 2 + 0.125 + 4) / 6 = 7.875 / 6 = 1.3125 exactly.
    P = np.zeros((3, 3, 3))
    P[1, 1, 0] = 0.5    # x-
    P[1, 1, 2] = 0.25   # x+
    P[1, 0, 1] = 1.0    # y-
    P[1, 2, 1] = 2.0    # y+
    P[0, 1, 1] = 0.125  # z-
    P[2, 1, 1] = 4.0    # z+
    for n in (1, 2, 5):
        assert oracle.sweep(P, n)[1, 1, 1] == 1.3125


def test_single_cell_summation_order():
    # Values chosen so the fixed left-to-right order x-,x+,y-,y+,z-,z+ gives a
    # different double than other orders: (((((1e16 + 1) + 1) - 1e16) ...
    P = np.zeros((3, 3, 3))
    P[1, 1, 0], P[1, 1, 2], P[1, 0, 1], P[1, 2, 1], P[0, 1, 1], P[2, 1, 1] = \
        1e16, 1.0, 1.0, -1e16, 3.0, 2.0
    s = 1e16 + 1.0
    s = s + 1.0
    s = s + -1e16
    s = s + 3.0
    s = s + 2.0
    want = s / 6.0
    alt = ((1e16 + -1e16) + 1.0 + 1.0 + 3.0 + 2.0) / 6.0
    assert want != alt
    assert oracle.sweep(P, 1)[1, 1, 1] == want


def test_sine_mode_decays_at_eigenvalue():
    # Shell 0 and interior sin(p pi x/(NX+1)) sin(q pi y/(NY+1)) sin(r pi z/(NZ+1))
    # is an eigenvector of the Jacobi operator with eigenvalue
    # (cos(p pi/(NX+1)) + cos(q pi/(NY+1)) + cos(r pi/(NZ+1))) / 3.
    nx, ny, nz = 12, 9, 10
    for (p, q, r) in [(1, 1, 1), (2, 3, 1), (5, 2, 4)]:
        z, y, x = np.meshgrid(np.arange(nz + 2), np.arange(ny + 2), np.arange(nx + 2), indexing="ij")
        P = (np.sin(p * np.pi * x / (nx + 1)) * np.sin(q * np.pi * y / (ny + 1))
             * np.sin(r * np.pi * z / (nz + 1)))
        P[0, :, :] = P[-1, :, :] = 0.0
        P[:, 0, :] = P[:, -1, :] = 0.0
        P[:, :, 0] = P[:, :, -1] = 0.0
        lam = (math.cos(p * math.pi / (nx + 1)) + math.cos(q * math.pi / (ny + 1))
               + math.cos(r * math.pi / (nz + 1))) / 3.0
        n = 20
        Q = oracle.sweep(P, n)
        want = P * lam**n
        assert np.max(np.abs(Q - want)) <= 200 * n * np.finfo(float).eps * np.max(np.abs(P))


# ---------------------------------------------------------------- brute force

def numpy_sweep(P, iters):
    """Independent whole-array Jacobi sweep (NumPy slices, same summation
    order), used as brute force against the C oracle."""
    u = P.copy()
    for _ in range(iters):
        v = u.copy()
        c = (slice(1, -1),) * 3
        s = u[1:-1, 1:-1, :-2] + u[1:-1, 1:-1, 2:]
        s = s + u[1:-1, :-2, 1:-1]
        s = s + u[1:-1, 2:, 1:-1]
        s = s + u[:-2, 1:-1, 1:-1]
        s = s + u[2:, 1:-1, 1:-1]
        v[c] = s / 6.0
        u = v
    return u


@pytest.mark.parametrize("dims", [(16, 16, 16), (5, 11, 3), (1, 1, 1), (2, 9, 1), (13, 2, 7)])
@pytest.mark.parametrize("mode", [0, 1])
def test_oracle_matches_numpy_brute_force(dims, mode):
    nx, ny, nz = dims
    P = oracle.init_padded(nx, ny, nz, seed=5, init_mode=mode)
    for iters in (0, 1, 4, 9):
        assert np.array_equal(oracle.sweep(P, iters), numpy_sweep(P, iters))


def test_threads_do_not_change_bits():
    P = oracle.init_padded(20, 17, 23, seed=9, init_mode=1)
    a = oracle.sweep(P, 6, threads=1)
    b = oracle.sweep(P, 6, threads=4)
    assert np.array_equal(a, b)


# ---------------------------------------------------------------- decomposition

def test_split_balanced():
    assert list(oracle.split(64, 2)) == [0, 32, 64]
    assert list(oracle.split(100, 6)) == [0, 17, 34, 51, 68, 84, 100]
    assert list(oracle.split(7, 7)) == list(range(8))
    assert list(oracle.split(512, 16)) == list(range(0, 513, 32))
    with pytest.raises(ValueError):
        oracle.split(3, 4)


def _random_edges(rng, n, pmax):
    p = int(rng.integers(1, min(n, pmax) + 1))
    inner = sorted(rng.choice(np.arange(1, n), size=p - 1, replace=False)) if p > 1 else []
    return [0] + [int(v) for v in inner] + [n]


def test_decomposed_equals_monolithic_config1():
    w = inputs.parity_64()
    P = oracle.init_padded(w.nx, w.ny, w.nz, w.seed, w.init_mode)
    mono = oracle.sweep(P, w.iters)
    e = oracle.split(64, 2)
    dec = oracle.sweep_decomposed(P, e, e, e, w.iters)
    assert np.array_equal(mono, dec)


def test_decomposed_equals_monolithic_random_cuts():
    rng = np.random.default_rng(1)
    for trial in range(12):
        nx, ny, nz = (int(v) for v in rng.integers(1, 14, 3))
        P = oracle.init_padded(nx, ny, nz, seed=100 + trial, init_mode=trial % 2)
        ex, ey, ez = (_random_edges(rng, n, 5) for n in (nx, ny, nz))
        iters = int(rng.integers(0, 8))
        assert np.array_equal(oracle.sweep(P, iters), oracle.sweep_decomposed(P, ex, ey, ez, iters)), \
            (nx, ny, nz, ex, ey, ez, iters)


def test_decomposed_one_wide_blocks():
    nx, ny, nz = 6, 4, 5
    P = oracle.init_padded(nx, ny, nz, seed=3, init_mode=1)
    ex, ey, ez = list(range(nx + 1)), list(range(ny + 1)), list(range(nz + 1))
    assert np.array_equal(oracle.sweep(P, 5), oracle.sweep_decomposed(P, ex, ey, ez, 5))


# ---------------------------------------------------------------- point cone

def test_point_matches_full_sweep():
    nx, ny, nz, seed, mode, iters = 21, 18, 15, 4, 1, 7
    full = oracle.solve(nx, ny, nz, seed, mode, iters)
    rng = np.random.default_rng(3)
    pts = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (10, 0, 7), (3, 17, 14)]
    pts += [tuple(int(v) for v in (rng.integers(0, nx), rng.integers(0, ny), rng.integers(0, nz)))
            for _ in range(10)]
    for (x, y, z) in pts:
        assert oracle.point(nx, ny, nz, seed, mode, iters, x, y, z) == full[x + nx * (y + ny * z)]
    # iters larger than the box: the cone is clipped everywhere
    full = oracle.solve(6, 5, 4, 8, 0, 11)
    for (x, y, z) in [(0, 0, 0), (5, 4, 3), (2, 2, 2)]:
        assert oracle.point(6, 5, 4, 8, 0, 11, x, y, z) == full[x + 6 * (y + 5 * z)]
