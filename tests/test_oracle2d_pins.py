"""Pins for the 2D 5-point oracle (the paper's own Jacobi2D application):
closed forms, invariants, a hand value, an eigenmode, brute force by an
independent NumPy sweep, and decomposition invariance."""
import math

import numpy as np
import pytest

import oracle


def test_init_2d_matches_generator():
    P = oracle.init_padded_2d(7, 5, seed=9, init_mode=1)
    sx = 7 + 2
    for (y, x) in [(0, 0), (3, 4), (6, 8), (2, 1)]:
        assert P[y, x] == oracle.uniform(9, x + sx * y)
    P0 = oracle.init_padded_2d(7, 5, seed=9, init_mode=0)
    assert np.all(P0[1:-1, 1:-1] == 0.0)
    assert np.array_equal(P0[0], P[0]) and np.array_equal(P0[:, -1], P[:, -1])


@pytest.mark.parametrize("c", [0.75, 0.3125, 1.0, 0.0, 12345 * 2.0**-20])
def test_constant_field_fixed_point(c):
    P = np.full((7, 9), c)
    assert np.array_equal(oracle.sweep_2d(P, 9), P)


@pytest.mark.parametrize("coef", [(3.0, 1.0, 2.0), (0.5, 0.25, -0.75), (-7.0, 4.0, 0.0)])
def test_affine_field_fixed_point(coef):
    # u = a + b x + c y is discrete-harmonic for the 5-point Laplacian
    a, b, c = coef
    nx, ny = 9, 7
    y, x = np.meshgrid(np.arange(ny + 2), np.arange(nx + 2), indexing="ij")
    P = a + b * x + c * y
    assert np.array_equal(oracle.sweep_2d(P, 6), P)
    assert np.array_equal(oracle.sweep_decomposed_2d(P, [0, 4, 9], [0, 1, 3, 7], 6), P)


def test_two_by_two_closed_form():
    # 2x2 interior at 0 in a shell of 1: u <- (2 + 2u)/4, u_n = 1 - 2^-n
    P = np.ones((4, 4))
    P[1:3, 1:3] = 0.0
    for n in [0, 1, 2, 7, 30, 51]:
        assert np.all(oracle.sweep_2d(P, n)[1:3, 1:3] == 1.0 - 2.0**-n), n


def test_single_cell_hand_value():
    # (0.5 + 0.25 + 1 + 4.25) / 4 = 6 / 4 = 1.5
    P = np.zeros((3, 3))
    P[1, 0], P[1, 2], P[0, 1], P[2, 1] = 0.5, 0.25, 1.0, 4.25
    assert oracle.sweep_2d(P, 1)[1, 1] == 1.5


def test_summation_order():
    P = np.zeros((3, 3))
    P[1, 0], P[1, 2], P[0, 1], P[2, 1] = 1e16, 1.0, -1e16, 3.0
    s = 1e16 + 1.0
    s = s + -1e16
    s = s + 3.0
    assert oracle.sweep_2d(P, 1)[1, 1] == s / 4.0
    assert s / 4.0 != (1e16 + -1e16 + 1.0 + 3.0) / 4.0


def test_sine_mode_decay():
    nx, ny = 14, 11
    for (p, q) in [(1, 1), (3, 2), (5, 7)]:
        y, x = np.meshgrid(np.arange(ny + 2), np.arange(nx + 2), indexing="ij")
        P = np.sin(p * np.pi * x / (nx + 1)) * np.sin(q * np.pi * y / (ny + 1))
        P[0, :] = P[-1, :] = 0.0
        P[:, 0] = P[:, -1] = 0.0
        lam = (math.cos(p * math.pi / (nx + 1)) + math.cos(q * math.pi / (ny + 1))) / 2.0
        n = 25
        Q = oracle.sweep_2d(P, n)
        assert np.max(np.abs(Q - P * lam**n)) <= 200 * n * np.finfo(float).eps


def numpy_sweep_2d(P, iters):
    u = P.copy()
    for _ in range(iters):
        v = u.copy()
        s = u[1:-1, :-2] + u[1:-1, 2:]
        s = s + u[:-2, 1:-1]
        s = s + u[2:, 1:-1]
        v[1:-1, 1:-1] = s / 4.0
        u = v
    return u


@pytest.mark.parametrize("dims", [(32, 32), (17, 5), (1, 1), (1, 9), (40, 3)])
@pytest.mark.parametrize("mode", [0, 1])
def test_brute_force(dims, mode):
    nx, ny = dims
    P = oracle.init_padded_2d(nx, ny, seed=4, init_mode=mode)
    for iters in (0, 1, 5, 12):
        assert np.array_equal(oracle.sweep_2d(P, iters), numpy_sweep_2d(P, iters))


def test_decomposed_equals_monolithic():
    rng = np.random.default_rng(2)
    for trial in range(15):
        nx, ny = (int(v) for v in rng.integers(1, 30, 2))
        P = oracle.init_padded_2d(nx, ny, seed=50 + trial, init_mode=trial % 2)
        def cuts(n):
            p = int(rng.integers(1, min(n, 6) + 1))
            inner = sorted(rng.choice(np.arange(1, n), size=p - 1, replace=False)) if p > 1 else []
            return [0] + [int(v) for v in inner] + [n]
        ex, ey = cuts(nx), cuts(ny)
        iters = int(rng.integers(0, 9))
        assert np.array_equal(oracle.sweep_2d(P, iters), oracle.sweep_decomposed_2d(P, ex, ey, iters))


def test_threads_do_not_change_bits():
    P = oracle.init_padded_2d(70, 53, seed=3, init_mode=1)
    assert np.array_equal(oracle.sweep_2d(P, 7, threads=1), oracle.sweep_2d(P, 7, threads=4))


def test_point_matches_sweep():
    nx, ny, seed, mode, iters = 37, 29, 6, 1, 11
    full = oracle.solve_2d(nx, ny, seed, mode, iters)
    for (x, y) in [(0, 0), (nx - 1, ny - 1), (18, 0), (5, 27), (20, 14)]:
        assert oracle.point_2d(nx, ny, seed, mode, iters, x, y) == full[x + nx * y]
