"""The kernels' integer-pipe binary64 routines (division by 6, addition) run on
the host through od_arith_host and must equal IEEE round-to-nearest results
(numpy on this CPU) bit for bit, on random, structured and special inputs."""
import numpy as np
import pytest

from paper_2605_12734_gb300 import build as od_build


@pytest.fixture(scope="module")
def od():
    od_build.build()
    import paper_2605_12734_gb300 as pkg
    return pkg


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def same(got, want):
    g, w = bits(got), bits(want)
    nan = np.isnan(want)
    ok = (g == w) | (nan & np.isnan(got))
    if not ok.all():
        i = int(np.flatnonzero(~ok)[0])
        raise AssertionError(f"{(~ok).sum()} mismatches; first input index {i}: got {got[i]!r} want {want[i]!r}")


def from_bits(u):
    return np.asarray(u, dtype=np.uint64).view(np.float64)


def positive_normals(rng, n, emin=1, emax=2046):
    e = rng.integers(emin, emax + 1, n, dtype=np.uint64)
    m = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    return from_bits((e << np.uint64(52)) | m)


SPECIALS = np.array([0.0, -0.0, 1.0, -1.0, 6.0, 3.0, 0.5, np.inf, -np.inf, np.nan,
                     5e-324, 2.2250738585072014e-308, 2.225073858507201e-308, 1.7976931348623157e308,
                     -2.5, 1e-310, 4.4e-308, 1.3e-307, 0.1, 1 / 3, 2 / 3], dtype=np.float64)


def test_div6_random_unit_interval(od):
    rng = np.random.default_rng(1)
    a = rng.random(2_000_000) * 6.0
    same(od.arith_host(0, a), a / 6.0)


def test_div6_all_binades(od):
    rng = np.random.default_rng(2)
    a = positive_normals(rng, 2_000_000)
    same(od.arith_host(0, a), a / 6.0)
    same(od.arith_host(0, -a), -a / 6.0)


def test_div6_structured_significands(od):
    # significands around the 3*2^51 split, multiples of 3 (exact quotients),
    # remainders 1 and 2, all-ones, for exponents at the fast-path edge
    M = []
    for base in (1 << 52, 3 << 51, (1 << 53) - 1):
        M += [base + d for d in range(-40, 41) if (1 << 52) <= base + d < (1 << 53)]
    M += [3 * k for k in range((1 << 52) // 3 + 1, (1 << 52) // 3 + 200)]
    M = np.array(M, dtype=np.uint64) - np.uint64(1 << 52)
    for e in (1, 2, 3, 4, 5, 1023, 2045, 2046):
        a = from_bits((np.uint64(e) << np.uint64(52)) | M)
        same(od.arith_host(0, a), a / 6.0)


def test_div6_specials_and_subnormals(od):
    rng = np.random.default_rng(3)
    sub = from_bits(rng.integers(1, 1 << 52, 100_000, dtype=np.uint64))
    a = np.concatenate([SPECIALS, sub, -sub])
    same(od.arith_host(0, a), a / 6.0)


def test_add_random_unit_interval(od):
    rng = np.random.default_rng(4)
    a = rng.random(2_000_000)
    b = rng.random(2_000_000) * rng.choice([1.0, 1e-3, 1e-9, 3.0], 2_000_000)
    same(od.arith_host(1, a, b), a + b)


def test_add_all_exponent_gaps(od):
    rng = np.random.default_rng(5)
    n = 20_000
    for gap in list(range(0, 70)) + [100, 500, 1000]:
        ea = rng.integers(gap + 1, 2046, n, dtype=np.uint64)
        eb = ea - np.uint64(gap)
        ma = rng.integers(0, 1 << 52, n, dtype=np.uint64)
        mb = rng.integers(0, 1 << 52, n, dtype=np.uint64)
        a = from_bits((ea << np.uint64(52)) | ma)
        b = from_bits((eb << np.uint64(52)) | mb)
        same(od.arith_host(1, a, b), a + b)
        same(od.arith_host(1, b, a), b + a)


def test_add_ties_and_carries(od):
    # exact halfway cases (round to even both ways), carries into a new binade,
    # rounding carries into the exponent, largest finite sums
    one = 1.0
    ulp = 2.0 ** -52
    cases = [
        (one, ulp / 2), (one + ulp, ulp / 2), (one, 3 * ulp / 2), (one + ulp, 3 * ulp / 2),
        (1.5, 1.5), (2 - ulp, 2 - ulp), (2 - ulp, ulp / 2), (2 - ulp, ulp), (2 - ulp, ulp / 4),
        (1.0, 1.0), (0.75, 0.25), (2 - ulp, 2 - 2 * ulp), (1.7976931348623157e308 / 2, 1.7976931348623157e308 / 2),
        (8.98846567431158e307, 8.98846567431158e307), (1.0, 2.0 ** -60), (1.0, 2.0 ** -53 + 2.0 ** -105),
    ]
    rng = np.random.default_rng(6)
    m = rng.integers(0, 1 << 52, 50_000, dtype=np.uint64)
    a = from_bits((np.uint64(1023) << np.uint64(52)) | m)
    # b = a's low half-ulp patterns: same exponent minus 53/54 with trailing bits
    b1 = from_bits((np.uint64(1023 - 53) << np.uint64(52)) | (m & np.uint64(0xFF)))
    b2 = from_bits((np.uint64(1023 - 52) << np.uint64(52)))
    A = np.concatenate([np.array([c[0] for c in cases]), a, a, 2.0 - a / 4])
    B = np.concatenate([np.array([c[1] for c in cases]), b1, np.full_like(a, b2[()] if b2.shape == () else b2),
                        a])
    same(od.arith_host(1, A, B), A + B)
    same(od.arith_host(1, B, A), B + A)


def test_add_specials_mixed_signs_subnormals(od):
    rng = np.random.default_rng(7)
    n = 200_000
    pool = np.concatenate([SPECIALS, -SPECIALS, positive_normals(rng, 1000),
                           from_bits(rng.integers(1, 1 << 52, 1000, dtype=np.uint64))])
    a = rng.choice(pool, n)
    b = rng.choice(pool, n)
    with np.errstate(all="ignore"):
        same(od.arith_host(1, a, b), a + b)


def test_jacobi_sum_chain(od):
    # the kernels' exact sequence (((((W+E)+S)+N)+D)+U)/6 assembled from the
    # host routines equals the IEEE chain
    rng = np.random.default_rng(8)
    v = rng.random((6, 1_000_000))
    v[:, ::7] = 0.0
    s_ieee = ((((v[0] + v[1]) + v[2]) + v[3]) + v[4]) + v[5]
    s = od.arith_host(1, v[0], v[1])
    for k in range(2, 6):
        s = od.arith_host(1, s, v[k])
    same(s, s_ieee)
    same(od.arith_host(0, s), s_ieee / 6.0)


def _update_inputs(rng, n):
    """Six operands per cell: mostly the solver's regime (values in [0,1)),
    plus zeros, negatives, subnormals, huge/tiny exponents and exact ties."""
    x = rng.random((n, 6))
    k = n // 8
    x[:k] = positive_normals(rng, 6 * k).reshape(k, 6) * rng.choice([1.0, 1e-300, 1e300], (k, 6))
    x[k:2 * k, rng.integers(0, 6)] = 0.0
    x[2 * k:3 * k] *= rng.choice([-1.0, 1.0], (k, 6))
    x[3 * k:3 * k + 100] = from_bits(rng.integers(1, 1 << 52, (100, 6), dtype=np.uint64))
    # chain partial sums landing on exact halves: 1 + 2^-53 patterns
    x[4 * k:4 * k + 1000, 0] = 1.0
    x[4 * k:4 * k + 1000, 1] = 2.0 ** -53
    x[4 * k:4 * k + 1000, 2] = 2.0 ** -53 * rng.integers(1, 4, 1000)
    # a partial sum of exactly 1.0 met by an operand just above half an ulp
    # whose excess lies far below the 64-bit alignment window (the sticky
    # bit alone decides the rounding), at every position of the chain
    base = 6 * k
    for t in range(1, 6):
        parts = [0.5 ** (i + 1) for i in range(t - 1)]
        parts.append(1.0 - sum(parts))
        rows = slice(base + (t - 1) * 200, base + t * 200)
        x[rows, :t] = parts
        x[rows, t] = 2.0 ** -53 * (1 + 2.0 ** -int(rng.integers(20, 52)))
    # exponents at the chain domain's edges (biased 3, 4, 2040, 2041)
    for j, e in enumerate((3, 4, 2040, 2041)):
        sl = slice(5 * k + j * 100, 5 * k + (j + 1) * 100)
        x[sl] = from_bits((np.uint64(e) << np.uint64(52)) | rng.integers(0, 1 << 52, (100, 6), dtype=np.uint64))
    return x


@pytest.mark.parametrize("mode", range(9))  # 7 / 8: the tail form (op 17 / 18)
def test_update_every_mode_matches_ieee(od, mode):
    rng = np.random.default_rng(100 + mode)
    x = _update_inputs(rng, 400_000)
    with np.errstate(all="ignore"):
        want = (((((x[:, 0] + x[:, 1]) + x[:, 2]) + x[:, 3]) + x[:, 4]) + x[:, 5]) / 6.0
    got = od.arith_host(10 + mode, np.ascontiguousarray(x).ravel())[: len(x)]
    same(got, want)


def _update2d_inputs(rng, n):
    """Four operands per cell (the 2D update): the 3D generator's regimes,
    plus the tie / sticky patterns at each of the three chain positions and
    sums whose quarter is subnormal (the division by 4 is then not exact)."""
    x = np.ascontiguousarray(_update_inputs(rng, n)[:, :4])
    base = 7 * (n // 8)
    for t in range(1, 4):
        parts = [0.5 ** (i + 1) for i in range(t - 1)]
        parts.append(1.0 - sum(parts))
        rows = slice(base + (t - 1) * 200, base + t * 200)
        x[rows] = 0.0
        x[rows, :t] = parts
        x[rows, t] = 2.0 ** -53 * (1 + 2.0 ** -int(rng.integers(20, 52)))
    # sums with biased exponent 0..5 (subnormal up to 2^-1018): one normal
    # operand of exponent 1..4, subnormal or zero partners, either sign; the
    # quarter is subnormal (and rounds) below exponent 3
    tail = slice(n - 2000, n)
    e = rng.integers(1, 5, 2000, dtype=np.uint64)
    x[tail] = 0.0
    x[tail, 0] = from_bits((e << np.uint64(52)) | rng.integers(0, 1 << 52, 2000, dtype=np.uint64))
    sub = from_bits(rng.integers(0, 1 << 52, (2000, 3), dtype=np.uint64))
    x[tail, 1:] = sub * rng.choice([-1.0, 0.0, 1.0], (2000, 3))
    # four normal operands of exponent 1..6 and mixed signs: cancellation
    # leaves sums of every small exponent inside the window chain's domain
    tail = slice(n - 4000, n - 2000)
    e = rng.integers(1, 7, (2000, 4), dtype=np.uint64)
    x[tail] = from_bits((e << np.uint64(52)) | rng.integers(0, 1 << 52, (2000, 4), dtype=np.uint64))
    x[tail] *= np.array([1.0, -1.0, 1.0, -1.0])
    # deep cancellation inside the chain's exponent domain (every operand of
    # biased exponent 4..8): v - v' leaves a few ulps, w - w cancels exactly,
    # so the sum is subnormal or barely normal
    tail = slice(n - 6000, n - 4000)
    e = rng.integers(4, 9, 2000, dtype=np.uint64)
    mv = rng.integers(1 << 20, 1 << 52, 2000, dtype=np.uint64)
    v = from_bits((e << np.uint64(52)) | mv)
    v2 = from_bits((e << np.uint64(52)) | (mv - rng.integers(0, 1 << 19, 2000, dtype=np.uint64)))
    w = from_bits((rng.integers(4, 9, 2000, dtype=np.uint64) << np.uint64(52)) | rng.integers(0, 1 << 52, 2000, dtype=np.uint64))
    x[tail] = np.stack([v, -v2, w, -w], axis=1)
    # a positive in-domain window sum cancelled by the IEEE adds after it
    # (modes with fewer than three window adds): tiny or subnormal sums
    tail = slice(n - 8000, n - 6000)
    a = from_bits((rng.integers(4, 9, 2000, dtype=np.uint64) << np.uint64(52))
                  | rng.integers(0, 1 << 52, 2000, dtype=np.uint64))
    b = from_bits((rng.integers(4, 9, 2000, dtype=np.uint64) << np.uint64(52))
                  | rng.integers(0, 1 << 52, 2000, dtype=np.uint64))
    ab = a + b
    c = -from_bits(ab.view(np.uint64) - (rng.integers(0, 1 << 52, 2000, dtype=np.uint64) >> rng.integers(0, 52, 2000, dtype=np.uint64)))
    d = from_bits(rng.integers(0, 1 << 52, 2000, dtype=np.uint64)) * rng.choice([-1.0, 0.0, 1.0], 2000)
    x[tail] = np.stack([a, b, c, d], axis=1)
    # the same with the cancelling operand last (after a third window add)
    h = slice(n - 7000, n - 6000)
    w3 = from_bits((rng.integers(4, 9, 1000, dtype=np.uint64) << np.uint64(52))
                   | rng.integers(0, 1 << 52, 1000, dtype=np.uint64))
    abw = (x[h, 0] + x[h, 1]) + w3
    x[h, 2] = w3
    x[h, 3] = -from_bits(abw.view(np.uint64) - (rng.integers(0, 1 << 52, 1000, dtype=np.uint64)
                                                >> rng.integers(0, 52, 1000, dtype=np.uint64)))
    return x


@pytest.mark.parametrize("mode", range(7))  # 5 / 6: the tail form (op 25 / 26)
def test_update2d_every_mode_matches_ieee(od, mode):
    rng = np.random.default_rng(200 + mode)
    x = _update2d_inputs(rng, 400_000)
    with np.errstate(all="ignore"):
        want = (((x[:, 0] + x[:, 1]) + x[:, 2]) + x[:, 3]) / 4.0
    got = od.arith_host(20 + mode, np.ascontiguousarray(x).ravel())
    same(got, want)


@pytest.mark.parametrize("op,n_ops", [(17, 6), (18, 6), (25, 4), (26, 4)])
def test_tail_forms_in_the_solver_regime(od, op, n_ops):
    # operands like a Jacobi field after some iterations: similar magnitudes,
    # so the tail window takes (nearly) every cell, with every rounding case
    rng = np.random.default_rng(op)
    x = 0.25 + 0.5 * rng.random((500_000, n_ops))
    x[::3] *= 2.0 ** rng.integers(-8, 1, (x[::3].shape[0], n_ops))
    with np.errstate(all="ignore"):
        want = x[:, 0] + x[:, 1]
        for k in range(2, n_ops):
            want = want + x[:, k]
        want = want / (6.0 if n_ops == 6 else 4.0)
    same(od.arith_host(op, np.ascontiguousarray(x).ravel()), want)
