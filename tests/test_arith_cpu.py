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


# ---------------------------------------------------------------- anchored window
#
# The anchored forms: op 30+f (3D) / 40+f (2D) with f adds on the FP64 pipe,
# the rest in one window anchored at the exponent b[0] for every cell; op
# 34+f / 44+f return the fast form alone (NaN where a cell leaves it), so a
# test can check both that the fast form is taken and that it is exact.

def _anchor(e0):
    return np.array([float(e0)])


def _regime(rng, n, k, lo=-7):
    """k operands per cell in a Jacobi field's regime: values in [2^lo, 1),
    most of them near 0.5 (after some smoothing), a tenth spread over every
    binade of the window, so that partial sums cross binades and round at
    every position with ties among them."""
    x = 0.4 + 0.2 * rng.random((n, k))
    m = n // 10
    x[:m] = rng.random((m, k)) * 2.0 ** rng.integers(lo, 0, (m, k))
    x[:m] = np.maximum(x[:m], 2.0 ** lo)
    return x


def _ieee3d(x):
    with np.errstate(all="ignore"):
        return (((((x[:, 0] + x[:, 1]) + x[:, 2]) + x[:, 3]) + x[:, 4]) + x[:, 5]) / 6.0


def _ieee2d(x):
    with np.errstate(all="ignore"):
        return (((x[:, 0] + x[:, 1]) + x[:, 2]) + x[:, 3]) / 4.0


@pytest.mark.parametrize("nf", range(4))
@pytest.mark.parametrize("e0", [4, 1016, 1020, 2030])
def test_anchored_update_matches_ieee_everywhere(od, nf, e0):
    # every kind of input (zeros, negatives, subnormals, huge and tiny
    # exponents, ties), with anchors inside and far from the data
    rng = np.random.default_rng(300 + 10 * nf + e0 % 7)
    x = _update_inputs(rng, 200_000)
    same(od.arith_host(30 + nf, np.ascontiguousarray(x).ravel(), _anchor(e0)), _ieee3d(x))


@pytest.mark.parametrize("nf", range(3))
@pytest.mark.parametrize("e0", [4, 1016, 1020, 2030])
def test_anchored_update2d_matches_ieee_everywhere(od, nf, e0):
    rng = np.random.default_rng(400 + 10 * nf + e0 % 7)
    x = _update2d_inputs(rng, 200_000)
    same(od.arith_host(40 + nf, np.ascontiguousarray(x).ravel(), _anchor(e0)), _ieee2d(x))


@pytest.mark.parametrize("nf", range(4))
def test_anchored_fast_form_is_taken_and_exact(od, nf):
    # in the solver's regime with the anchor the library derives for a field
    # in [0, 1) (largest exponent 1022), every cell takes the fast form and
    # gives the IEEE bits -- including the many rounding ties of sums whose
    # operands sit in different binades
    rng = np.random.default_rng(500 + nf)
    e0 = 1022 - (5 if nf >= 2 else 6)
    x = _regime(rng, 1_000_000, 6, lo=e0 - 1023)
    got = od.arith_host(34 + nf, np.ascontiguousarray(x).ravel(), _anchor(e0))
    assert not np.isnan(got).any(), f"{int(np.isnan(got).sum())} cells left the fast form"
    same(got, _ieee3d(x))


@pytest.mark.parametrize("nf", range(3))
def test_anchored2d_fast_form_is_taken_and_exact(od, nf):
    rng = np.random.default_rng(600 + nf)
    x = _regime(rng, 1_000_000, 4)
    got = od.arith_host(44 + nf, np.ascontiguousarray(x).ravel(), _anchor(1016))
    assert not np.isnan(got).any()
    same(got, _ieee2d(x))


def test_anchored_window_edges(od):
    # operands at the window's two ends (exponents E0 and E0+7, all-ones and
    # all-zero significands), partial sums just below powers of two that a
    # round-up carries into the next binade, and one binade past each end
    # (which must leave the fast form, not give a wrong value)
    e0 = 1016
    rng = np.random.default_rng(700)
    n = 200_000
    e = rng.choice([e0, e0 + 1, e0 + 6, e0 + 7], (n, 6)).astype(np.uint64)
    mant = rng.choice([0, (1 << 52) - 1, (1 << 51), (1 << 52) - 2, 1, 3], (n, 6)).astype(np.uint64)
    mant[::2] = rng.integers(0, 1 << 52, (n // 2, 6), dtype=np.uint64)
    x = from_bits((e << np.uint64(52)) | mant)
    # with no FP64 add every such cell stays in the fast form; with FP64 adds
    # first, a partial sum past the window's top leaves it (exact either way)
    for nf in range(4):
        same(od.arith_host(30 + nf, np.ascontiguousarray(x).ravel(), _anchor(e0)), _ieee3d(x))
    fast = od.arith_host(34, np.ascontiguousarray(x).ravel(), _anchor(e0))
    assert not np.isnan(fast).any()
    x2 = np.ascontiguousarray(x[:, :4])
    for nf in range(3):
        same(od.arith_host(40 + nf, x2.ravel(), _anchor(e0)), _ieee2d(x2))
    assert not np.isnan(od.arith_host(44, x2.ravel(), _anchor(e0))).any()
    out = x.copy()
    out[:, 5] = from_bits((np.uint64(e0 - 1) << np.uint64(52)) | mant[:, 5])
    out[::2, 5] = from_bits((np.uint64(e0 + 8) << np.uint64(52)) | mant[::2, 5])
    for nf in range(4):
        same(od.arith_host(30 + nf, np.ascontiguousarray(out).ravel(), _anchor(e0)), _ieee3d(out))
        fast = od.arith_host(34 + nf, np.ascontiguousarray(out).ravel(), _anchor(e0))
        assert np.isnan(fast).all(), "an operand outside the window must leave the fast form"


def test_anchored_planted_rounding_mistakes_are_caught(od):
    # the solver-regime inputs distinguish round-to-nearest-even from the
    # nearby wrong roundings: round half up, truncation and a per-step
    # rounding at the wrong binade all differ from the IEEE bits on them
    # (computed here in plain integer arithmetic as the fast form does), so
    # the tests above would catch such a mistake in the fast form
    rng = np.random.default_rng(800)
    x = _regime(rng, 20_000, 6)
    e0 = 1016

    def fixed(v):
        b = v.view(np.uint64)
        e = (b >> np.uint64(52)).astype(np.int64)
        m = (b & np.uint64((1 << 52) - 1)) | np.uint64(1 << 52)
        return [int(mi) << int(ei - e0) for mi, ei in zip(m, e)]

    def chain(rule):
        cols = [fixed(x[:, t]) for t in range(6)]
        out = []
        for i in range(len(x)):
            F = cols[0][i]
            for t in range(1, 6):
                F += cols[t][i]
                d = F.bit_length() - 53
                q, r = divmod(F, 1 << d)
                half = 1 << (d - 1)
                if rule == "even":
                    q += 1 if (r > half or (r == half and q & 1)) else 0
                elif rule == "half_up":
                    q += 1 if r >= half else 0
                elif rule == "shifted":  # rounds one bit too low
                    d -= 1
                    q, r = divmod(F, 1 << d)
                    if d > 0:
                        q += 1 if (r > (1 << (d - 1)) or (r == 1 << (d - 1) and q & 1)) else 0
                F = q << d
            out.append(F)
        return np.array([float(F) * 2.0 ** (e0 - 1075) for F in out])

    want = ((((x[:, 0] + x[:, 1]) + x[:, 2]) + x[:, 3]) + x[:, 4]) + x[:, 5]
    assert np.array_equal(chain("even"), want)
    for rule in ("half_up", "trunc", "shifted"):
        assert not np.array_equal(chain(rule), want), rule


def test_anchored_last_rounding_carries_into_next_binade(od):
    # operand sets whose last partial sum rounds up to an exact power of two
    # (the window word's top bit moves up one place): the division by 6 and
    # the 2D division by 4 must read the carried word correctly
    rng = np.random.default_rng(900)
    e0 = 1016
    rows = []
    for _ in range(20_000):
        k = int(rng.integers(-4, 2))  # target power 2^k + a little less
        parts = 0.9 + 0.2 * rng.random(5)
        parts = parts / parts.sum() * (2.0 ** k) * (1 + 2.0 ** -50)
        last = 2.0 ** k - np.sum(parts[:-1])
        v = np.concatenate([parts[:-1], [last]])
        v = np.maximum(v, 2.0 ** -7)
        s = ((((v[0] + v[1]) + v[2]) + v[3]) + v[4])
        # choose the sixth operand so the total sits within an ulp of 2^(k+1)
        sixth = 2.0 ** (k + 1) - s
        sixth = np.nextafter(sixth, 0.0) if rng.random() < 0.5 else sixth
        rows.append(np.concatenate([v[:5], [sixth]]))
    x = np.array(rows)
    x = x[(x >= 2.0 ** -7).all(axis=1) & (x < 1.0).all(axis=1)]
    assert len(x) > 1000
    tot = _ieee3d(x) * 6.0
    assert np.any(np.log2(tot) == np.round(np.log2(tot))), "no sum landed on a power of two"
    for nf in range(3):
        same(od.arith_host(30 + nf, np.ascontiguousarray(x).ravel(), _anchor(e0)), _ieee3d(x))
        assert not np.isnan(od.arith_host(34 + nf, np.ascontiguousarray(x).ravel(), _anchor(e0))).any()
    x2 = np.ascontiguousarray(x[:, [0, 1, 2, 5]])
    for nf in range(3):
        same(od.arith_host(40 + nf, x2.ravel(), _anchor(e0)), _ieee2d(x2))
