"""On the GPU, the integer-pipe division by 6 and addition must equal both
CUDA's own IEEE operations (__ddiv_rn, __dadd_rn) and the host's IEEE results,
bit for bit, on tens of millions of inputs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_12734_gb300 import build
    build.build()
    import paper_2605_12734_gb300 as pkg
    return pkg, torch


def _bits(t):
    return t.view(dtype=__import__("torch").int64)


def test_div6_device(env):
    pkg, torch = env
    g = torch.Generator(device="cuda:0").manual_seed(1)
    for scale in (6.0, 1e-300, 1e300):
        a = torch.rand(32_000_000, dtype=torch.float64, device="cuda:0", generator=g) * scale
        fast = pkg.arith_device(0, a)
        ieee = pkg.arith_device(2, a)
        assert torch.equal(_bits(fast), _bits(ieee))
    # random bit patterns over every binade (and sign)
    u = torch.randint(0, 2**62, (16_000_000,), device="cuda:0", generator=g, dtype=torch.int64)
    a = u.view(torch.float64)
    a = torch.where(torch.isfinite(a), a, torch.zeros_like(a))
    assert torch.equal(_bits(pkg.arith_device(0, a)), _bits(pkg.arith_device(2, a)))
    assert torch.equal(_bits(pkg.arith_device(0, -a)), _bits(pkg.arith_device(2, -a)))
    host = a[:2_000_000].cpu().numpy()
    assert np.array_equal(pkg.arith_device(0, a[:2_000_000]).cpu().numpy().view(np.uint64),
                          (host / 6.0).view(np.uint64))


def test_add_device(env):
    pkg, torch = env
    g = torch.Generator(device="cuda:0").manual_seed(2)
    n = 32_000_000
    a = torch.rand(n, dtype=torch.float64, device="cuda:0", generator=g)
    for scale in (1.0, 1e-5, 1e-12, 3.0, 2.0 ** -53):
        b = torch.rand(n, dtype=torch.float64, device="cuda:0", generator=g) * scale
        assert torch.equal(_bits(pkg.arith_device(1, a, b)), _bits(pkg.arith_device(3, a, b)))
    u = torch.randint(0, 2**62, (2, 16_000_000), device="cuda:0", generator=g, dtype=torch.int64)
    x = u.view(torch.float64)
    x = torch.where(torch.isfinite(x), x, torch.ones_like(x))
    assert torch.equal(_bits(pkg.arith_device(1, x[0], x[1])), _bits(pkg.arith_device(3, x[0], x[1])))
    ha, hb = x[0, :2_000_000].cpu().numpy(), x[1, :2_000_000].cpu().numpy()
    with np.errstate(all="ignore"):
        want = (ha + hb).view(np.uint64)
    assert np.array_equal(pkg.arith_device(1, x[0, :2_000_000].contiguous(),
                                           x[1, :2_000_000].contiguous()).cpu().numpy().view(np.uint64), want)


@pytest.mark.parametrize("mode", range(9))  # 7 / 8: the tail form (op 17 / 18)
def test_update_every_mode_device(env, mode):
    # the full update on the GPU in every arithmetic mode equals the host IEEE
    # chain, on the same mix of inputs as the host test
    pkg, torch = env
    import test_arith_cpu as host
    rng = np.random.default_rng(200 + mode)
    x = host._update_inputs(rng, 2_000_000)
    with np.errstate(all="ignore"):
        want = (((((x[:, 0] + x[:, 1]) + x[:, 2]) + x[:, 3]) + x[:, 4]) + x[:, 5]) / 6.0
    xd = torch.from_numpy(np.ascontiguousarray(x).ravel()).to("cuda:0")
    got = pkg.arith_device(10 + mode, xd).cpu().numpy()
    host.same(got, want)


def _anchor_dev(torch, e0):
    return torch.tensor([float(e0)], dtype=torch.float64, device="cuda:0")


@pytest.mark.parametrize("nf", range(4))
def test_anchored_update_device(env, nf):
    # the anchored window on the GPU (multiply-adds on the FMA pipe, the
    # binary32 rounding of the low word) equals the host IEEE chain on every
    # kind of input, and in the solver's regime takes the fast form on every
    # cell with every result exact
    pkg, torch = env
    import test_arith_cpu as host
    rng = np.random.default_rng(300 + nf)
    x = host._update_inputs(rng, 2_000_000)
    xd = torch.from_numpy(np.ascontiguousarray(x).ravel()).to("cuda:0")
    for e0 in (4, 1016, 1017, 2030):
        host.same(pkg.arith_device(30 + nf, xd, _anchor_dev(torch, e0)).cpu().numpy(), host._ieee3d(x))
    e0 = 1022 - (5 if nf >= 2 else 6)
    r = host._regime(rng, 4_000_000, 6, lo=e0 - 1023)
    rd = torch.from_numpy(np.ascontiguousarray(r).ravel()).to("cuda:0")
    fast = pkg.arith_device(34 + nf, rd, _anchor_dev(torch, e0)).cpu().numpy()
    assert not np.isnan(fast).any()
    host.same(fast, host._ieee3d(r))


@pytest.mark.parametrize("nf", range(3))
def test_anchored_update2d_device(env, nf):
    pkg, torch = env
    import test_arith_cpu as host
    rng = np.random.default_rng(400 + nf)
    x = host._update2d_inputs(rng, 2_000_000)
    xd = torch.from_numpy(np.ascontiguousarray(x).ravel()).to("cuda:0")
    for e0 in (4, 1016, 1017, 2030):
        host.same(pkg.arith_device(40 + nf, xd, _anchor_dev(torch, e0)).cpu().numpy(), host._ieee2d(x))
    r = host._regime(rng, 4_000_000, 4, lo=-6 if nf == 2 else -7)
    rd = torch.from_numpy(np.ascontiguousarray(r).ravel()).to("cuda:0")
    fast = pkg.arith_device(44 + nf, rd, _anchor_dev(torch, 1017 if nf == 2 else 1016)).cpu().numpy()
    assert not np.isnan(fast).any()
    host.same(fast, host._ieee2d(r))
