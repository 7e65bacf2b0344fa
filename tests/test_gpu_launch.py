"""Launch-overhead microbenchmarks (the paper's Sec. III measurements) on the
GPU: they run, report plausible numbers, and the release benchmark's kernels
do exactly their share of the work (checked against a host LCG)."""
import numpy as np
import pytest

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


def lcg(x0, work):
    x = np.asarray(x0, dtype=np.uint64)
    for _ in range(work):
        x = (np.uint64(1664525) * x + np.uint64(1013904223)) & np.uint64(0xFFFFFFFF)
    return x


@pytest.mark.parametrize("wait", ["sync", "event", "callback"])
def test_launch_latency(od, wait):
    us = od.bench_launch_latency(wait, reps=500)
    assert 0.5 < us < 5000, us


@pytest.mark.parametrize("nkernels", [1, 7, 64])
def test_release_does_all_the_work(od, nkernels):
    import torch
    n, work = (1 << 18) + 13, 50
    out = torch.zeros(n, dtype=torch.int32, device="cuda:0")
    us = od.bench_release(n, nkernels, work, out=out)
    assert 0 < us < 1e6
    got = out.cpu().numpy().view(np.uint32)
    idx = np.unique(np.concatenate([np.arange(8), np.arange(n - 8, n),
                                    np.random.default_rng(nkernels).integers(0, n, 64)]))
    # every kernel's first and last thread
    idx = np.unique(np.concatenate([idx, [n * k // nkernels for k in range(nkernels)],
                                    [n * (k + 1) // nkernels - 1 for k in range(nkernels)]]))
    assert np.array_equal(got[idx].astype(np.uint64), lcg(idx, work))


def test_release_scratch_buffer(od):
    assert od.bench_release(1 << 20, 16, 0) > 0


@pytest.mark.parametrize("threads,chares", [(1, 1), (2, 4)])
def test_launch_rate(od, threads, chares):
    r = od.bench_launch_rate(threads, chares, kernels=200)
    assert 1e3 < r < 1e8, r
