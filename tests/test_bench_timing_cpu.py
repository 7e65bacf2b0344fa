"""The CPU-rate measurement behind the benchmark's cpu_baseline and its
reference arm: calls of growing length, the rate from the difference of the
last two, so a per-call one-off cost (the oracle copies the field and touches
fresh pages on every call) cancels.  Checked against a fake oracle on a fake
clock: the rate must come out right under a large one-off cost and call-to-
call noise, and must never come out absurd when the noise swamps the
difference (it then counts the whole call)."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


class FakeOracle:
    """sweep(n) advances a fake clock by overhead + n * t_iter + jitter (a
    call can be slowed down, never sped up)."""

    def __init__(self, t_iter, overhead, noise, seed=0):
        self.t = 0.0
        self.t_iter, self.overhead, self.noise = t_iter, overhead, noise
        self.rng = np.random.default_rng(seed)
        self.calls = []

    def clock(self):
        return self.t

    def sweep(self, n):
        self.calls.append(n)
        self.t += self.overhead + n * self.t_iter + self.noise * abs(self.rng.standard_normal())


@pytest.mark.parametrize("t_iter,overhead,noise", [(0.025, 0.3, 0.0), (0.025, 0.3, 0.05), (0.08, 1.0, 0.1),
                                                   (0.002, 0.5, 0.02)])
def test_rate_from_growing_calls(monkeypatch, t_iter, overhead, noise):
    fake = FakeOracle(t_iter, overhead, noise)
    monkeypatch.setattr(bench.time, "perf_counter", fake.clock)
    cells = 512 ** 3
    rate, n, t = bench._time_oracle(fake.sweep, cells, 10.0)
    want = cells / t_iter
    assert abs(rate / want - 1) < 0.05, (rate, want, fake.calls)
    assert sum(fake.calls) * t_iter + len(fake.calls) * overhead < 40  # a bounded sample


def test_noise_never_gives_an_absurd_rate(monkeypatch):
    # noise far above the work of the calls: the difference is meaningless,
    # so the whole last call is counted (a rate below the true one, never 1e17)
    for seed in range(20):
        fake = FakeOracle(0.001, 0.3, 2.0, seed=seed)
        monkeypatch.setattr(bench.time, "perf_counter", fake.clock)
        rate, n, t = bench._time_oracle(fake.sweep, 1000, 1.0)
        assert 0 < rate < 10 * 1000 / 0.001
