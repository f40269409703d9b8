"""Poisson pseudo-data on the device (fit_poisson_sample) against the oracle's implementation
of the same generator (Philox4x32-10 counters, multiplication method / PTRS).

Integer results, so the bar is bit-exact. Both sides decide every draw with the same IEEE
single-precision steps (no contraction) and a double-precision acceptance test; the only
library functions involved are exp (rounded to float) and log/lgamma in double, which differ
between the two math libraries by at most a few units in the last place, far below any
decision margin met at these sample sizes.
"""
import numpy as np
import pytest

import oracle
from paper_2502_15253_gb300 import fitcore

pytestmark = pytest.mark.gpu


def _gpu(mu, seed, offset=0):
    mu = np.ascontiguousarray(mu, np.float32)
    out = np.zeros_like(mu)
    fitcore.fit_poisson_sample(mu.size, mu, seed, offset, out)
    return out


def test_bit_exact_against_oracle_mixed_means():
    rng = np.random.default_rng(5)
    mu = np.concatenate([
        rng.uniform(0, 12, 300_000),              # multiplication method and the switch at 10
        rng.uniform(10, 500, 100_000),            # PTRS
        10 ** rng.uniform(2.5, 6, 20_000),        # large means
        np.array([0.0, 1e-30, 9.999999, 10.0, 4194303.0]),
    ]).astype(np.float32)
    got = _gpu(mu, 250215253)
    ref = oracle.poisson_sample(mu, 250215253)
    bad = np.flatnonzero(got != ref)
    assert bad.size == 0, (bad[:10], mu[bad[:10]], got[bad[:10]], ref[bad[:10]])


def test_offset_and_launch_shape_invariance():
    mu = np.linspace(0.01, 900.0, 50_001).astype(np.float32)
    full = _gpu(mu, 42)
    part = _gpu(mu[1000:], 42, offset=1000)
    np.testing.assert_array_equal(full[1000:], part)
    np.testing.assert_array_equal(full, oracle.poisson_sample(mu, 42))


def test_edge_values():
    mu = np.array([0.0, -1.0, np.nan, np.inf, 4194304.0], np.float32)
    got = _gpu(mu, 1)
    assert got[0] == 0.0 and np.all(np.isnan(got[1:]))


def test_device_buffers_and_large_batch():
    torch = pytest.importorskip("torch")
    n = 8_000_000
    mu = torch.full((n,), 37.5, dtype=torch.float32, device="cuda")
    out = torch.empty_like(mu)
    fitcore.fit_poisson_sample(n, mu, 7, 0, out)
    torch.cuda.synchronize()
    x = out.double()
    assert abs(float(x.mean()) - 37.5) < 5 * np.sqrt(37.5 / n)
    assert abs(float(x.var()) - 37.5) < 5 * 37.5 * np.sqrt(2.0 / n)
    tail = oracle.poisson_sample(np.full(1000, 37.5, np.float32), 7, offset=n - 1000)
    np.testing.assert_array_equal(out[-1000:].cpu().numpy(), tail)
