"""Pins of the oracle's counter-based generator and Poisson sampler (CPU only).

Philox4x32-10 is pinned to the generator's published known-answer vectors; the Poisson
sampler (multiplication method below mu = 10, Hormann's PTRS above) to the exact Poisson law:
a chi-square test against the PMF, the first two moments, and the counter invariances that
make a draw independent of how a batch is split.
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, expect in rows:
        assert oracle.philox4x32_10(ctr, key) == expect


def _chi2_pvalue(x, mu):
    """Chi-square goodness of fit of integer draws x against Poisson(mu), tail bins merged
    so that every expected count is at least 20."""
    n = len(x)
    lo, hi = int(stats.poisson.ppf(1e-7, mu)), int(stats.poisson.ppf(1 - 1e-7, mu)) + 1
    ks = np.arange(lo, hi + 1)
    pmf = stats.poisson.pmf(ks, mu)
    pmf[0] += stats.poisson.cdf(lo - 1, mu)
    pmf[-1] += stats.poisson.sf(hi, mu)
    obs = np.bincount(np.clip(x.astype(np.int64), lo, hi) - lo, minlength=len(ks)).astype(float)
    exp = pmf * n
    # merge adjacent bins from the left and the right until every expected count >= 20
    groups, cur_o, cur_e = [], 0.0, 0.0
    for o, e in zip(obs, exp):
        cur_o += o
        cur_e += e
        if cur_e >= 20:
            groups.append((cur_o, cur_e))
            cur_o = cur_e = 0.0
    if cur_e > 0:
        o, e = groups.pop()
        groups.append((o + cur_o, e + cur_e))
    o = np.array([g[0] for g in groups])
    e = np.array([g[1] for g in groups])
    chi2 = float(((o - e) ** 2 / e).sum())
    return stats.chi2.sf(chi2, len(groups) - 1)


@pytest.mark.parametrize("mu", [0.3, 2.5, 9.99, 10.0, 37.5, 480.0, 12345.6])
def test_poisson_matches_pmf(mu):
    n = 400_000
    x = oracle.poisson_sample(np.full(n, mu, np.float32), seed=250215253 + int(mu * 100))
    assert np.all(x == np.floor(x)) and np.all(x >= 0)
    mu32 = float(np.float32(mu))
    # moments: mean within 5 standard errors, variance within 5 standard errors
    se_mean = np.sqrt(mu32 / n)
    assert abs(x.mean() - mu32) < 5 * se_mean
    se_var = mu32 * np.sqrt(2.0 / n + 1.0 / (mu32 * n))
    assert abs(x.var() - mu32) < 5 * se_var
    assert _chi2_pvalue(x, mu32) > 1e-4


def test_poisson_mixed_means_and_edges():
    rng = np.random.default_rng(7)
    mu = rng.uniform(0, 60, 200_000).astype(np.float32)
    x = oracle.poisson_sample(mu, seed=11)
    # the sum of independent Poisson draws is Poisson(sum mu)
    tot = float(mu.astype(np.float64).sum())
    assert abs(x.sum() - tot) < 5 * np.sqrt(tot)
    edge = np.array([0.0, -1.0, np.nan, np.inf, 4194304.0, 4194303.0], np.float32)
    y = oracle.poisson_sample(edge, seed=3)
    assert y[0] == 0.0
    assert np.isnan(y[1]) and np.isnan(y[2]) and np.isnan(y[3]) and np.isnan(y[4])
    assert abs(y[5] - 4194303.0) < 6 * np.sqrt(4194303.0)


def test_poisson_counter_invariance():
    mu = np.linspace(0.1, 80.0, 1000).astype(np.float32)
    full = oracle.poisson_sample(mu, seed=99)
    # element i depends only on (seed, i + offset): a split batch reproduces the whole
    tail = oracle.poisson_sample(mu[400:], seed=99, offset=400)
    np.testing.assert_array_equal(full[400:], tail)
    other = oracle.poisson_sample(mu, seed=100)
    assert np.mean(full != other) > 0.5


@pytest.mark.parametrize("mu", [10.0, 37.5, 480.0, 12345.6])
def test_ptrs_law_by_integration(mu):
    """The transformed-rejection step, integrated over a fine grid of (U, V), accepts each k
    with an area proportional to the Poisson PMF (the method is exact)."""
    n = 2000
    u = ((np.arange(n) + 0.5) / n - 0.5).astype(np.float32)
    v = ((np.arange(n) + 0.5) / n).astype(np.float32)
    U, V = np.meshgrid(u, v, indexing="ij")
    k = oracle.ptrs_step(mu, U, V)
    acc = k >= 0
    assert 0.7 < acc.mean() < 0.95
    law = np.bincount(k[acc].astype(np.int64)) / acc.sum()
    pmf = stats.poisson.pmf(np.arange(len(law)), float(np.float32(mu)))
    assert np.abs(law - pmf).max() < 1e-3
