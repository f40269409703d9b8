"""Host-side statistics helpers of the C ABI (no GPU needed): the chi-square survival function
behind the goodness-of-fit p-value, and the Wilks-interval crossing of a 1-D profile."""
import numpy as np
import pytest
from scipy import stats

from paper_2502_15253_gb300 import fitcore


@pytest.mark.parametrize("chi2,dof", [(0.5, 1), (3.84, 1), (10.0, 3), (120.0, 114), (500.0, 438),
                                      (0.01, 5), (30.0, 4), (1e-8, 2), (700.0, 40)])
def test_chi2_sf_matches_scipy(chi2, dof):
    fitcore.load()
    assert fitcore.fit_chi2_sf(chi2, dof) == pytest.approx(stats.chi2.sf(chi2, dof), rel=1e-10,
                                                          abs=1e-300)


def test_chi2_sf_edges():
    assert fitcore.fit_chi2_sf(0.0, 3) == 1.0
    assert np.isnan(fitcore.fit_chi2_sf(-1.0, 3)) and np.isnan(fitcore.fit_chi2_sf(1.0, 0))


def test_wilks_interval_of_a_parabola():
    x = np.linspace(-3, 3, 61)
    d = ((x - 0.37) / 0.8) ** 2          # -2 ln lambda of a Gaussian with sigma 0.8
    lo, hi, op = fitcore.fit_wilks_interval(x, d, 1.0)
    assert op == 0
    assert lo == pytest.approx(0.37 - 0.8, abs=2e-3) and hi == pytest.approx(0.37 + 0.8, abs=2e-3)
    lo, hi, op = fitcore.fit_wilks_interval(x, d, 100.0)
    assert op == 3 and lo == -3 and hi == 3
    with pytest.raises(fitcore.FitError):
        fitcore.fit_wilks_interval(x[::-1], d, 1.0)


def test_ensemble_coverage_and_goodness_of_fit_on_pseudo_experiments():
    """Wilks' theorem on an ensemble (the statistical reading of Eq. 7-8 and of the paper's
    ensemble studies): 1000 pseudo-experiments of the two-parameter 1 km model at the nominal
    point, fitted by the FP64 oracle. Each draws Poisson counts (~26k events) and an auxiliary
    measurement of dm2_ee (the centre of its Gaussian prior, width 1e-4, Eq. 5), which keeps the
    fit out of the amplitude / dm2 valley of a 1 km baseline. Then:
      * the library's 1-D Wilks interval (profile of sin^2 2th13 over dm2_ee, dchi2 = 1 and
        3.84) covers the true value in 68.3 % / 95 % of the experiments,
      * -2 ln lambda at the true point (two parameters) is chi^2(2): fit_chi2_sf of it is
        uniform,
      * -2lnL at the best fit is chi^2(N_bins + 1 - 2) (the bins plus the auxiliary
        measurement), so its GoF p-value is uniform.
    Bands are 3.5 binomial standard errors and a KS p-value of 1e-3, so a wrong crossing,
    level or number of degrees of freedom fails."""
    import copy
    import oracle
    from paper_2502_15253_gb300 import synth
    base = synth.make_model("c0_tiny")
    truth, sp = base.theta0.copy(), 1e-4
    mu = oracle.OracleModel(base).expected(truth)
    rng = np.random.default_rng(77)
    n_exp, fixed = 1000, np.array([True, False])
    cover = {1.0: 0, 3.84: 0}
    p_true, p_gof = [], []
    sig = None
    for e in range(n_exp):
        s = copy.copy(base)
        s.theta0 = truth.copy()
        s.theta0[1] += sp * rng.standard_normal()
        s.prior_sigma = np.array([0.0, sp])
        om = oracle.OracleModel(s)
        if sig is None:
            sig = om.sigma(truth, mu)[0]
        data = synth.poisson_data(mu, 7700000 + e)
        g = om.fit(data)
        assert g["status"] == 0
        p_true.append(fitcore.fit_chi2_sf(om.nll(truth, data) - g["nll"], 2))
        p_gof.append(fitcore.fit_chi2_sf(g["nll"], len(mu) - 1))
        x = g["theta"][0] + sig * np.linspace(-4.5, 4.5, 37)
        prof = []
        for a in x:
            r = om.fit(data, start=[a, g["theta"][1]], fixed=fixed)
            assert r["status"] == 0
            prof.append(r["nll"] - g["nll"])
        for level in cover:
            lo, hi, op = fitcore.fit_wilks_interval(x, np.array(prof), level)
            assert op == 0
            cover[level] += lo <= truth[0] <= hi
    for level, p in ((1.0, 0.6827), (3.84, 0.95)):
        se = np.sqrt(p * (1 - p) / n_exp)
        assert abs(cover[level] / n_exp - p) < 3.5 * se, (level, cover[level])
    for pv in (p_true, p_gof):
        assert stats.kstest(pv, "uniform").pvalue > 1e-3
