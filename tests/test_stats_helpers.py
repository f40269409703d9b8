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
