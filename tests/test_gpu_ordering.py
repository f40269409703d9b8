"""Mass ordering at 53 km: profiles of -2lnL in dm2_31 under the normal and the inverted
hypothesis (the exact vacuum survival at dm2_31 > 0 and < 0, i.e. Eq. 10 with +phi and -phi)
fitted to an Asimov data set of the injected normal ordering, as in the paper's medium-baseline
application. The device scans are checked point by point against the oracle's constrained fits
(-2lnL within 1e-3, the fit bar) and for the physics: the normal profile has its minimum at the
injected value, the inverted one is disfavoured and its best |dm2_ee| is shifted."""
import numpy as np
import pytest

import oracle
from paper_2502_15253_gb300 import fitcore, synth

pytestmark = pytest.mark.gpu


def dm2_ee(spec, theta):
    """Eq. 2: cos^2 th12 |dm2_31| + sin^2 th12 |dm2_32| (magnitudes: both orderings)."""
    s12 = theta[spec.index("sin2_th12")]
    dm21, dm31 = theta[spec.index("dm2_21")], theta[spec.index("dm2_31")]
    return (1 - s12) * abs(dm31) + s12 * abs(dm31 - dm21)


@pytest.fixture(scope="module")
def c2():
    spec = synth.make_model("c2")
    om = oracle.OracleModel(spec)
    gm = fitcore.Model(spec)
    data = om.expected(spec.theta0).astype(np.float32)   # Asimov, normal ordering
    return spec, om, gm, data


def test_expectation_at_inverted_ordering_matches_oracle(c2):
    spec, om, gm, _ = c2
    th = spec.theta0.copy()
    th[spec.index("dm2_31")] = -2.455e-3
    mu, st = fitcore.expected_numpy(gm, th[None, :])
    assert st[0] == 0
    ref = om.expected(th)
    np.testing.assert_allclose(mu[0], ref, rtol=2e-5)


def test_normal_and_inverted_profiles(c2):
    spec, om, gm, data = c2
    i31 = spec.index("dm2_31")
    no = np.linspace(2.47e-3, 2.53e-3, 13)
    io = -np.linspace(2.425e-3, 2.485e-3, 13)
    st_io = spec.theta0.copy()
    st_io[i31] = io[6]
    r_no = fitcore.fit_profile_scan(gm, data, spec.all_mask(), [i31], no)
    r_io = fitcore.fit_profile_scan(gm, data, spec.all_mask(), [i31], io, start=st_io)
    assert np.all(r_no["status"] == 0) and np.all(r_io["status"] == 0)
    # the unconstrained fit lands on the injected normal-ordering point
    nll0 = min(r_no["nll_min"], r_io["nll_min"])
    assert abs(nll0) < 1e-3
    d_no = r_no["dchi2"] + r_no["nll_min"] - nll0
    d_io = r_io["dchi2"] + r_io["nll_min"] - nll0
    # point-by-point parity with the oracle's constrained fits
    fx = np.zeros(spec.n_params, bool)
    fx[i31] = True
    for grid, d, k_list in ((no, d_no, (0, 6, 12)), (io, d_io, (0, 6, 12))):
        for k in k_list:
            st = spec.theta0.copy()
            st[i31] = grid[k]
            ref = om.fit(data, start=st, fixed=fx)
            assert ref["status"] == 0
            assert abs(d[k] - (ref["nll"] - nll0)) <= 1e-3, (grid[k], d[k], ref["nll"] - nll0)
    # physics: NO minimum at the injected value, IO disfavoured with a shifted dm2_ee
    assert no[np.argmin(d_no)] == pytest.approx(spec.theta0[i31], abs=0.6 * (no[1] - no[0]))
    k_io = int(np.argmin(d_io))
    assert 0 < k_io < len(io) - 1          # the raster brackets the inverted minimum
    assert d_io[k_io] > 1.0
    ee_no = dm2_ee(spec, r_no["theta"][int(np.argmin(d_no))])
    ee_io = dm2_ee(spec, r_io["theta"][k_io])
    assert abs(ee_io - ee_no) > 1e-5
