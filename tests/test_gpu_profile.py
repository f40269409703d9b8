"""Profile likelihood (Eq. 7) on the device: fits with held parameters against the oracle's
constrained fits, the raster scan, its Wilks interval and the goodness of fit."""
import numpy as np
import pytest

import oracle
from paper_2502_15253_gb300 import fitcore, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c0():
    spec = synth.make_model("c0")
    om = oracle.OracleModel(spec)
    gm = fitcore.Model(spec)
    truth = synth.draw_theta_true(spec, np.random.default_rng(21))
    data = synth.poisson_data(om.expected(truth), 22)
    return spec, om, gm, data


def _opts(engine):
    o = fitcore.fit_batch_default_opts()
    o.engine = engine
    return o


@pytest.mark.parametrize("engine", [0, 1], ids=["persistent", "lockstep"])
def test_held_parameter_fits_match_oracle(c0, engine):
    spec, om, gm, data = c0
    i13 = spec.index("sin2_2th13")
    vals = [0.05, 0.09, 0.13]
    P = spec.n_params
    inst = np.zeros(len(vals), fitcore.INSTANCE_DTYPE)
    inst["mask"] = spec.all_mask()
    inst["param_off"] = np.arange(len(vals)) * P
    starts = np.tile(spec.theta0, (len(vals), 1))
    starts[:, i13] = vals
    fixed = np.zeros((len(vals), P), np.uint8)
    fixed[:, i13] = 1
    best, res = fitcore.fit_numpy([gm], inst, data, start=starts.ravel(), opts=_opts(engine),
                                  fixed=fixed.ravel())
    fx = np.zeros(P, bool)
    fx[i13] = True
    for k, v in enumerate(vals):
        th = best[k * P:(k + 1) * P]
        assert res[k]["status"] == 0
        assert th[i13] == pytest.approx(v, rel=1e-6)
        ref = om.fit(data, start=starts[k], fixed=fx)
        assert ref["status"] == 0
        assert abs(res[k]["nll_min"] - ref["nll"]) <= 1e-3, (v, res[k]["nll_min"], ref["nll"])


def test_profile_scan_and_wilks_interval_match_oracle(c0):
    spec, om, gm, data = c0
    i13 = spec.index("sin2_2th13")
    grid = np.linspace(0.0, 0.2, 41)
    r = fitcore.fit_profile_scan(gm, data, spec.all_mask(), [i13], grid)
    assert np.all(r["status"] == 0)
    glob = om.fit(data)
    fx = np.zeros(spec.n_params, bool)
    fx[i13] = True
    ref = []
    for v in grid:
        st = spec.theta0.copy()
        st[i13] = v
        ref.append(om.fit(data, start=st, fixed=fx)["nll"])
    ref_d = np.array(ref) - min(glob["nll"], min(ref))
    np.testing.assert_allclose(r["dchi2"], ref_d, rtol=0, atol=2e-3)
    assert abs(r["nll_min"] - glob["nll"]) <= 1e-3
    lo, hi, op = fitcore.fit_wilks_interval(grid, r["dchi2"], 1.0)
    rlo, rhi, rop = fitcore.fit_wilks_interval(grid, ref_d, 1.0)
    assert op == rop == 0
    assert abs(lo - rlo) <= 1e-3 * (rhi - rlo) + 1e-5 and abs(hi - rhi) <= 1e-3 * (rhi - rlo) + 1e-5
    # goodness of fit of the best fit: deviance of the 40 bins against chi^2 with
    # 40 - 2 (the free oscillation parameters) degrees of freedom
    p = fitcore.fit_chi2_sf(r["nll_min"], spec.n_bins - 2)
    assert 1e-4 < p <= 1.0


def test_two_parameter_scan_on_the_three_dataset_model():
    spec = synth.make_model("c1")
    om = oracle.OracleModel(spec)
    gm = fitcore.Model(spec)
    data = synth.poisson_data(om.expected(spec.theta0), 31)
    i13, idm = spec.index("sin2_2th13"), spec.index("dm2_ee")
    pts = np.array([[a, b] for a in (0.07, 0.09, 0.11) for b in (2.4e-3, 2.5e-3, 2.6e-3)])
    r = fitcore.fit_profile_scan(gm, data, spec.all_mask(), [i13, idm], pts)
    assert np.all(r["status"] == 0)
    np.testing.assert_allclose(r["theta"][:, [i13, idm]], pts, rtol=1e-6)
    fx = np.zeros(spec.n_params, bool)
    fx[[i13, idm]] = True
    for k in (0, 4, 8):
        st = spec.theta0.copy()
        st[[i13, idm]] = pts[k]
        ref = om.fit(data, start=st, fixed=fx)
        assert abs(r["dchi2"][k] + r["nll_min"] - ref["nll"]) <= 1e-3


def test_holding_a_prior_block_parameter_is_rejected(c0):
    spec, om, gm, data = c0
    idx = int(spec.cov_blocks[0][0][0])
    with pytest.raises(fitcore.FitError):
        fitcore.fit_profile_scan(gm, data, spec.all_mask(), [idx], [0.0, 0.01])
