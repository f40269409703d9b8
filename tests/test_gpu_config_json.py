"""A model created from its JSON configuration (fit_model_create_json) is the model created
from the description: the same expectation, -2lnL, gradient and fit results bit for bit,
and the parameter names the configuration gives."""
import numpy as np
import pytest

from paper_2502_15253_gb300 import fitcore, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["c0", "c1s", "c2/spline"])
def models(request):
    name = request.param.split("/")[0]
    spec = synth.make_model(name, remap=int(request.param.endswith("spline")))
    return spec, fitcore.Model(spec), fitcore.Model.from_json(spec.to_json(), spec)


def test_names_and_sizes(models):
    spec, gs, gj = models
    assert gj.param_names() == list(spec.param_names)
    assert gs.param_names() is None
    assert (gj.n_params, gj.n_data, gj.n_datasets) == (gs.n_params, gs.n_data, gs.n_datasets)
    assert gj.device_bytes == gs.device_bytes


def test_expectation_and_gradient_are_identical(models):
    spec, gs, gj = models
    rng = np.random.default_rng(5)
    sc = np.where(spec.prior_sigma > 0, spec.prior_sigma, spec.scale)
    th = spec.theta0 + 0.5 * sc * rng.standard_normal((6, spec.n_params))
    mu_s, st_s = fitcore.expected_numpy(gs, th)
    mu_j, st_j = fitcore.expected_numpy(gj, th)
    assert np.all(st_s == 0)
    np.testing.assert_array_equal(mu_j, mu_s)
    np.testing.assert_array_equal(st_j, st_s)
    data = np.random.default_rng(6).poisson(mu_s.astype(np.float64)).astype(np.float32)
    nll_s, g_s, _ = fitcore.eval_numpy(gs, th, data)
    nll_j, g_j, _ = fitcore.eval_numpy(gj, th, data)
    np.testing.assert_array_equal(nll_j, nll_s)
    np.testing.assert_array_equal(g_j, g_s)


def test_fits_are_identical(models):
    spec, gs, gj = models
    B = 16
    mu, _ = fitcore.expected_numpy(gs, np.repeat(spec.theta0[None], B, 0))
    data = np.random.default_rng(7).poisson(mu.astype(np.float64)).astype(np.float32)
    inst = np.zeros(B, fitcore.INSTANCE_DTYPE)
    inst["mask"] = spec.all_mask()
    inst["data_off"] = np.arange(B) * spec.n_bins
    inst["param_off"] = np.arange(B) * spec.n_params
    best_s, r_s = fitcore.fit_numpy([gs], inst, data)
    best_j, r_j = fitcore.fit_numpy([gj], inst, data)
    assert np.isin(r_s["status"], [0, 7]).all()
    np.testing.assert_array_equal(r_j["status"], r_s["status"])
    np.testing.assert_array_equal(best_j, best_s)
    np.testing.assert_array_equal(r_j["nll_min"], r_s["nll_min"])
    np.testing.assert_array_equal(r_j["iters"], r_s["iters"])


def test_params_report_nominal_values_and_prior_widths(models):
    spec, gs, gj = models
    sig = spec.prior_sigma.copy()
    for ix, cov in spec.cov_blocks:
        sig[np.asarray(ix)] = np.sqrt(np.diag(cov))
    for g in (gs, gj):
        th, sg = g.params()
        np.testing.assert_array_equal(th, spec.theta0)
        np.testing.assert_array_equal(sg, sig)


def test_result_json_round_trips_the_fit(models):
    """fit_result_json writes the best fit with the configuration's names; every number reads
    back exactly ([S]: the output component's JSON record)."""
    import json
    spec, gs, gj = models
    mu, _ = fitcore.expected_numpy(gj, spec.theta0[None])
    data = np.random.default_rng(8).poisson(mu.astype(np.float64)).astype(np.float32)
    inst = np.zeros(1, fitcore.INSTANCE_DTYPE)
    inst["mask"] = spec.all_mask()
    best, r = fitcore.fit_numpy([gj], inst, data)
    rec = json.loads(fitcore.fit_result_json(gj, best, r[0]))
    assert rec["status"] == fitcore.STATUS[int(r[0]["status"])]
    assert rec["nll_min"] == r[0]["nll_min"] and rec["edm"] == r[0]["edm"]
    assert (rec["iters"], rec["n_evals"]) == (r[0]["iters"], r[0]["n_evals"])
    assert list(rec["params"]) == list(spec.param_names)
    np.testing.assert_array_equal(np.array(list(rec["params"].values())), best)
    # a model built from a description names its parameters p0, p1, ...
    rec = json.loads(fitcore.fit_result_json(gs, best, r[0]))
    assert list(rec["params"])[:3] == ["p0", "p1", "p2"]
