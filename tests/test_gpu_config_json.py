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


def test_linear_map_prior_is_the_equivalent_block():
    """A prior on b = A theta (Eq. 6, linear generalised parametrisation) enters the model as
    the covariance block (A^T V^-1 A)^-1 with mean (A^T V^-1 A)^-1 A^T V^-1 b0 (oracle's
    linear_prior_block): the library's prior widths and nominal values match it, and -2lnL
    matches the oracle model built with that block."""
    import copy
    import oracle
    from test_config_json import _mapped_config
    cfg, A, b0, V, esc = _mapped_config()
    gj = fitcore.Model.from_json(cfg)
    spec = copy.deepcopy(synth.make_model("c1"))
    t, Cb, _ = oracle.linear_prior_block(A, b0, V)
    ix = np.array([spec.index(n) for n in esc], np.int32)
    spec.theta0 = spec.theta0.copy()
    spec.theta0[ix] = t
    spec.prior_sigma = spec.prior_sigma.copy()
    spec.prior_sigma[ix] = 0.0
    spec.cov_blocks = list(spec.cov_blocks) + [(ix, Cb)]
    th, sg = gj.params()
    # two FP64 evaluations of the same closed form (Cholesky solves against numpy's inverse):
    # agreement to 1e-12, a 1e-9 fraction of the coefficients' prior widths
    np.testing.assert_allclose(th, spec.theta0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(sg[ix], np.sqrt(np.diag(Cb)), rtol=1e-10)
    om = oracle.OracleModel(spec)
    rng = np.random.default_rng(4)
    mu = om.expected(spec.theta0)
    data = rng.poisson(mu).astype(np.float32)
    thetas = np.stack([om.theta_of_z(0.3 * rng.standard_normal(spec.n_params)) for _ in range(3)])
    nll, _, st = fitcore.eval_numpy(gj, thetas, data[None].repeat(3, 0))
    assert np.all(st == 0)
    for b in range(3):
        ref = om.nll(thetas[b], data)
        assert abs(nll[b] - ref) <= 1e-3 + 2e-7 * np.abs(om.expected(thetas[b]) - data).sum()
