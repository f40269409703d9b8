"""A prior on b = A theta in a JSON configuration (Eq. 6 with a linear generalised
parametrisation) against the oracle, which evaluates Eq. 6 as written:
(A theta - b0)^T V^-1 (A theta - b0) with its gradient A^T 2 V^-1 (A theta - b0)."""
import numpy as np
import pytest

import oracle
from paper_2502_15253_gb300 import fitcore, synth
from test_config_json import _mapped_config

pytestmark = pytest.mark.gpu


def _models():
    cfg, A, b0, V, esc = _mapped_config()
    gj = fitcore.Model.from_json(cfg)
    spec = synth.ModelSpec.from_config(cfg)       # keeps the map as written
    om = oracle.OracleModel(spec)
    _, _, const = oracle.linear_prior_block(A, b0, V)
    return cfg, gj, spec, om, const, esc


def test_linear_map_prior_matches_eq6_as_written():
    """The library converts the map prior into an equivalent block on the parameters and drops
    its theta-independent constant c = min over theta of the quadratic form. So -2lnL of the
    library + c equals the oracle's literal Eq. 6 -2lnL, and the gradients agree, at points
    away from the nominal one (eval-parity bars of the other models)."""
    cfg, gj, spec, om, const, esc = _models()
    rng = np.random.default_rng(4)
    data = synth.poisson_data(om.expected(spec.theta0), 41).astype(np.float32)
    thetas = np.stack([om.theta_of_z(0.3 * rng.standard_normal(spec.n_params)) for _ in range(4)])
    nll, g, st = fitcore.eval_numpy(gj, thetas, data[None].repeat(4, 0))
    assert np.all(st == 0)
    s = np.where(spec.prior_sigma > 0, spec.prior_sigma, spec.scale)
    for b in range(4):
        ref, gref = om.nll(thetas[b], data, grad=True)
        tol = 1e-3 + 2e-7 * np.abs(om.expected(thetas[b]) - data).sum()
        assert abs(nll[b] + const - ref) <= tol, (nll[b] + const, ref)
        assert np.linalg.norm((g[b] - gref) * s) <= 1e-5 * np.linalg.norm(gref * s)


def test_linear_map_prior_fit_matches_eq6_as_written():
    """Fits of the JSON model on the device reach the oracle's minimum of the literal Eq. 6
    likelihood: -2lnL_min + c within 1e-3, the nine constrained coefficients within 1e-3 of
    their oracle uncertainties."""
    cfg, gj, spec, om, const, esc = _models()
    ix = [spec.index(n) for n in esc]
    P = spec.n_params
    datas = [synth.poisson_data(om.expected(spec.theta0), 50 + i) for i in range(3)]
    inst = np.zeros(3, fitcore.INSTANCE_DTYPE)
    for i in range(3):
        inst[i] = (0, spec.all_mask(), i * spec.n_bins, i * P)
    start = np.tile(gj.params()[0], 3)
    best, res = fitcore.fit_numpy([gj], inst, np.concatenate(datas), start=start)
    for i, d in enumerate(datas):
        r = om.fit(d, start=gj.params()[0])
        assert r["status"] == 0 and res[i]["status"] == 0
        assert abs(res[i]["nll_min"] + const - r["nll"]) <= 1e-3, (res[i]["nll_min"] + const, r["nll"])
        sig = om.sigma(r["theta"], d)
        dz = np.abs(best[i * P:(i + 1) * P][ix] - r["theta"][ix]) / sig[ix]
        assert np.all(dz <= 1e-2), dz
        assert np.mean(dz <= 1e-3) >= 7 / 9, dz


def test_linear_map_prior_nominal_and_widths():
    """The library reports the block's mean (A^T V^-1 A)^-1 A^T V^-1 b0 as the nominal values
    of the mapped parameters and sqrt of the block's diagonal as their widths."""
    cfg, A, b0, V, esc = _mapped_config()
    gj = fitcore.Model.from_json(cfg)
    spec = synth.make_model("c1")
    t, Cb, _ = oracle.linear_prior_block(A, b0, V)
    ix = np.array([spec.index(n) for n in esc], np.int32)
    th, sg = gj.params()
    np.testing.assert_allclose(th[ix], t, rtol=0, atol=1e-12)
    np.testing.assert_allclose(sg[ix], np.sqrt(np.diag(Cb)), rtol=1e-10)
