"""A prior on b = A theta in a JSON configuration (Eq. 6 with a linear generalised
parametrisation) against the oracle's equivalent covariance block."""
import copy

import numpy as np
import pytest

import oracle
from paper_2502_15253_gb300 import fitcore, synth
from test_config_json import _mapped_config

pytestmark = pytest.mark.gpu


def test_linear_map_prior_is_the_equivalent_block():
    """A prior on b = A theta (Eq. 6, linear generalised parametrisation) enters the model as
    the covariance block (A^T V^-1 A)^-1 with mean (A^T V^-1 A)^-1 A^T V^-1 b0 (oracle's
    linear_prior_block): the library's prior widths and nominal values match it, and -2lnL
    matches the oracle model built with that block."""
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
