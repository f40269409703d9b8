"""The torch autograd wrapper of the evaluation: forward equals fit_model_eval and backward
returns grad_output times the library's gradient."""
import numpy as np
import pytest

from paper_2502_15253_gb300 import fitcore, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_fit_nll_forward_and_backward():
    spec = synth.make_model("c0")
    gm = fitcore.Model(spec)
    rng = np.random.default_rng(3)
    B = 5
    th = np.tile(spec.theta0, (B, 1)) + 0.3 * rng.standard_normal((B, spec.n_params)) * np.where(
        spec.prior_sigma > 0, spec.prior_sigma, spec.scale)
    mu, _ = fitcore.expected_numpy(gm, spec.theta0[None, :])
    data = rng.poisson(np.tile(mu, (B, 1)).astype(np.float64)).astype(np.float32)
    theta = torch.tensor(th, dtype=torch.float64, device="cuda", requires_grad=True)
    dd = torch.tensor(data, device="cuda")
    nll = fitcore.fit_nll(theta, dd, gm)
    w = torch.arange(1, B + 1, dtype=torch.float64, device="cuda")
    (w * nll).sum().backward()
    ref_nll, ref_g, st = fitcore.eval_numpy(gm, th, data)
    assert np.all(st == 0)
    np.testing.assert_allclose(nll.detach().cpu().numpy(), ref_nll, rtol=1e-12)
    np.testing.assert_allclose(theta.grad.cpu().numpy(), np.arange(1, B + 1)[:, None] * ref_g,
                               rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("name", ["c1/spline", "c2", "c0"])
def test_fit_nll_backward_matches_oracle_and_central_differences(name):
    """The adjoint gradient that fit_nll's backward returns, at non-stationary points (1 sigma
    offsets in whitened units): (1) against the FP64 oracle's analytic gradient (1e-5 relative
    in whitened units, the eval-parity bar) and (2) against central differences of the
    library's own forward -2lnL along random unit directions in whitened units.

    Bar of (2): the FP32 expectation (relative error <= 1e-7 per bin) moves -2lnL by at most
    eps_f = 2e-7 sum_j |mu_j - n_j| (+ 1e-7 |f| for the FP32 deviance terms), so a difference
    quotient with step h carries up to eps_f / h of rounding; h = 1e-2 keeps that and the
    truncation term (h^2 / 6 times the third derivative, below 1e-3 of the slope here) small.
    The directions skip the energy-scale coefficients, where the overlap rule's creases would
    sit inside a step."""
    import oracle
    spec = synth.make_model(name.split("/")[0], remap=int(name.endswith("spline")))
    om = oracle.OracleModel(spec)
    gm = fitcore.Model(spec)
    rng = np.random.default_rng(31)
    B = 4
    th = np.stack([om.theta_of_z(rng.standard_normal(spec.n_params)) for _ in range(B)])
    data = synth.poisson_data(om.expected(spec.theta0), 32).astype(np.float32)
    theta = torch.tensor(th, dtype=torch.float64, device="cuda", requires_grad=True)
    dd = torch.tensor(np.tile(data, (B, 1)), device="cuda")
    fitcore.fit_nll(theta, dd, gm).sum().backward()
    g = theta.grad.cpu().numpy()
    s = np.where(spec.prior_sigma > 0, spec.prior_sigma, spec.scale)
    esc = np.zeros(spec.n_params, bool)
    for ds in spec.datasets:
        esc[[i for i in ds.escale_idx if i >= 0]] = True
    h = 1e-2
    for b in range(B):
        fref, gref = om.nll(th[b], data, grad=True)
        assert np.linalg.norm((g[b] - gref) * s) <= 1e-5 * np.linalg.norm(gref * s), b
        eps_f = 2e-7 * np.abs(om.expected(th[b]) - data).sum() + 1e-7 * abs(fref)
        for k in range(3):
            # the steepest direction first (the largest slope against the rounding), then
            # random ones
            u = g[b] * s if k == 0 else rng.standard_normal(spec.n_params)
            u[esc] = 0.0
            u /= np.linalg.norm(u)
            v = u * s                          # unit step in whitened units
            pts = torch.tensor(np.stack([th[b] + h * v, th[b] - h * v]), dtype=torch.float64,
                               device="cuda")
            with torch.no_grad():
                f = fitcore.fit_nll(pts, dd[:2], gm).cpu().numpy()
            fd = (f[0] - f[1]) / (2 * h)
            an = float(g[b] @ v)
            assert abs(fd - an) <= 2 * eps_f / h + 1e-3 * abs(an), (b, fd, an, eps_f)
