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
