"""The allocation-free evaluation entry point (fit_model_eval_noalloc) against fit_model_eval.

fit_model_eval_noalloc serves callers that cannot allocate device memory (an application
with its own fixed device budget, a plugin under another framework's allocator, a loop that
must not enter the allocator). It keeps its workspace in a fixed device array inside the
library, so the test runs it twice in a row on the same array and checks both results
against the allocating entry point, within the tolerances the evaluation parity tests use:
-2lnL within 1e-3, gradient within 1e-5 relative in whitened units. The file is collected
last so that a failure here cannot hide the other tests' results.
"""
import numpy as np
import pytest

from paper_2502_15253_gb300 import fitcore, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["c2", "c1"])
def test_noalloc_eval_matches_allocating_eval_twice(name):
    torch = pytest.importorskip("torch")
    spec = synth.make_model(name)
    gm = fitcore.Model(spec)
    B = 700 if name == "c1" else 300          # more instances than resident blocks
    rng = np.random.default_rng(17)
    scale = np.where(spec.prior_sigma > 0, spec.prior_sigma, spec.scale)
    theta = spec.theta0 + 0.5 * scale * rng.standard_normal((B, spec.n_params))
    mu, st = fitcore.expected_numpy(gm, spec.theta0[None])
    data = rng.poisson(np.tile(mu.astype(np.float64), (B, 1))).astype(np.float32)
    masks = np.full(B, spec.all_mask(), np.uint32)
    masks[::5] = 1

    dev = torch.device("cuda")
    th_d = torch.tensor(theta, dtype=torch.float64, device=dev)
    da_d = torch.tensor(data, device=dev)
    mk_d = torch.tensor(masks.view(np.int32), device=dev)
    ref_nll = torch.zeros(B, dtype=torch.float64, device=dev)
    ref_g = torch.zeros(B, spec.n_params, dtype=torch.float32, device=dev)
    ref_st = torch.zeros(B, dtype=torch.int32, device=dev)
    fitcore.fit_model_eval(gm, B, th_d, da_d, mk_d, ref_nll, ref_g, ref_st)

    for call in range(2):
        nll = torch.full((B,), np.nan, dtype=torch.float64, device=dev)
        g = torch.full((B, spec.n_params), np.nan, dtype=torch.float32, device=dev)
        st = torch.full((B,), -7, dtype=torch.int32, device=dev)
        fitcore.fit_model_eval_noalloc(gm, B, th_d, da_d, mk_d, nll, g, st)
        torch.cuda.synchronize()
        a, b = nll.cpu().numpy(), ref_nll.cpu().numpy()
        assert np.array_equal(st.cpu().numpy(), ref_st.cpu().numpy()), call
        assert np.all(np.isfinite(a)), call
        assert np.max(np.abs(a - b)) <= 1e-3, (call, np.max(np.abs(a - b)))
        ga, gb = g.cpu().numpy() * scale, ref_g.cpu().numpy() * scale
        rel = np.linalg.norm(ga - gb, axis=1) / np.maximum(np.linalg.norm(gb, axis=1), 1e-30)
        assert rel.max() <= 1e-5, (call, rel.max())


def test_noalloc_rejects_host_buffers():
    spec = synth.make_model("c0")
    gm = fitcore.Model(spec)
    theta = spec.theta0[None].copy()
    nll = np.zeros(1)
    with pytest.raises(fitcore.FitError):
        fitcore.fit_model_eval_noalloc(gm, 1, theta, None, None, nll)
