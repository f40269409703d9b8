"""GPU parity of the expectation, -2lnL and gradient against the FP64 oracle (through the C ABI).

Tolerances (derived from FP32 arithmetic, stated with the reason):
  * expectation mu: relative 2e-5 per bin. The survival phase is carried as a float pair, so
    P has absolute error ~2e-7; the fold sums <= 400 FP32 products (relative ~1e-7 each); the
    energy map's overlaps are computed relative to the target bin (abs. error ~1e-7 of a bin).
  * -2lnL: |diff| <= 1e-3 (the tolerance on -2lnL at a fit minimum) at points 0.3 sigma from
    the minimum. Farther away every bin's deviance slope 2(1 - n/mu) grows, so an FP32
    expectation with relative error <= 1e-7 moves -2lnL by up to 2e-7 sum_j |mu_j - n_j|:
    at 1 sigma the bar is 1e-3 + 2e-7 sum_j |mu_j - n_j|.
  * gradient: ||(g - g_oracle) s|| <= 1e-5 ||g_oracle s|| where s is each parameter's step
    scale (the gradient in whitened units), at non-stationary points.
  * far from any fit (empty bins where mu ~ 4000, -2lnL ~ 6e4) the deviance terms are large
    and FP32 rounds each to ~6e-8 relative: there the bar is max(1e-3, 2e-7 |nll|).
"""
import numpy as np
import pytest

import oracle
from paper_2502_15253_gb300 import fitcore, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["c0", "c1", "c2", "c1s", "c0/spline", "c1/spline", "c2/spline",
                                                "c1_flux41"])
def pair(request):
    spec = synth.make_model(request.param.split("/")[0], remap=int(request.param.endswith("spline")))
    return spec, oracle.OracleModel(spec), fitcore.Model(spec)


def _scale(spec):
    return np.where(spec.prior_sigma > 0, spec.prior_sigma, spec.scale)


def _thetas(spec, om, n, amp, seed):
    rng = np.random.default_rng(seed)
    return np.stack([om.theta_of_z(amp * rng.standard_normal(spec.n_params)) for _ in range(n)])


def test_expected_matches_oracle(pair):
    spec, om, gm = pair
    th = _thetas(spec, om, 5, 0.7, 1)
    mu, st = fitcore.expected_numpy(gm, th)
    assert np.all(st == 0)
    for b in range(len(th)):
        ref = om.expected(th[b])
        np.testing.assert_allclose(mu[b], ref, rtol=2e-5, atol=1e-6 * ref.max())


def test_asimov_data_is_expectation_at_nominal(pair):
    spec, om, gm = pair
    nll, g, st = fitcore.eval_numpy(gm, spec.theta0[None, :], data=None)
    assert st[0] == 0
    assert abs(nll[0]) < 1e-3


@pytest.mark.parametrize("amp", [0.3, 1.0])
def test_nll_and_gradient_match_oracle(pair, amp):
    spec, om, gm = pair
    th = _thetas(spec, om, 6, amp, 2)
    data = synth.poisson_data(om.expected(spec.theta0), 3)
    nll, g, st = fitcore.eval_numpy(gm, th, np.tile(data, (len(th), 1)))
    assert np.all(st == 0)
    s = _scale(spec)
    for b in range(len(th)):
        ref, gref = om.nll(th[b], data, grad=True)
        bar = 1e-3 if amp < 0.5 else 1e-3 + 2e-7 * np.abs(om.expected(th[b]) - data).sum()
        assert abs(nll[b] - ref) <= bar, (b, nll[b], ref, bar)
        err = np.linalg.norm((g[b] - gref) * s) / np.linalg.norm(gref * s)
        assert err <= 1e-5, (b, err)


def test_dataset_masks_and_zero_counts(pair):
    spec, om, gm = pair
    th = _thetas(spec, om, 1, 0.5, 4)[0]
    data = synth.poisson_data(om.expected(spec.theta0), 5)
    data[::7] = 0.0                                  # empty bins: D = 2 mu
    n_ds = len(spec.datasets)
    masks = np.array([(1 << n_ds) - 1, 1, (1 << n_ds) - 2 if n_ds > 1 else 1, 0], np.uint32)
    B = len(masks)
    nll, g, st = fitcore.eval_numpy(gm, np.tile(th, (B, 1)), np.tile(data, (B, 1)), masks)
    s = _scale(spec)
    for b in range(B):
        ref, gref = om.nll(th, data, mask=int(masks[b]), grad=True)
        assert abs(nll[b] - ref) <= max(1e-3, 2e-7 * abs(ref)), (b, nll[b], ref)
        err = np.linalg.norm((g[b] - gref) * s) / max(np.linalg.norm(gref * s), 1e-30)
        assert err <= 1e-5


def test_invalid_points_return_status_not_fault(pair):
    spec, om, gm = pair
    th = np.tile(spec.theta0, (3, 1))
    ds0 = spec.datasets[0]
    if ds0.escale_idx[1] >= 0:
        th[0, ds0.escale_idx[1]] = -0.5                # decreasing energy map
    if ds0.norm_idx >= 0:
        th[1, ds0.norm_idx] = -2.0                     # negative expectation
    elif ds0.eff_idx >= 0:
        th[1, ds0.eff_idx] = -2.0
    nll, g, st = fitcore.eval_numpy(gm, th, None)
    if ds0.escale_idx[1] >= 0:
        assert st[0] == 5 and np.isinf(nll[0])
    assert st[1] == 4 and np.isinf(nll[1])
    assert st[2] == 0 and np.isfinite(nll[2])


def test_large_batch_grid_stride_matches_small_batch(pair):
    spec, om, gm = pair
    B = 1200 if spec.name != "c2" else 400
    th = _thetas(spec, om, B, 0.5, 6)
    data = synth.poisson_data(om.expected(spec.theta0), 7)
    nll, g, st = fitcore.eval_numpy(gm, th, np.tile(data, (B, 1)))
    idx = [0, 1, B // 2, B - 1]
    nll1, g1, _ = fitcore.eval_numpy(gm, th[idx], np.tile(data, (len(idx), 1)))
    np.testing.assert_array_equal(nll[idx], nll1)
    np.testing.assert_array_equal(g[idx], g1)
    for b in idx[:2]:
        assert abs(nll[b] - om.nll(th[b], data)) <= 1e-3


def test_device_buffers_and_empty_batch(pair):
    torch = pytest.importorskip("torch")
    spec, om, gm = pair
    th = torch.tensor(_thetas(spec, om, 3, 0.4, 8), dtype=torch.float64, device="cuda")
    data = torch.tensor(np.tile(synth.poisson_data(om.expected(spec.theta0), 9), (3, 1)),
                        dtype=torch.float32, device="cuda")
    nll = torch.zeros(3, dtype=torch.float64, device="cuda")
    g = torch.zeros(3, spec.n_params, dtype=torch.float32, device="cuda")
    fitcore.fit_model_eval(gm, 3, th, data, None, nll, g)
    torch.cuda.synchronize()
    nll_h, g_h, _ = fitcore.eval_numpy(gm, th.cpu().numpy(), data.cpu().numpy())
    np.testing.assert_array_equal(nll.cpu().numpy(), nll_h)
    np.testing.assert_array_equal(g.cpu().numpy(), g_h)
    fitcore.fit_model_eval(gm, 0, th, data, None, nll, g)   # B = 0 is a no-op
