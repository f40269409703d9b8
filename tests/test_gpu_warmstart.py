"""Warm start on the device: training-sample draws, a short training run, and fits started
from the network's predictions against cold fits of the same pseudo-experiments."""
import numpy as np
import pytest

from paper_2502_15253_gb300 import fitcore, synth, warmstart

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def c1():
    spec = synth.make_model("c1")
    return spec, fitcore.Model(spec)


@pytest.fixture(scope="module")
def c2():
    spec = synth.make_model("c2")
    return spec, fitcore.Model(spec)


def _draw(model, geom, B, seed, offset=0):
    th = torch.zeros((B, model.n_params), dtype=torch.float64, device="cuda")
    mk = torch.zeros(B, dtype=torch.int32, device="cuda")
    fitcore.fit_warmstart_draw(model, geom, B, seed, offset, th, mk)
    torch.cuda.synchronize()
    return th.cpu().numpy(), mk.cpu().numpy().view(np.uint32)


def test_draws_follow_priors_and_windows(c1):
    spec, model = c1
    geom = warmstart.geometry(spec)
    B = 40_000
    th, mk = _draw(model, geom, B, 77)
    d = th - spec.theta0
    # uniform windows of the parameters of interest
    for t in range(geom.n_uniform):
        i, h = geom.uniform_idx[t], geom.uniform_half[t]
        assert np.all(np.abs(d[:, i]) <= h * (1 + 1e-12))
        assert abs(d[:, i].mean()) < 5 * h / np.sqrt(3 * B)
        assert abs(d[:, i].var() / (h * h / 3) - 1) < 0.03
    # individual priors
    for i in np.flatnonzero(spec.prior_sigma > 0):
        if i in list(geom.uniform_idx)[:geom.n_uniform]:
            continue
        s = spec.prior_sigma[i]
        assert abs(d[:, i].mean()) < 5 * s / np.sqrt(B)
        assert abs(d[:, i].std() / s - 1) < 0.03
    # covariance blocks: sample covariance against V (first block, leading 6 x 6 entries)
    idx, V = spec.cov_blocks[0]
    k = min(6, len(idx))
    S = np.cov(d[:, idx[:k]].T)
    sd = np.sqrt(np.diag(V)[:k])
    assert np.abs((S - V[:k, :k]) / np.outer(sd, sd)).max() < 0.04
    # masks uniformly over the geometry's choices
    choices = list(geom.masks)[:geom.n_masks]
    counts = np.array([(mk == c).sum() for c in choices])
    assert counts.sum() == B
    assert np.all(np.abs(counts / B - 1 / len(choices)) < 0.02)


def test_draws_are_counter_based(c1):
    spec, model = c1
    geom = warmstart.geometry(spec)
    a, ma = _draw(model, geom, 64, 5)
    b, mb = _draw(model, geom, 64, 5)
    np.testing.assert_array_equal(a, b)
    c, mc = _draw(model, geom, 32, 5, offset=32)
    np.testing.assert_array_equal(a[32:], c)
    np.testing.assert_array_equal(ma[32:], mc)
    d, _ = _draw(model, geom, 64, 6)
    assert np.mean(a != d) > 0.5


def test_training_learns_and_warm_fits_agree_with_cold(c1, c2):
    spec1, m1 = c1
    spec2, m2 = c2
    net = warmstart.network(seed=3)
    losses = warmstart.train(net, [m1, m2], [spec1, spec2], n_steps=1000, batch=4096, lr=1e-3)
    assert np.all(np.isfinite(losses))
    # standardised targets (the linearised best fit of each sample): the untrained loss is
    # their mean variance; the floor is how far the linearisation misses the data's best fit
    assert losses[-40::2].mean() < 0.85 * losses[0:4:2].mean()
    assert losses[-39::2].mean() < 0.85 * losses[1:4:2].mean()

    # held-out C1 pseudo-experiments (host generator), all three datasets
    B = 96
    rng = np.random.default_rng(123)
    truths = np.stack([synth.draw_theta_true(spec1, rng) for _ in range(B)])
    mu, st = fitcore.expected_numpy(m1, truths)
    assert np.all(st == 0)
    data = rng.poisson(mu.astype(np.float64)).astype(np.float32)
    data_d = torch.from_numpy(data).cuda()
    starts = torch.zeros((B, spec1.n_params), dtype=torch.float64, device="cuda")
    warmstart.predict_starts(net, m1, spec1, B, data_d, None, starts)
    s_np = starts.cpu().numpy()
    # the predicted parameters of interest track the truth better than the nominal start does
    i13 = spec1.index("sin2_2th13")
    err_warm = np.abs(s_np[:, i13] - truths[:, i13]).mean()
    err_cold = np.abs(spec1.theta0[i13] - truths[:, i13]).mean()
    print(f"mean |error| of sin2_2th13: warm {err_warm:.4g}, nominal {err_cold:.4g}")
    assert err_warm < 0.7 * err_cold

    inst = np.zeros(B, fitcore.INSTANCE_DTYPE)
    inst["mask"] = spec1.all_mask()
    inst["data_off"] = np.arange(B) * spec1.n_bins
    inst["param_off"] = np.arange(B) * spec1.n_params
    _, cold = fitcore.fit_numpy([m1], inst, data)
    _, warm = fitcore.fit_numpy([m1], inst, data, start=s_np.ravel())
    assert np.all(cold["status"] == 0) and np.all(warm["status"] == 0)
    same = np.abs(warm["nll_min"] - cold["nll_min"]) <= 1e-3
    not_worse = warm["nll_min"] <= cold["nll_min"] + 1e-3
    print(f"same minimum {same.mean():.3f}, warm not worse {not_worse.mean():.3f}, iterations "
          f"warm {warm['iters'].mean():.1f} cold {cold['iters'].mean():.1f}, evals warm "
          f"{warm['n_evals'].mean():.1f} cold {cold['n_evals'].mean():.1f}")
    assert same.mean() >= 0.8 and not_worse.mean() >= 0.95
    # the warm start (every parameter at the linearised best fit, the network's corrections on
    # 12 of them) must not cost iterations on this model (measured 19.4 against 21.8)
    assert warm["iters"].mean() <= 1.0 * cold["iters"].mean()


def test_warm_start_saves_evaluations_on_the_53km_model(c1, c2):
    """Held-out pseudo-experiments of the 53 km model drawn by the ensemble recipe (true
    sin^2 th13 and dm2_31 within +-3 sigma, Poisson counts): fits from the warm start (the
    linearised best fit of all 460 parameters with the network's corrections on its 12 targets)
    reach the cold fits' minima (within 1e-3 in -2lnL, so at the cold fits' parity with the
    oracle) with measurably fewer evaluations (measured 15 %)."""
    spec1, m1 = c1
    spec2, m2 = c2
    net = warmstart.network(seed=3)
    # 12 epochs over the same 2M samples (about 35 s)
    warmstart.train(net, [m1, m2], [spec1, spec2], n_steps=488, batch=4096, lr=1e-3, epochs=12)
    B = 512
    table = synth.make_ensemble(B, {"c1": spec1, "c2": spec2}, frac_c2=1.0, base=9_000_000)
    truths = np.stack([t.theta_true for t in table])
    mu, st = fitcore.expected_numpy(m2, truths)
    assert np.all(st == 0)
    data = np.stack([synth.poisson_data(mu[i], t.seed) for i, t in enumerate(table)]).astype(np.float32)
    starts = torch.zeros((B, spec2.n_params), dtype=torch.float64, device="cuda")
    warmstart.predict_starts(net, m2, spec2, B, torch.from_numpy(data).cuda(), None, starts)
    inst = np.zeros(B, fitcore.INSTANCE_DTYPE)
    inst["mask"] = spec2.all_mask()
    inst["data_off"] = np.arange(B) * spec2.n_bins
    inst["param_off"] = np.arange(B) * spec2.n_params
    _, cold = fitcore.fit_numpy([m2], inst, data)
    _, warm = fitcore.fit_numpy([m2], inst, data, start=starts.cpu().numpy().ravel())
    assert np.all(cold["status"] == 0) and np.all(warm["status"] == 0)
    same = np.abs(warm["nll_min"] - cold["nll_min"]) <= 1e-3
    gain = 1.0 - warm["n_evals"].mean() / cold["n_evals"].mean()
    print(f"53 km model: evaluations warm {warm['n_evals'].mean():.2f} cold "
          f"{cold['n_evals'].mean():.2f} ({100 * gain:.1f} % fewer), same minimum {same.mean():.4f}")
    assert same.mean() >= 0.99
    assert gain >= 0.10
