"""The 3+1 sterile-neutrino search on the device: the three-dataset model with the exact 3+1
vacuum survival (two new parameters, sin^2 2th14 and dm2_41; "Sterile neutrino searches")
against the FP64 oracle — expectation, -2lnL and gradient away from the null point, fits with
the sterile parameters held (both engines), and a raster of the two parameters (Eq. 7) — and
per-event reweighting with the 3+1 formula.

Bars as in the other parity tests: expectation 2e-5 per bin, -2lnL 1e-3 (+2e-7 sum|mu - n|
away from the minimum), gradient 1e-5 in whitened units, fit minima 1e-3, event spectra 2e-6
of the unoscillated bin content."""
import numpy as np
import pytest

import oracle
from paper_2502_15253_gb300 import fitcore, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1s():
    spec = synth.make_model("c1s")
    om = oracle.OracleModel(spec)
    gm = fitcore.Model(spec)
    return spec, om, gm


def _sterile(spec, theta, s14, dm41):
    th = theta.copy()
    th[spec.index("sin2_2th14")] = s14
    th[spec.index("dm2_41")] = dm41
    return th


def test_expectation_and_gradient_with_sterile_mixing(c1s):
    spec, om, gm = c1s
    rng = np.random.default_rng(3)
    data = synth.poisson_data(om.expected(spec.theta0), 4)
    scale = np.where(spec.prior_sigma > 0, spec.prior_sigma, spec.scale)
    pts = [(0.1, 0.5), (0.05, 2e-3), (0.2, 3.0)]
    th = np.stack([_sterile(spec, om.theta_of_z(0.3 * rng.standard_normal(spec.n_params)), a, b)
                   for a, b in pts])
    mu, st = fitcore.expected_numpy(gm, th)
    assert np.all(st == 0)
    nll, g, st = fitcore.eval_numpy(gm, th, np.tile(data, (len(th), 1)))
    assert np.all(st == 0)
    for b in range(len(th)):
        ref = om.expected(th[b])
        np.testing.assert_allclose(mu[b], ref, rtol=2e-5, atol=1e-6 * ref.max())
        nref, gref = om.nll(th[b], data, grad=True)
        assert abs(nll[b] - nref) <= 1e-3 + 2e-7 * np.abs(ref - data).sum(), (b, nll[b], nref)
        err = np.linalg.norm((g[b] - gref) * scale) / np.linalg.norm(gref * scale)
        assert err <= 1e-5, (b, err)
    # the sterile term changes the spectrum where it should (short baselines, large dm2_41)
    mu0, _ = fitcore.expected_numpy(gm, _sterile(spec, th[0], 0.0, 0.5)[None, :])
    assert np.abs(mu[0] - mu0[0]).max() > 1e-2 * mu0[0].max()


def test_tensor_core_expectation(c1s):
    spec, om, gm = c1s
    th = np.stack([_sterile(spec, spec.theta0, 0.1, 0.5), _sterile(spec, spec.theta0, 0.03, 0.01)])
    mu = np.zeros((2, spec.n_bins), np.float32)
    st = np.zeros(2, np.int32)
    fitcore.fit_model_expected_tc(gm, 2, th, mu, st, 1)
    assert np.all(st == 0)
    for b in range(2):
        np.testing.assert_allclose(mu[b], om.expected(th[b]), rtol=2e-5)


@pytest.mark.parametrize("engine", [0, 1], ids=["persistent", "lockstep"])
def test_fits_with_held_sterile_parameters(c1s, engine):
    spec, om, gm = c1s
    i14, i41 = spec.index("sin2_2th14"), spec.index("dm2_41")
    truth = _sterile(spec, spec.theta0, 0.08, 0.3)
    data = synth.poisson_data(om.expected(truth), 6)
    pts = [(0.0, 0.3), (0.08, 0.3), (0.15, 0.05)]
    P = spec.n_params
    inst = np.zeros(len(pts), fitcore.INSTANCE_DTYPE)
    inst["mask"] = spec.all_mask()
    inst["param_off"] = np.arange(len(pts)) * P
    starts = np.stack([_sterile(spec, spec.theta0, a, b) for a, b in pts])
    fixed = np.zeros((len(pts), P), np.uint8)
    fixed[:, [i14, i41]] = 1
    o = fitcore.fit_batch_default_opts()
    o.engine = engine
    best, res = fitcore.fit_numpy([gm], inst, data, start=starts.ravel(), opts=o, fixed=fixed.ravel())
    fx = np.zeros(P, bool)
    fx[[i14, i41]] = True
    for k in range(len(pts)):
        assert res[k]["status"] == 0
        th = best[k * P:(k + 1) * P]
        assert th[i14] == pytest.approx(pts[k][0], abs=1e-12) and th[i41] == pytest.approx(pts[k][1], rel=1e-9)
        ref = om.fit(data, start=starts[k], fixed=fx)
        assert ref["status"] == 0
        assert abs(res[k]["nll_min"] - ref["nll"]) <= 1e-3, (k, res[k]["nll_min"], ref["nll"])


def test_sterile_raster_scan(c1s):
    """A 3 x 3 raster in (sin^2 2th14, dm2_41) on pseudo-data with an injected sterile signal:
    device scan against the oracle's constrained fits, and the raster minimum at the injected
    point."""
    spec, om, gm = c1s
    i14, i41 = spec.index("sin2_2th14"), spec.index("dm2_41")
    data = om.expected(_sterile(spec, spec.theta0, 0.1, 0.4)).astype(np.float32)   # Asimov
    pts = np.array([[a, b] for a in (0.0, 0.1, 0.2) for b in (0.2, 0.4, 0.8)])
    r = fitcore.fit_profile_scan(gm, data, spec.all_mask(), [i14, i41], pts)
    assert np.all(r["status"] == 0)
    np.testing.assert_allclose(r["theta"][:, [i14, i41]], pts, rtol=1e-9, atol=1e-12)
    assert int(np.argmin(r["dchi2"])) == 4            # (0.1, 0.4)
    fx = np.zeros(spec.n_params, bool)
    fx[[i14, i41]] = True
    for k in (0, 4, 8):
        ref = om.fit(data, start=_sterile(spec, spec.theta0, *pts[k]), fixed=fx)
        assert abs(r["dchi2"][k] + r["nll_min"] - ref["nll"]) <= 1e-3, (k, r["dchi2"][k], ref["nll"])


def test_event_spectrum_with_sterile_state():
    ev = synth.make_mc_events(300_000, "dc_fd")
    ev.osc_mode = synth.OSC_STERILE4
    ev.osc_nominal = np.array([0.307, 0.0231, 7.53e-5, 2.5e-3, 0.0, 0.1])
    params = np.array([[0.307, 0.0231, 7.53e-5, 2.5e-3, 0.0, 0.1],
                       [0.307, 0.0231, 7.53e-5, 2.5e-3, 0.1, 0.5],
                       [0.30, 0.025, 7.4e-5, -2.45e-3, 0.05, 2.0]])
    mc = fitcore.McEventSet(ev)
    out = np.zeros((3, ev.n_bins))
    mc.spectrum(3, params, out)
    W = np.bincount(ev.bin, weights=ev.weight.astype(np.float64), minlength=ev.n_bins)
    for b in range(3):
        ref = oracle.event_spectrum(ev, params[b])
        assert np.all(np.abs(out[b] - ref) <= 2e-6 * W + 1e-300), b
    assert np.abs(out[1] - out[0]).max() > 1e-2 * out[0].max()
