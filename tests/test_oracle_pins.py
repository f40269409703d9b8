"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks one oracle function against an independent source: a brute-force PMNS
amplitude sum, the paper's closed forms (Eq. 1, the corrected Eq. 10, Eq. 2), library
probability routines (scipy Poisson PMF, multivariate normal), a fine-grid integration of the
energy map, closed-form minima, and a brute-force grid scan. A plausible slip in the oracle
(a dropped term, a wrong sign, a transposed response, a wrong prior matrix) fails at least one.
"""
import copy

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2502_15253_gb300 import synth

K = 1.266932679815373  # dm2[eV^2] L[m] / (4 E[MeV])


# ---------------------------------------------------------------------------------------
# independent survival probabilities
# ---------------------------------------------------------------------------------------
def p_amplitude(s12, s13, dm21, dm31, L, E, delta=0.0):
    """|sum_i |U_ei|^2 exp(-i m_i^2 L / 2E)|^2 from the PMNS first row (m_1 = 0)."""
    ue = np.array([np.sqrt((1 - s12) * (1 - s13)), np.sqrt(s12 * (1 - s13)),
                   np.sqrt(s13) * np.exp(-1j * delta)])
    m2 = np.array([0.0, dm21, dm31])
    amp = (np.abs(ue) ** 2 * np.exp(-1j * 2.0 * K * m2 * L / E)).sum()
    return abs(amp) ** 2


def p_amplitude4(s12, s13, dm21, dm31, S14, dm41, L, E):
    """3+1: |sum_i |U_ei|^2 exp(-i m_i^2 L / 2E)|^2 with the first row (c12 c13 c14,
    s12 c13 c14, s13 c14, s14) of the 4x4 mixing matrix (m_1 = 0)."""
    s14 = 0.5 * (1.0 - np.sqrt(1.0 - S14))          # sin^2 th14 for th14 <= pi/4
    c14 = 1.0 - s14
    ue2 = np.array([(1 - s12) * (1 - s13) * c14, s12 * (1 - s13) * c14, s13 * c14, s14])
    m2 = np.array([0.0, dm21, dm31, dm41])
    amp = (ue2 * np.exp(-1j * 2.0 * K * m2 * L / E)).sum()
    return abs(amp) ** 2


def p_two_flavour_amplitude(theta, dm2, L, E):
    """2x2 rotation amplitude: |cos^2 th + sin^2 th exp(-i dm2 L / 2E)|^2."""
    amp = np.cos(theta) ** 2 + np.sin(theta) ** 2 * np.exp(-1j * 2.0 * K * dm2 * L / E)
    return abs(amp) ** 2


def p_eq10_corrected(s12, s13, dm21, dm31, L, E, sign=1.0):
    """Eq. 10 in its corrected reading: +phi for normal ordering, -phi (sign = -1) for
    inverted ordering; Delta m^2_ee of Eq. 2 taken in magnitude."""
    t12, t13 = np.arcsin(np.sqrt(s12)), np.arcsin(np.sqrt(s13))
    S12, S13 = np.sin(2 * t12) ** 2, np.sin(2 * t13) ** 2
    dmee = np.cos(t12) ** 2 * abs(dm31) + np.sin(t12) ** 2 * abs(dm31 - dm21)   # Eq. 2
    d21, dee = K * dm21 * L / E, K * dmee * L / E
    phi = np.arctan2(np.cos(2 * t12) * np.sin(d21), np.cos(d21)) - d21 * np.cos(2 * t12)
    return (1 - 0.5 * S13 * (1 - np.sqrt(1 - S12 * np.sin(d21) ** 2) * np.cos(2 * dee + sign * phi))
            - S12 * np.cos(t13) ** 4 * np.sin(d21) ** 2)


GRID = [(L, E) for L in (400.0, 1050.0, 52500.0) for E in np.linspace(1.8, 10.0, 37)]


def test_survival_zero_mixing_is_one():
    for L, E in GRID:
        assert oracle.survival(0, [0.0, 2.5e-3, 0.0, 7.5e-5], L, E) == 1.0
        assert oracle.survival(1, [0.0, 0.0, 7.5e-5, 2.5e-3], L, E) == 1.0
        assert oracle.survival(2, [0.0, 0.0, 7.5e-5, 2.5e-3, 0.0, 0.5], L, E) == 1.0


def test_sterile_matches_four_flavour_amplitude():
    rng = np.random.default_rng(4)
    for _ in range(300):
        s12, s13 = rng.uniform(0.05, 0.6), rng.uniform(0.0, 0.2)
        dm21, dm31 = rng.uniform(1e-5, 2e-4), rng.choice([-1, 1]) * rng.uniform(1e-3, 4e-3)
        S14, dm41 = rng.uniform(0.0, 0.99), 10 ** rng.uniform(-3.5, 0.5)
        L, E = rng.uniform(10, 6e4), rng.uniform(1.8, 10)
        p = [s12, s13, dm21, dm31, S14, dm41]
        # both sides take sines of phases up to ~1e5 rad: a few ulps of the phase each
        tol = 1e-13 + 1e-15 * 2.0 * K * dm41 * L / E
        assert oracle.survival(2, p, L, E) == pytest.approx(p_amplitude4(*p, L, E), abs=tol)


def test_sterile_without_sterile_mixing_is_three_flavour():
    for L, E in GRID:
        for dm41 in (1e-3, 0.05, 2.0):
            p3 = [0.307, 0.022, 7.5e-5, 2.5e-3]
            assert oracle.survival(2, p3 + [0.0, dm41], L, E) == pytest.approx(
                oracle.survival(1, p3, L, E), abs=4e-16)


def test_sterile_two_flavour_limit_matches_rotation_amplitude():
    """th12 = th13 = 0: P = 1 - sin^2 2th14 sin^2 x_41, the 2x2 rotation by th14."""
    for L, E in GRID:
        for S14, dm41 in ((0.1, 0.05), (0.3, 1.2)):
            th = 0.5 * np.arcsin(np.sqrt(S14))
            got = oracle.survival(2, [0.0, 0.0, 7.5e-5, 2.5e-3, S14, dm41], L, E)
            tol = 1e-14 + 1e-15 * 2.0 * K * dm41 * L / E   # ulps of phases up to ~5e4 rad
            assert got == pytest.approx(p_two_flavour_amplitude(th, dm41, L, E), abs=tol)


def test_vacuum3_matches_pmns_amplitude():
    rng = np.random.default_rng(0)
    for _ in range(200):
        s12, s13 = rng.uniform(0.05, 0.6), rng.uniform(0.0, 0.2)
        dm21, dm31 = rng.uniform(1e-5, 2e-4), rng.uniform(1e-3, 4e-3)
        L, E = rng.uniform(100, 6e4), rng.uniform(1.8, 10)
        delta = rng.uniform(0, 2 * np.pi)          # P_ee does not depend on the CP phase
        got = oracle.survival(1, [s12, s13, dm21, dm31], L, E)
        assert got == pytest.approx(p_amplitude(s12, s13, dm21, dm31, L, E, delta), abs=1e-13)


def test_vacuum3_matches_corrected_eq10():
    for L, E in GRID:
        p = [0.307, 0.022, 7.5e-5, 2.5e-3]
        assert oracle.survival(1, p, L, E) == pytest.approx(p_eq10_corrected(*p, L, E), abs=1e-13)


def test_inverted_ordering_is_eq10_with_minus_phi():
    """The exact vacuum formula at negative dm2_31 (inverted ordering) is the PMNS amplitude
    sum with m_3^2 < 0 and the corrected Eq. 10 with the sign of phi flipped; with +phi it is
    not (the two orderings differ at 53 km)."""
    s12, s13, dm21 = 0.307, 0.022, 7.5e-5
    worst_plus = 0.0
    for L, E in GRID:
        for dm31 in (-2.4e-3, -2.5e-3):
            p = [s12, s13, dm21, dm31]
            got = oracle.survival(1, p, L, E)
            assert got == pytest.approx(p_amplitude(*p, L, E), abs=1e-13)
            assert got == pytest.approx(p_eq10_corrected(*p, L, E, sign=-1.0), abs=1e-13)
            if L > 5e4:
                worst_plus = max(worst_plus, abs(got - p_eq10_corrected(*p, L, E, sign=1.0)))
    assert worst_plus > 1e-2


def test_eq1_two_flavour_limit_matches_rotation_amplitude():
    for L, E in GRID:
        th = 0.5 * np.arcsin(np.sqrt(0.09))
        got = oracle.survival(0, [0.09, 2.5e-3, 0.0, 7.53e-5], L, E)
        assert got == pytest.approx(p_two_flavour_amplitude(th, 2.5e-3, L, E), abs=1e-14)


def test_eq1_with_eq2_close_to_exact_at_short_baseline_only():
    """Eq. 1 + Eq. 2 approximates the exact probability to < 5e-5 at ~1 km, not at 52 km."""
    s12, s13, dm21, dm31 = 0.307, 0.022, 7.5e-5, 2.5e-3
    t12, t13 = np.arcsin(np.sqrt(s12)), np.arcsin(np.sqrt(s13))
    S12, S13 = np.sin(2 * t12) ** 2, np.sin(2 * t13) ** 2
    dmee = np.cos(t12) ** 2 * dm31 + np.sin(t12) ** 2 * (dm31 - dm21)
    short, far = 0.0, 0.0
    for E in np.linspace(1.8, 10.0, 400):
        for L, acc in ((1050.0, "s"), (52500.0, "f")):
            d = abs(oracle.survival(0, [S13, dmee, S12, dm21], L, E)
                    - p_amplitude(s12, s13, dm21, dm31, L, E))
            if acc == "s":
                short = max(short, d)
            else:
                far = max(far, d)
    assert short < 5e-5
    assert far > 1e-2


@pytest.mark.parametrize("mode,p", [(0, [0.09, 2.5e-3, 0.851, 7.53e-5]),
                                    (1, [0.307, 0.022, 7.5e-5, 2.5e-3]),
                                    (2, [0.307, 0.022, 7.5e-5, 2.5e-3, 0.05, 0.3])])
def test_survival_partials_match_central_differences(mode, p):
    for L, E in GRID[::5]:
        _, dp = oracle.survival(mode, p, L, E, with_grad=True)
        for i in range(len(p)):
            h = 1e-6 * abs(p[i])
            if p[i] < 1e-2 or i == 5:   # a mass splitting: keep the phase step below 1e-4 rad
                h = min(h, 1e-4 / (K * L / E))
            pp, pm = list(p), list(p)
            pp[i] += h
            pm[i] -= h
            fd = (oracle.survival(mode, pp, L, E) - oracle.survival(mode, pm, L, E)) / (2 * h)
            assert dp[i] == pytest.approx(fd, rel=1e-6, abs=1e-9 / abs(p[i]))


# ---------------------------------------------------------------------------------------
# energy correction (remap)
# ---------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c0():
    spec = synth.make_model("c0")
    return spec, oracle.OracleModel(spec)


def test_remap_identity_bit_exact(c0):
    spec, om = c0
    u = np.random.default_rng(1).uniform(0, 10, spec.n_true)
    assert np.array_equal(om.remap([0.0, 1.0, 0.0], u), u)


def test_remap_whole_bin_shift(c0):
    spec, om = c0
    de = (spec.e_hi - spec.e_lo) / spec.n_true
    u = np.random.default_rng(2).uniform(0, 10, spec.n_true)
    for m in (1, 3, -2):
        v = om.remap([m * de, 1.0, 0.0], u)
        ref = np.zeros_like(u)
        if m > 0:
            ref[m:] = u[:-m]
        else:
            ref[:m] = u[-m:]
        np.testing.assert_allclose(v, ref, rtol=1e-9, atol=1e-9)


# area-conserving spline remap ---------------------------------------------------------
@pytest.fixture(scope="module")
def c0s():
    spec = synth.make_model("c0", remap=1)
    return spec, oracle.OracleModel(spec)


def _spline_reference(spec, a, u):
    """The same definition through a library interpolant: scipy's cubic Hermite spline of the
    cumulative content at the edges with the averaged-density edge slopes, differenced at the
    inverse-mapped edges (roots of the quadratic by numpy)."""
    from scipy.interpolate import CubicHermiteSpline
    n = spec.n_true
    edges = np.linspace(spec.e_lo, spec.e_hi, n + 1)
    de = edges[1] - edges[0]
    rho = u / de
    slope = np.concatenate([[rho[0]], 0.5 * (rho[:-1] + rho[1:]), [rho[-1]]])
    F = CubicHermiteSpline(edges, np.concatenate([[0.0], np.cumsum(u)]), slope)
    x = np.array([max(np.roots([a[2], a[1], a[0] - e]).real, key=lambda r: -abs(r - e))
                  if a[2] != 0 else (e - a[0]) / a[1] for e in edges])
    Fx = np.where(x <= edges[0], 0.0, np.where(x >= edges[-1], u.sum(), F(np.clip(x, edges[0], edges[-1]))))
    return np.diff(Fx)


def test_spline_remap_identity_and_whole_bin_shift(c0s):
    spec, om = c0s
    de = (spec.e_hi - spec.e_lo) / spec.n_true
    u = np.random.default_rng(5).uniform(0, 10, spec.n_true)
    np.testing.assert_allclose(om.remap([0.0, 1.0, 0.0], u), u, rtol=1e-12, atol=1e-12)
    for m in (1, 3, -2):
        ref = np.zeros_like(u)
        if m > 0:
            ref[m:] = u[:-m]
        else:
            ref[:m] = u[-m:]
        np.testing.assert_allclose(om.remap([m * de, 1.0, 0.0], u), ref, rtol=1e-10, atol=1e-10)


def test_spline_remap_matches_library_hermite_spline(c0s):
    spec, om = c0s
    u = np.random.default_rng(6).uniform(1, 5, spec.n_true)
    for a in ([0.02, 1.003, -0.0005], [-0.03, 0.99, 0.001], [0.013, 1.0, 0.0], [0.0, 1.02, 0.0]):
        np.testing.assert_allclose(om.remap(a, u), _spline_reference(spec, a, u), rtol=1e-10,
                                   atol=1e-10 * u.sum())


def test_spline_remap_is_smooth_where_the_overlap_rule_kinks(c0, c0s):
    """At a0 = one or two bins every mapped edge sits on a grid edge: there the overlap rule's
    derivative jumps, the spline's left and right derivatives agree. (Content that starts
    abruptly at a grid end would still kink the spline where a mapped edge crosses that end;
    the spectra, like the model's, go to zero there.)"""
    (spec, om), (_, oms) = c0, c0s
    de = (spec.e_hi - spec.e_lo) / spec.n_true
    u = np.zeros(spec.n_true)
    u[10:-10] = np.random.default_rng(7).uniform(1, 5, spec.n_true - 20)
    gv = np.random.default_rng(8).standard_normal(spec.n_true)
    h = 1e-6 * de
    for a0 in (de, 2 * de):
        def phi(m, x):
            return m.remap([x, 1.0, 0.0], u) @ gv
        right_s = (phi(oms, a0 + h) - phi(oms, a0)) / h
        left_s = (phi(oms, a0) - phi(oms, a0 - h)) / h
        right_o = (phi(om, a0 + h) - phi(om, a0)) / h
        left_o = (phi(om, a0) - phi(om, a0 - h)) / h
        assert abs(right_s - left_s) <= 1e-4 * max(abs(right_s), 1.0)
        assert abs(right_o - left_o) > 1e-2 * max(abs(right_o), 1.0)


def test_remap_conserves_content_inside_grid(c0):
    spec, om = c0
    u = np.zeros(spec.n_true)
    u[30:170] = np.random.default_rng(3).uniform(1, 5, 140)
    for a in ([0.02, 1.003, -0.0005], [-0.03, 0.99, 0.001], [0.0, 1.0, 0.0008]):
        assert om.remap(a, u).sum() == pytest.approx(u.sum(), rel=1e-12)


def test_remap_matches_fine_grid_integration(c0):
    """Brute force: split every source bin into 4000 equal pieces, map each piece's centre."""
    spec, om = c0
    edges = spec.true_edges
    u = np.random.default_rng(4).uniform(1, 5, spec.n_true)
    a = np.array([0.013, 1.004, 0.0007])
    n_sub = 4000
    frac = (np.arange(n_sub) + 0.5) / n_sub
    ref = np.zeros(spec.n_true)
    for k in range(spec.n_true):
        x = edges[k] + frac * (edges[k + 1] - edges[k])
        y = a[0] + a[1] * x + a[2] * x * x
        t = np.floor((y - spec.e_lo) / (edges[1] - edges[0])).astype(int)
        ok = (t >= 0) & (t < spec.n_true)
        np.add.at(ref, t[ok], u[k] / n_sub)
    np.testing.assert_allclose(om.remap(a, u), ref, rtol=0, atol=2e-3 * u.max())


# ---------------------------------------------------------------------------------------
# deviance, priors, expectation
# ---------------------------------------------------------------------------------------
def test_deviance_is_saturated_poisson_ratio():
    for n in (0, 1, 3, 17, 250, 4000):
        for mu in (0.3, 2.5, 17.2, 260.0, 3900.0):
            ref = -2.0 * (stats.poisson.logpmf(n, mu) - stats.poisson.logpmf(n, n)) if n else 2 * mu
            assert oracle.deviance(n, mu) == pytest.approx(ref, rel=1e-10, abs=1e-10)
    assert oracle.deviance(42.0, 42.0) == 0.0
    assert oracle.deviance(5.0, 0.0) == np.inf


def test_prior_only_nll_is_gaussian_logpdf():
    """No dataset enabled: -2lnL is the prior of Eq. 6, i.e. -2 ln N(theta) up to a constant."""
    spec = synth.make_model("c1")
    om = oracle.OracleModel(spec)
    rng = np.random.default_rng(5)
    theta = om.theta_of_z(rng.standard_normal(spec.n_params))
    ref = 0.0
    for i in range(spec.n_params):
        if spec.prior_sigma[i] > 0:
            ref += -2 * (stats.norm.logpdf(theta[i], spec.theta0[i], spec.prior_sigma[i])
                         - stats.norm.logpdf(spec.theta0[i], spec.theta0[i], spec.prior_sigma[i]))
    for idx, cov in spec.cov_blocks:
        mvn = stats.multivariate_normal(spec.theta0[idx], cov)
        ref += -2 * (mvn.logpdf(theta[idx]) - mvn.logpdf(spec.theta0[idx]))
    assert om.nll(theta, np.zeros(spec.n_bins), mask=0) == pytest.approx(ref, rel=1e-9)


def test_transformation_layer_whitens_the_prior():
    spec = synth.make_model("c1")
    om = oracle.OracleModel(spec)
    z = np.random.default_rng(6).standard_normal(spec.n_params)
    theta = om.theta_of_z(z)
    np.testing.assert_allclose(om.z_of_theta(theta), z, atol=1e-10)
    prior_only = om.nll(theta, np.zeros(spec.n_bins), mask=0)
    constrained = (spec.prior_sigma > 0) | np.isin(np.arange(spec.n_params),
                                                   np.concatenate([i for i, _ in spec.cov_blocks]))
    assert prior_only == pytest.approx((z[constrained] ** 2).sum(), rel=1e-9)


def test_response_column_sums_equal_efficiency_times_coverage():
    for name in ("c0", "c1", "c2"):
        spec = synth.make_model(name)
        ec = 0.5 * (spec.true_edges[:-1] + spec.true_edges[1:])
        for det, res in zip(spec.detectors, {"c0": [0.08], "c1": [0.08, 0.08],
                                             "c2": [0.03, 0.03]}[name]):
            evis = ec - synth.PROMPT_SHIFT_MEV
            sig = res * np.sqrt(evis)
            cover = (stats.norm.cdf((det.reco_edges[-1] - evis) / sig)
                     - stats.norm.cdf((det.reco_edges[0] - evis) / sig))
            np.testing.assert_allclose(det.response.sum(0), synth.RESPONSE_EPS0 * cover,
                                       atol=1e-10)


def test_expected_matches_matrix_form_with_amplitude_probability():
    """mu = eps R (t n s sum_c p_c w_c P_c) + backgrounds at nominal energy scale, with P from
    the PMNS amplitude and the fold as a library matrix product."""
    spec = synth.make_model("c2")
    om = oracle.OracleModel(spec)
    theta = spec.theta0.copy()
    rng = np.random.default_rng(7)
    for i in range(spec.n_params):
        if not spec.param_names[i].startswith("a"):
            theta[i] += 0.5 * rng.standard_normal() * (spec.prior_sigma[i] or spec.scale[i])
    mu = om.expected(theta)
    s12, s13, dm21, dm31 = theta[spec.osc_idx]
    ec = 0.5 * (spec.true_edges[:-1] + spec.true_edges[1:])
    off = spec.data_offsets()
    for d, ds in enumerate(spec.datasets):
        ptot = np.zeros(spec.n_true)
        for c in range(spec.n_cores):
            pw = theta[spec.core_power_idx[c]]
            ptot += pw * ds.weight[c] * np.array(
                [p_amplitude(s12, s13, dm21, dm31, ds.baseline[c], e) for e in ec])
        u = ds.t * theta[ds.norm_idx] * theta[ds.shape_idx] * ptot
        ref = spec.detectors[ds.det].response @ u
        np.testing.assert_allclose(mu[off[d]:off[d + 1]], ref, rtol=1e-11)


def test_expected_backgrounds_and_efficiency_c1():
    spec = synth.make_model("c1")
    om = oracle.OracleModel(spec)
    theta = spec.theta0.copy()
    s13 = spec.index("sin2_2th13")
    theta[s13] = 0.0
    theta[spec.index("sin2_2th12")] = 0.0           # no oscillation: P = 1
    rng = np.random.default_rng(8)
    bkg = [i for i, n in enumerate(spec.param_names) if "rate" in n or "li9_shape" in n
           or "acc_shape" in n or n.startswith("eff")]
    theta[bkg] += 0.05 * rng.standard_normal(len(bkg))
    mu = om.expected(theta)
    off = spec.data_offsets()
    for d, ds in enumerate(spec.datasets):
        u = ds.t * theta[ds.shape_idx] * (theta[spec.core_power_idx] * ds.weight).sum()
        ref = theta[ds.eff_idx] * (spec.detectors[ds.det].response @ u)
        for b in ds.backgrounds:
            sh = np.where(b.shape_idx >= 0, theta[np.maximum(b.shape_idx, 0)], 0.0)
            ref = ref + theta[b.rate_idx] * b.template * (1 + sh)
        np.testing.assert_allclose(mu[off[d]:off[d + 1]], ref, rtol=1e-11)


# ---------------------------------------------------------------------------------------
# -2lnL and gradient
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["c0", "c1", "c2", "c1s", "c0/spline", "c1/spline", "c1_flux41"])
def test_asimov_nll_is_zero(name):
    spec = synth.make_model(name.split("/")[0], remap=int(name.endswith("spline")))
    om = oracle.OracleModel(spec)
    v, g = om.nll(spec.theta0, om.expected(spec.theta0), grad=True)
    assert abs(v) < 1e-9
    assert np.abs(g).max() < 1e-6


def test_poisson_part_equals_library_pmf_sum():
    spec = synth.make_model("c1")
    om = oracle.OracleModel(spec)
    theta = spec.theta0.copy()
    mu = om.expected(theta)
    data = synth.poisson_data(mu, 11)
    ref = -2.0 * (stats.poisson.logpmf(data, mu) - stats.poisson.logpmf(data, data)).sum()
    assert om.nll(theta, data) == pytest.approx(ref, rel=1e-10)
    # masking datasets drops exactly their bins
    off = spec.data_offsets()
    m = 0b101
    keep = np.concatenate([np.arange(off[d], off[d + 1]) for d in (0, 2)])
    ref_m = -2.0 * (stats.poisson.logpmf(data[keep], mu[keep])
                    - stats.poisson.logpmf(data[keep], data[keep])).sum()
    assert om.nll(theta, data, mask=m) == pytest.approx(ref_m, rel=1e-10)


@pytest.mark.parametrize("name", ["c0", "c1", "c2", "c1s", "c0/spline", "c1/spline", "c2/spline",
                                  "c1_flux41"])
def test_gradient_matches_central_differences(name):
    spec = synth.make_model(name.split("/")[0], remap=int(name.endswith("spline")))
    om = oracle.OracleModel(spec)
    rng = np.random.default_rng(9)
    data = synth.poisson_data(om.expected(spec.theta0), 12)
    theta = om.theta_of_z(0.4 * rng.standard_normal(spec.n_params))
    _, g = om.nll(theta, data, grad=True)
    scale = np.where(spec.prior_sigma > 0, spec.prior_sigma, spec.scale)
    idx = np.arange(spec.n_params) if spec.n_params < 60 else np.unique(
        np.concatenate([np.arange(20), rng.choice(spec.n_params, 40, replace=False)]))
    for i in idx:
        h = 1e-6 * scale[i]
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (om.nll(tp, data) - om.nll(tm, data)) / (2 * h)
        # compare in units of the parameter's scale (z units)
        assert abs(fd - g[i]) * scale[i] < 1e-5 * (1 + abs(g[i]) * scale[i]), spec.param_names[i]


# ---------------------------------------------------------------------------------------
# minimiser
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["c0", "c1"])
def test_asimov_fit_recovers_injected_parameters(name):
    spec = synth.make_model(name)
    om = oracle.OracleModel(spec)
    # shift only parameters without a prior, so the injected point has -2lnL = 0 exactly
    truth = spec.theta0.copy()
    free = [i for i in range(spec.n_params) if spec.prior_sigma[i] == 0
            and not any(i in idx for idx, _ in spec.cov_blocks)]
    truth[free] += 1.5 * spec.scale[free]
    data = om.expected(truth)
    assert om.nll(truth, data) == pytest.approx(0.0, abs=1e-9)
    r = om.fit(data)
    assert r["status"] == 0
    assert abs(r["nll"]) < 1e-7
    sig = om.sigma(r["theta"], data)
    assert np.all(np.abs(r["theta"] - truth) < 1e-3 * sig + 1e-12)


def _norm_only(spec):
    """C0 geometry with one free parameter: the signal normalisation; no backgrounds."""
    s = copy.deepcopy(spec)
    inorm = s.index("norm")
    ds = s.datasets[0]
    ds.backgrounds = []
    ds.escale_idx = np.array([-1, -1, -1], np.int32)
    ds.shape_idx = np.full(s.n_true, -1, np.int32)
    s.osc_idx = np.array([-1, -1, -1, -1], np.int32)
    s.cov_blocks = []
    s.param_names = ["norm"]
    s.theta0 = np.array([1.0])
    s.prior_sigma = np.array([0.0])
    s.scale = np.array([0.01])
    ds.norm_idx = 0
    del inorm
    return s


def test_pure_scale_fit_closed_form():
    """mu = s mu0 gives the Poisson MLE s_hat = sum n / sum mu0 (Eq. 3-5)."""
    spec = _norm_only(synth.make_model("c0"))
    om = oracle.OracleModel(spec)
    mu0 = om.expected(np.array([1.0]))
    data = synth.poisson_data(1.07 * mu0, 13)
    r = om.fit(data, edm_tol=1e-14)
    assert r["theta"][0] == pytest.approx(data.sum() / mu0.sum(), rel=1e-9)


def test_prior_only_fit_returns_prior_means_and_covariance():
    spec = synth.make_model("c0")
    om = oracle.OracleModel(spec)
    start = om.theta_of_z(np.random.default_rng(14).standard_normal(spec.n_params))
    zero = np.zeros(spec.n_bins)
    r = om.fit(zero, mask=0, start=start)
    constrained = spec.prior_sigma > 0
    for idx, _ in spec.cov_blocks:
        constrained[idx] = True
    np.testing.assert_allclose(r["theta"][constrained], spec.theta0[constrained], atol=1e-7)
    H = om.hessian(spec.theta0, zero, mask=0)
    sub = np.flatnonzero(constrained)
    V = 2.0 * np.linalg.inv(H[np.ix_(sub, sub)])
    ref = np.zeros((spec.n_params, spec.n_params))
    for i in sub:
        ref[i, i] = spec.prior_sigma[i] ** 2
    for idx, cov in spec.cov_blocks:
        ref[np.ix_(idx, idx)] = cov
    np.testing.assert_allclose(V, ref[np.ix_(sub, sub)], rtol=1e-6, atol=1e-12)


def test_grid_scan_matches_fit_minimum():
    """Two free parameters (sin^2 2th13, dm2_ee): a 401 x 401 scan plus local refinement."""
    spec = synth.make_model("c0_tiny")
    om = oracle.OracleModel(spec)
    truth = np.array([0.085, 2.45e-3])
    data = synth.poisson_data(om.expected(truth), 15)
    r = om.fit(data)
    assert r["status"] == 0
    s13 = np.linspace(0.0, 0.2, 401)
    dm = np.linspace(1.5e-3, 3.5e-3, 401)
    vals = np.array([[om.nll([a, b], data) for b in dm] for a in s13])
    i, j = np.unravel_index(np.argmin(vals), vals.shape)
    best = vals[i, j]
    ca, cb = s13[i], dm[j]
    wa, wb = s13[1] - s13[0], dm[1] - dm[0]
    wa, wb = 3 * wa, 3 * wb
    for _ in range(14):                     # zoomed 21 x 21 rescans around the best point
        aa = np.linspace(ca - wa, ca + wa, 21)
        bb = np.linspace(cb - wb, cb + wb, 21)
        v2 = np.array([[om.nll([a, b], data) for b in bb] for a in aa])
        i, j = np.unravel_index(np.argmin(v2), v2.shape)
        ca, cb, best = aa[i], bb[j], min(best, v2[i, j])
        wa, wb = wa / 3, wb / 3
    assert r["nll"] == pytest.approx(best, abs=1e-6)
    assert r["nll"] <= best + 1e-9


def test_fixed_parameter_fit_is_the_profile_minimum():
    """Profile likelihood (Eq. 7): with sin^2 2th13 held at a, the fit over dm2_ee returns the
    minimum of -2lnL(a, .) found by a brute-force 1-D scan with zoomed refinement; the profile
    is >= the global minimum and touches it at the unconstrained best fit."""
    spec = synth.make_model("c0_tiny")
    om = oracle.OracleModel(spec)
    data = synth.poisson_data(om.expected(np.array([0.085, 2.45e-3])), 15)
    glob = om.fit(data)
    assert glob["status"] == 0
    fixed = np.array([True, False])
    for a in (0.04, 0.085, 0.13, glob["theta"][0]):
        r = om.fit(data, start=[a, 2.5e-3], fixed=fixed)
        assert r["status"] == 0 and r["theta"][0] == pytest.approx(a, rel=1e-14)
        dm = np.linspace(1.5e-3, 3.5e-3, 2001)
        v = np.array([om.nll([a, b], data) for b in dm])
        c, w, best = dm[np.argmin(v)], 3 * (dm[1] - dm[0]), v.min()
        for _ in range(14):
            bb = np.linspace(c - w, c + w, 21)
            v2 = np.array([om.nll([a, b], data) for b in bb])
            c, best, w = bb[np.argmin(v2)], min(best, v2.min()), w / 3
        assert r["nll"] == pytest.approx(best, abs=1e-6)
        assert r["nll"] >= glob["nll"] - 1e-9
    r = om.fit(data, start=glob["theta"], fixed=fixed)
    assert r["nll"] == pytest.approx(glob["nll"], abs=1e-8)


def test_fixing_a_parameter_inside_a_prior_block_is_rejected():
    spec = synth.make_model("c0")
    om = oracle.OracleModel(spec)
    idx = spec.cov_blocks[0][0][0]
    fixed = np.zeros(spec.n_params, bool)
    fixed[idx] = True
    r = om.fit(om.expected(spec.theta0), fixed=fixed)
    assert r["status"] == 4


# ---------------------------------------------------------------------------------------
# event-level reweighting
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("geometry", ["dc_fd", "juno_fd"])
def test_event_spectrum_zero_mixing_is_weighted_counts(geometry):
    ev = synth.make_mc_events(200_000, geometry)
    p = np.array([0.0, 2.5e-3, 0.0, 7.5e-5]) if ev.osc_mode == 0 else np.array([0.0, 0.0, 7.5e-5, 2.5e-3])
    got = oracle.event_spectrum(ev, p)
    ref = np.bincount(ev.bin, weights=ev.weight.astype(np.float64), minlength=ev.n_bins)
    np.testing.assert_allclose(got, ref, rtol=1e-12)


@pytest.mark.parametrize("geometry", ["dc_fd", "juno_fd"])
def test_event_spectrum_is_the_per_event_sum(geometry):
    ev = synth.make_mc_events(3000, geometry)
    p = ev.osc_nominal
    ref = np.zeros(ev.n_bins)
    for e, c, w, b in zip(ev.energy, ev.core, ev.weight, ev.bin):
        ref[b] += float(w) * oracle.survival(ev.osc_mode, p, ev.core_L[c], float(e))
    np.testing.assert_allclose(oracle.event_spectrum(ev, p), ref, rtol=1e-13, atol=1e-15)


# ---------------------------------------------------------------------------------------
# Eq. 6 with a linear generalised parametrisation b = A theta
# ---------------------------------------------------------------------------------------
def _spd(rng, n):
    Q = rng.standard_normal((n, n))
    return Q @ Q.T + n * np.eye(n)


def test_linear_prior_block_reproduces_the_quadratic_form():
    """9 constrained coefficients from 7 parameters (the energy-scale case of the detector
    response): at random points the two quadratic forms differ by one constant, which is >= 0
    and equals the form's minimum over theta."""
    rng = np.random.default_rng(11)
    m, k = 9, 7
    A, b0, V = rng.standard_normal((m, k)), rng.standard_normal(m), _spd(rng, m)
    t, Cb, const = oracle.linear_prior_block(A, b0, V)
    Vi, Ci = np.linalg.inv(V), np.linalg.inv(Cb)
    for _ in range(20):
        th = t + rng.standard_normal(k)
        full = (A @ th - b0) @ Vi @ (A @ th - b0)
        assert full == pytest.approx((th - t) @ Ci @ (th - t) + const, rel=1e-10, abs=1e-10)
    assert const >= -1e-12
    # the minimum over theta by a generic minimiser sits at t with value const
    from scipy.optimize import minimize
    f = lambda th: (A @ th - b0) @ Vi @ (A @ th - b0)
    r = minimize(f, np.zeros(k), method="BFGS", options={"gtol": 1e-10})
    np.testing.assert_allclose(r.x, t, atol=1e-6)
    assert r.fun == pytest.approx(const, abs=1e-8)


def test_linear_prior_block_special_cases():
    rng = np.random.default_rng(12)
    V, b0 = _spd(rng, 4), rng.standard_normal(4)
    t, Cb, const = oracle.linear_prior_block(np.eye(4), b0, V)
    np.testing.assert_allclose(t, b0, rtol=1e-12)
    np.testing.assert_allclose(Cb, V, rtol=1e-10)
    assert abs(const) < 1e-10
    # one parameter measured twice with independent errors: inverse-variance mean
    t, Cb, const = oracle.linear_prior_block([[1.0], [1.0]], [1.0, 3.0], np.diag([1.0, 4.0]))
    assert t[0] == pytest.approx((1.0 / 1 + 3.0 / 4) / (1 / 1 + 1 / 4), rel=1e-14)
    assert Cb[0, 0] == pytest.approx(1 / (1 + 1 / 4), rel=1e-14)
    assert const == pytest.approx((1.0 - t[0]) ** 2 + (3.0 - t[0]) ** 2 / 4, rel=1e-12)


# ---------------------------------------------------------------------------------------
# Eq. 6 with a generalised parametrisation, evaluated as written: (A theta - b0)^T V^-1 (A theta - b0)
# ---------------------------------------------------------------------------------------
def _with_maps(spec, maps, free=()):
    """A copy of spec with map priors added; the parameters in `free` lose their individual
    Gaussian priors (a map then constrains them)."""
    s = copy.deepcopy(spec)
    s.prior_sigma = s.prior_sigma.copy()
    for i in free:
        s.prior_sigma[i] = 0.0
    s.map_priors = list(maps)
    return s


def test_map_prior_term_is_the_hand_computed_quadratic_form():
    """Two parameters (a0, a1 of the single-detector model) and three measured combinations
    b = (a0, a1, a0 + a1) with the covariance V = [[4, 2, 0], [2, 4, 0], [0, 0, 1]] (10^-4).
    By hand: V^-1 = 10^4 [[1/3, -1/6, 0], [-1/6, 1/3, 0], [0, 0, 1]], so with residuals
    r = (b - b0) the term is 10^4 (r1^2/3 - r1 r2/3 + r2^2/3 + r3^2); its gradient is
    A^T 2 V^-1 r. The term is isolated as the difference to the model without the map."""
    base = synth.make_model("c0")
    i0, i1 = base.index("a0"), base.index("a1")
    A = np.array([[1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    b0 = np.array([0.003, 1.001, 1.0])
    V = 1e-4 * np.array([[4.0, 2.0, 0.0], [2.0, 4.0, 0.0], [0.0, 0.0, 1.0]])
    ix = np.array([i0, i1], np.int32)
    with_map = oracle.OracleModel(_with_maps(base, [(ix, A, b0, V)], free=ix))
    without = oracle.OracleModel(_with_maps(base, [], free=ix))
    data = synth.poisson_data(without.expected(base.theta0), 21)
    theta = base.theta0.copy()
    theta[i0], theta[i1] = 0.012, 0.995
    r1, r2, r3 = theta[i0] - 0.003, theta[i1] - 1.001, theta[i0] + theta[i1] - 1.0
    hand = 1e4 * (r1 * r1 / 3 - r1 * r2 / 3 + r2 * r2 / 3 + r3 * r3)
    v1, g1 = with_map.nll(theta, data, grad=True)
    v0, g0 = without.nll(theta, data, grad=True)
    assert v1 - v0 == pytest.approx(hand, rel=1e-12)
    # gradient by hand: d/da0 = 1e4 (2 r1/3 - r2/3 + 2 r3), d/da1 = 1e4 (2 r2/3 - r1/3 + 2 r3)
    dg = g1 - g0
    assert dg[i0] == pytest.approx(1e4 * (2 * r1 / 3 - r2 / 3 + 2 * r3), rel=1e-10)
    assert dg[i1] == pytest.approx(1e4 * (2 * r2 / 3 - r1 / 3 + 2 * r3), rel=1e-10)
    others = np.ones(base.n_params, bool)
    others[ix] = False
    assert np.all(dg[others] == 0.0)


def test_map_prior_with_identity_map_is_a_covariance_block():
    """A = I makes Eq. 6's generalised term the plain correlated prior of Eq. 6 on the
    parameters themselves with mean b0: both oracle paths give the same -2lnL and gradient."""
    base = synth.make_model("c0")
    rng = np.random.default_rng(22)
    names = ["a0", "a1", "a2"]
    ix = np.array([base.index(n) for n in names], np.int32)
    sig = np.array([0.01, 0.005, 0.001])
    R = np.array([[1.0, 0.3, -0.2], [0.3, 1.0, 0.1], [-0.2, 0.1, 1.0]])
    V = R * np.outer(sig, sig)
    b0 = base.theta0[ix] + sig * rng.standard_normal(3)
    m = oracle.OracleModel(_with_maps(base, [(ix, np.eye(3), b0, V)], free=ix))
    blk = _with_maps(base, [], free=ix)
    blk.theta0 = blk.theta0.copy()
    blk.theta0[ix] = b0
    blk.cov_blocks = list(blk.cov_blocks) + [(ix, V)]
    b = oracle.OracleModel(blk)
    data = synth.poisson_data(b.expected(base.theta0), 23)
    for _ in range(5):
        th = base.theta0.copy()
        th[ix] += 2 * sig * rng.standard_normal(3)
        v1, g1 = m.nll(th, data, grad=True)
        v2, g2 = b.nll(th, data, grad=True)
        assert v1 == pytest.approx(v2, rel=1e-12)
        np.testing.assert_allclose(g1, g2, rtol=1e-9, atol=1e-9 * np.abs(g2).max())


def test_map_prior_gradient_matches_central_differences():
    """c1 with its nine energy-scale coefficients constrained through a 12-row map: the
    analytic gradient of the whole -2lnL against central differences."""
    base = synth.make_model("c1")
    rng = np.random.default_rng(24)
    esc = [f"a{k}[{d}]" for d in range(3) for k in range(3)]
    ix = np.array([base.index(n) for n in esc], np.int32)
    A = np.vstack([np.eye(9), rng.standard_normal((3, 9))])
    w = np.array([0.01, 0.005, 0.001] * 3 + [0.005] * 3)
    V = _spd(rng, 12)
    V = V / np.sqrt(np.outer(np.diag(V), np.diag(V))) * np.outer(w, w)
    b0 = A @ base.theta0[ix] + 0.5 * w * rng.standard_normal(12)
    spec = _with_maps(base, [(ix, A, b0, V)], free=ix)
    om = oracle.OracleModel(spec)
    data = synth.poisson_data(om.expected(base.theta0), 25)
    theta = om.theta_of_z(0.4 * rng.standard_normal(spec.n_params))
    _, g = om.nll(theta, data, grad=True)
    for i in ix:
        h = 1e-6 * spec.scale[i]
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (om.nll(tp, data) - om.nll(tm, data)) / (2 * h)
        assert abs(fd - g[i]) * spec.scale[i] < 1e-5 * (1 + abs(g[i]) * spec.scale[i])


def test_map_prior_is_rejected_when_not_positive_definite():
    base = synth.make_model("c0")
    ix = np.array([base.index("a0")], np.int32)
    with pytest.raises(ValueError, match="positive"):
        oracle.OracleModel(_with_maps(base, [(ix, np.ones((2, 1)), np.zeros(2),
                                              np.array([[1.0, 2.0], [2.0, 1.0]]))]))
