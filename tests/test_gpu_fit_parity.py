"""GPU batched L-BFGS fits against the FP64 oracle's BFGS fits on the same pseudo-data.

Bar per instance:
  * |nll_min - nll_min_oracle| <= 1e-3 (the tolerance on -2lnL at the minimum), and
  * every best-fit parameter within 1e-3 of its oracle sigma (the strict bar).
sigma = sqrt(2 (H^-1)_ii) at the oracle minimum, H from central differences of the analytic
gradient. Parameters without curvature (no data, no prior under the dataset mask) have
sigma = inf and only need a finite value.

The strict bar holds for every instance of every test (min_strict = 1, no other minimum)
except on the three-dataset model with the overlap-length energy correction. There the
correction is only continuous in (a0, a1, a2): the gradient jumps where a mapped bin edge
crosses a grid edge, and the FP32 evaluation places each such crease within ~1e-7 of a bin
of where the FP64 oracle places it. Along the nearly flat directions that cross the creases
(the Li-9 rates against the common mode of their 38 shape parameters) this moves the minimum
of the FP32 likelihood by more than 1e-3 sigma in some instances, while the same fits on the
C1-continuous spline correction meet the strict bar in all instances. For those tests the
strict bar is asserted for the measured share and 1e-2 sigma for all.

Several minima: the creases can also hold separate local minima. Where the GPU result is not
the oracle's minimum (|dnll| > 1e-3 or a parameter beyond 1e-2 sigma), the test requires it
to be a minimum of the FP64 likelihood: the oracle restarted there stays within 1e-2 sigma and
1e-4 in -2lnL; tests that allow this say how many instances may.
"""
import numpy as np
import pytest

import oracle
from paper_2502_15253_gb300 import fitcore, synth

pytestmark = pytest.mark.gpu

SPECS = {}


def spec_of(name):
    """"c1" etc.; "c1/spline" is the same model with the area-conserving spline remap."""
    if name not in SPECS:
        s = synth.make_model(name.split("/")[0], remap=int(name.endswith("/spline")))
        SPECS[name] = (s, oracle.OracleModel(s), fitcore.Model(s))
    return SPECS[name]


def make_instances(name, n, seed, masks=None):
    spec, om, _ = spec_of(name)
    rng = np.random.default_rng(seed)
    datas, ms, truths = [], [], []
    for i in range(n):
        th = synth.draw_theta_true(spec, rng)
        datas.append(synth.poisson_data(om.expected(th), int(rng.integers(1 << 31))))
        ms.append(spec.all_mask() if masks is None else masks[i % len(masks)])
        truths.append(th)
    return datas, ms, truths


def engine_opts(engine):
    o = fitcore.fit_batch_default_opts()
    o.engine = engine
    return o


ENGINES = pytest.mark.parametrize("engine", [0, 1, 2], ids=["persistent", "lockstep", "lockstep_tc"])


def run_gpu(names_per_inst, datas, masks, starts=None, opts=None):
    names = sorted(set(names_per_inst))
    models = [spec_of(n)[2] for n in names]
    inst = np.zeros(len(datas), fitcore.INSTANCE_DTYPE)
    doff = poff = 0
    for i, (n, d) in enumerate(zip(names_per_inst, datas)):
        inst[i] = (names.index(n), masks[i], doff, poff)
        doff += len(d)
        poff += spec_of(n)[0].n_params
    flat_start = None if starts is None else np.concatenate(starts)
    best, res = fitcore.fit_numpy(models, inst, np.concatenate(datas), flat_start, opts)
    thetas = [best[int(r["param_off"]):int(r["param_off"]) + spec_of(n)[0].n_params]
              for r, n in zip(inst, names_per_inst)]
    return thetas, res


def check_against_oracle(name, datas, masks, thetas, res, max_other=0, min_strict=1.0):
    spec, om, _ = spec_of(name)
    n_other = n_strict = 0
    for i, (d, m) in enumerate(zip(datas, masks)):
        ref = om.fit(d, mask=m)
        assert ref["status"] == 0
        assert res[i]["status"] == 0, (i, fitcore.STATUS[int(res[i]["status"])], res[i])
        assert np.all(np.isfinite(thetas[i]))
        sig = om.sigma(ref["theta"], d, mask=m)
        fin = np.isfinite(sig)
        dev = np.abs(thetas[i][fin] - ref["theta"][fin]) / sig[fin]
        dnll = abs(res[i]["nll_min"] - ref["nll"])
        n_strict += int(dev.max() <= 1e-3 and dnll <= 1e-3)
        if dnll <= 1e-3 and dev.max() <= 1e-2:
            continue
        # another minimum: certify it with the oracle restarted at the GPU point
        cert = om.fit(d, mask=m, start=thetas[i])
        assert cert["status"] == 0
        assert abs(cert["nll"] - om.nll(thetas[i], d, mask=m)) <= 1e-4, (i, cert["nll"])
        assert abs(res[i]["nll_min"] - cert["nll"]) <= 1e-3, (i, res[i]["nll_min"], cert["nll"])
        dev2 = np.abs(thetas[i][fin] - cert["theta"][fin]) / sig[fin]
        assert dev2.max() <= 1e-2, (i, spec.param_names[np.flatnonzero(fin)[dev2.argmax()]], dev2.max())
        n_other += 1
    assert n_other <= max_other, (n_other, len(datas))
    assert n_strict >= min_strict * len(datas), (n_strict, len(datas))
    print(f"{name}: {n_strict}/{len(datas)} instances meet the strict 1e-3 sigma bar, "
          f"{n_other} stopped in another certified minimum")
    return n_other, n_strict


@ENGINES
def test_fit_c0_matches_oracle(engine):
    datas, masks, _ = make_instances("c0", 12, 100)
    th, res = run_gpu(["c0"] * 12, datas, masks, opts=engine_opts(engine))
    check_against_oracle("c0", datas, masks, th, res)


@ENGINES
def test_fit_c1_with_dataset_masks_matches_oracle(engine):
    datas, masks, _ = make_instances("c1", 6, 200, masks=list(synth.C1_MASKS))
    th, res = run_gpu(["c1"] * 6, datas, masks, opts=engine_opts(engine))
    # overlap-rule creases on the three-dataset model (module docstring)
    check_against_oracle("c1", datas, masks, th, res, max_other=1, min_strict=0.5)


@ENGINES
def test_fit_c2_matches_oracle(engine):
    datas, masks, _ = make_instances("c2", 2, 300)
    th, res = run_gpu(["c2"] * 2, datas, masks, opts=engine_opts(engine))
    check_against_oracle("c2", datas, masks, th, res)


@ENGINES
def test_fit_c1_ensemble_statistics(engine):
    """64 pseudo-experiments of the three-dataset model: at most 1 in 8 may stop in another
    (certified) minimum; all others match the oracle's minimum within 1e-3 in -2lnL and
    1e-2 sigma in every parameter, and at least 85 % within 1e-3 sigma (60/64 measured with
    the 32-pair history; the share moves with FP32 rounding in the flat Li-9 direction and was
    64-75 % with 16 pairs)."""
    datas, masks, _ = make_instances("c1", 64, 600)
    th, res = run_gpu(["c1"] * 64, datas, masks, opts=engine_opts(engine))
    check_against_oracle("c1", datas, masks, th, res, max_other=8, min_strict=0.85)


@ENGINES
def test_fit_c1_spline_ensemble(engine):
    """The three-dataset model with the area-conserving spline energy correction: -2lnL
    continuously differentiable in (a0, a1, a2), so no crease can hold a second minimum. 32
    pseudo-experiments; all must reach the oracle's minimum within 1e-3 in -2lnL and 1e-3
    sigma in every parameter."""
    datas, masks, _ = make_instances("c1/spline", 32, 700)
    th, res = run_gpu(["c1/spline"] * 32, datas, masks, opts=engine_opts(engine))
    check_against_oracle("c1/spline", datas, masks, th, res)


@ENGINES
def test_fit_c0_and_c2_spline_match_oracle(engine):
    for name, n, seed in (("c0/spline", 8, 710), ("c2/spline", 2, 720)):
        datas, masks, _ = make_instances(name, n, seed)
        th, res = run_gpu([name] * n, datas, masks, opts=engine_opts(engine))
        check_against_oracle(name, datas, masks, th, res)


def test_plain_coordinates_match_oracle():
    """Fits without the Fisher preconditioner (plain whitened coordinates, the lockstep
    engine's and the option precondition = 0) on the three-dataset and the 53 km model."""
    o = fitcore.fit_batch_default_opts()
    o.precondition = 0
    datas, masks, _ = make_instances("c1", 16, 740, masks=list(synth.C1_MASKS))
    th, res = run_gpu(["c1"] * 16, datas, masks, opts=o)
    check_against_oracle("c1", datas, masks, th, res, max_other=2, min_strict=0.5)
    datas, masks, _ = make_instances("c2", 2, 750)
    th, res = run_gpu(["c2"] * 2, datas, masks, opts=o)
    check_against_oracle("c2", datas, masks, th, res)


def test_preconditioned_and_plain_fits_agree_on_smooth_models():
    """On a model without kinks (spline correction) both coordinate systems reach the same
    minimum of every pseudo-experiment; the preconditioned one in fewer iterations."""
    datas, masks, _ = make_instances("c1/spline", 64, 760)
    o0 = fitcore.fit_batch_default_opts()
    o0.precondition = 0
    th0, r0 = run_gpu(["c1/spline"] * 64, datas, masks, opts=o0)
    th1, r1 = run_gpu(["c1/spline"] * 64, datas, masks)
    assert np.all(r0["status"] == 0) and np.all(r1["status"] == 0)
    assert np.max(np.abs(r0["nll_min"] - r1["nll_min"])) <= 1e-3
    assert r1["iters"].mean() < 0.6 * r0["iters"].mean()


def test_fit_c1_on_the_41_bin_flux_grid():
    """Signal shape parameters on the uniform 41-bin flux grid (3 x 41, eight per dataset
    without data: prior only) instead of the reco binning."""
    datas, masks, _ = make_instances("c1_flux41", 8, 730)
    th, res = run_gpu(["c1_flux41"] * 8, datas, masks)
    check_against_oracle("c1_flux41", datas, masks, th, res, max_other=1, min_strict=0.5)


@ENGINES
def test_uneven_mixed_batch_equals_separate_runs(engine):
    d1, m1, _ = make_instances("c1", 5, 400, masks=list(synth.C1_MASKS))
    d2, m2, _ = make_instances("c2", 2, 401)
    names = ["c1", "c2", "c1", "c1", "c2", "c1", "c1"]
    datas = [d1[0], d2[0], d1[1], d1[2], d2[1], d1[3], d1[4]]
    masks = [m1[0], m2[0], m1[1], m1[2], m2[1], m1[3], m1[4]]
    o = engine_opts(engine)
    th, res = run_gpu(names, datas, masks, opts=o)
    th1, r1 = run_gpu(["c1"] * 5, d1, m1, opts=o)
    th2, r2 = run_gpu(["c2"] * 2, d2, m2, opts=o)
    sep = {0: (th1[0], r1[0]), 1: (th2[0], r2[0]), 2: (th1[1], r1[1]), 3: (th1[2], r1[2]),
           4: (th2[1], r2[1]), 5: (th1[3], r1[3]), 6: (th1[4], r1[4])}
    for i in range(len(names)):
        assert res[i]["status"] == 0
        assert abs(res[i]["nll_min"] - sep[i][1]["nll_min"]) <= 1e-4
        assert res[i]["iters"] > 0


def test_asimov_fit_recovers_truth_and_zero_nll():
    spec, om, gm = spec_of("c1")
    truth = spec.theta0.copy()
    free = [i for i in range(spec.n_params) if spec.prior_sigma[i] == 0
            and not any(i in idx for idx, _ in spec.cov_blocks)]
    truth[free] += 1.0 * spec.scale[free]
    data = om.expected(truth)
    th, res = run_gpu(["c1"], [data], [spec.all_mask()])
    assert res[0]["status"] == 0
    assert abs(res[0]["nll_min"]) < 1e-3
    sig = om.sigma(truth, data)
    assert np.max(np.abs(th[0] - truth) / sig) < 1e-2


@ENGINES
def test_start_points_iteration_limit_and_empty_batch(engine):
    spec, om, gm = spec_of("c0")
    datas, masks, truths = make_instances("c0", 3, 500)
    o = engine_opts(engine)
    o.max_iter = 0
    th, res = run_gpu(["c0"] * 3, datas, masks, starts=truths, opts=o)
    # the start passes through the FP32 fit coordinates (whitened, and Fisher-preconditioned
    # by default): it comes back within 1e-6 of each parameter's scale
    scale = np.where(spec.prior_sigma > 0, spec.prior_sigma, spec.scale)
    for i in range(3):
        assert res[i]["status"] == 1 and res[i]["iters"] == 0
        assert np.all(np.abs(th[i] - truths[i]) <= 1e-6 * (scale + np.abs(truths[i]))), i
        assert abs(res[i]["nll_min"] - om.nll(truths[i], datas[i])) <= 1e-3
    empty = np.zeros(0, fitcore.INSTANCE_DTYPE)
    fitcore.fit_batch([gm], empty, np.zeros(1, np.float32), None, np.zeros(1),
                      np.zeros(1, fitcore.RESULT_DTYPE), o)


@ENGINES
def test_clock_budget_ends_every_fit_with_timeout(engine):
    """A clock budget far below one evaluation (1 ns) ends every fit with FIT_STATUS_TIMEOUT:
    the device limit gives up and returns (no wait is left open), each fit reports its start
    point, and the next call on the same models runs normally."""
    spec, om, _ = spec_of("c1")
    datas, masks, _ = make_instances("c1", 40, 810, masks=list(synth.C1_MASKS))
    o = engine_opts(engine)
    o.time_budget_s = 1e-9
    th, res = run_gpu(["c1"] * 40, datas, masks, opts=o)
    assert np.all(res["status"] == 6), np.unique(res["status"])   # FIT_STATUS_TIMEOUT
    assert res["iters"].max() <= 1
    scale = np.where(spec.prior_sigma > 0, spec.prior_sigma, spec.scale)
    for t in th:
        assert np.all(np.isfinite(t))
        assert np.all(np.abs(t - spec.theta0) <= 1e-5 * (scale + np.abs(spec.theta0)))
    th2, res2 = run_gpu(["c1"] * 4, datas[:4], masks[:4], opts=engine_opts(engine))
    assert np.all(res2["status"] == 0)
