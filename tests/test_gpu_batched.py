"""Batched expectation with the response fold on tensor cores (fit_model_expected_tc) against
the FP64 oracle.

Tolerances:
  * precision 1 (split 3xTF32): relative 2e-5 per bin, the bar of the CUDA-core expectation.
    Each operand is split x = x_hi + x_lo with x_hi exact in TF32 (|x_lo| <= 2^-11 |x|); the
    three products keep everything but x_lo y_lo (<= 2^-22 relative) and the hardware's
    reading of x_lo (10 mantissa bits, <= 2^-21 relative); the true spectrum itself carries the
    FP32 errors of the CUDA-core path.
  * precision 0 (plain TF32): every operand rounded to nearest with 10 mantissa bits, so each
    product is within 2^-10 relative and a bin (a sum of positive products) within 1.5e-3.
"""
import numpy as np
import pytest

import oracle
from paper_2502_15253_gb300 import fitcore, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["c0", "c1", "c2", "c1s", "c0/spline", "c1/spline", "c2/spline"])
def pair(request):
    spec = synth.make_model(request.param.split("/")[0], remap=int(request.param.endswith("spline")))
    return spec, oracle.OracleModel(spec), fitcore.Model(spec)


def _thetas(spec, om, n, amp, seed):
    rng = np.random.default_rng(seed)
    return np.stack([om.theta_of_z(amp * rng.standard_normal(spec.n_params)) for _ in range(n)])


def _expected_tc(gm, th, precision):
    th = np.ascontiguousarray(th, np.float64)
    mu = np.zeros((len(th), gm.n_data), np.float32)
    st = np.zeros(len(th), np.int32)
    fitcore.fit_model_expected_tc(gm, len(th), th, mu, st, precision)
    return mu, st


@pytest.mark.parametrize("B", [1, 5, 130])
def test_split_tf32_matches_oracle(pair, B):
    spec, om, gm = pair
    th = _thetas(spec, om, B, 0.8, 10 + B)
    mu, st = _expected_tc(gm, th, 1)
    assert np.all(st == 0)
    idx = range(B) if B <= 8 else [0, 1, 63, 64, 127, 128, 129]
    for b in idx:
        ref = om.expected(th[b])
        np.testing.assert_allclose(mu[b], ref, rtol=2e-5, atol=1e-6 * ref.max())


def test_plain_tf32_within_its_bound(pair):
    spec, om, gm = pair
    th = _thetas(spec, om, 4, 0.8, 21)
    mu, st = _expected_tc(gm, th, 0)
    assert np.all(st == 0)
    for b in range(len(th)):
        ref = om.expected(th[b])
        np.testing.assert_allclose(mu[b], ref, rtol=1.5e-3, atol=1e-5 * ref.max())


def test_agrees_with_cuda_core_path_on_device(pair):
    torch = pytest.importorskip("torch")
    spec, om, gm = pair
    th = torch.tensor(_thetas(spec, om, 257, 1.0, 31), dtype=torch.float64, device="cuda")
    mu_tc = torch.zeros((257, gm.n_data), dtype=torch.float32, device="cuda")
    mu_cc = torch.zeros_like(mu_tc)
    st_tc = torch.zeros(257, dtype=torch.int32, device="cuda")
    st_cc = torch.zeros_like(st_tc)
    fitcore.fit_model_expected_tc(gm, 257, th, mu_tc, st_tc, 1)
    fitcore.fit_model_expected(gm, 257, th, mu_cc, st_cc)
    torch.cuda.synchronize()
    assert torch.equal(st_tc, st_cc)
    rel = ((mu_tc - mu_cc).abs() / mu_cc.abs().clamp_min(1e-3 * float(mu_cc.max()))).max()
    assert float(rel) < 2e-5


def test_invalid_energy_map_flags_instance(pair):
    spec, om, gm = pair
    ds = spec.datasets[0]
    a1 = int(ds.escale_idx[1])
    if a1 < 0:
        pytest.skip("energy scale fixed in this model")
    th = np.tile(spec.theta0, (3, 1))
    th[1, a1] = 5.0                 # slope far outside (1/4, 4)
    mu, st = _expected_tc(gm, th, 1)
    _, st_cc = fitcore.expected_numpy(gm, th)
    assert st[0] == 0 and st[2] == 0
    assert st[1] == 5 and st_cc[1] == 5
    assert np.all(np.isnan(mu[1])) and np.all(np.isfinite(mu[0]))


def test_zero_batch_is_a_no_op(pair):
    _, _, gm = pair
    fitcore.fit_model_expected_tc(gm, 0, np.zeros((1, gm.n_params)), np.zeros((1, gm.n_data),
                                  np.float32), None, 1)
