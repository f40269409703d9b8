"""Event-level reweighting on the device (fit_mc_spectrum) against the oracle's FP64 sum over
the same events.

Bar: every bin within 2e-6 of its unoscillated content W_j = sum of the weights in bin j.
Per event the kernel forms P in FP32: float-pair phases reduced to |r| <= 1/2 half-turns
(error a few 1e-8), a fitted polynomial for sin^2(pi r) (within 1.8e-7), the coefficients
rounded once to FP32 (6e-8 relative) and two or three FMAs (~1.2e-7): |dP| < 4e-7. A warp
sums a chunk of 256 events in FP32 (8 in a lane, then 5 pairwise levels: below 13 x 2^-24 =
8e-7 of the chunk's sum <= its weight); chunks are added as float pairs and in FP64. So
|S_j - S_j(oracle)| < 1.2e-6 W_j. (Relative to S_j itself the bound would be looser where
P is small, down to ~0.1 near the solar minimum at 53 km.)
"""
import numpy as np
import pytest

import oracle
from paper_2502_15253_gb300 import fitcore, synth

pytestmark = pytest.mark.gpu

TOL = 2e-6


def _sets(ev, n, seed):
    """n survival parameter sets scattered around the nominal values (the first is nominal)."""
    rng = np.random.default_rng(seed)
    p0 = np.asarray(ev.osc_nominal, np.float64)
    out = np.tile(p0, (n, 1))
    if n > 1:
        out[1:] *= rng.uniform(0.7, 1.3, (n - 1, 4))
    return out


def _check(ev, params, out):
    W = np.bincount(ev.bin, weights=ev.weight.astype(np.float64), minlength=ev.n_bins)
    for b in range(params.shape[0]):
        ref = oracle.event_spectrum(ev, params[b])
        err = np.abs(out[b] - ref)
        bad = np.flatnonzero(err > TOL * W + 1e-300)
        assert bad.size == 0, (b, bad[:5], out[b][bad[:5]], ref[bad[:5]], W[bad[:5]])


@pytest.mark.parametrize("geometry,n", [("dc_fd", 300_000), ("juno_fd", 400_000)])
def test_spectrum_matches_oracle(geometry, n):
    ev = synth.make_mc_events(n, geometry)
    params = _sets(ev, 6, 1)
    mc = fitcore.McEventSet(ev)
    out = np.zeros((6, ev.n_bins))
    mc.spectrum(6, params, out)
    mc.status()
    _check(ev, params, out)


def test_inverted_ordering_and_device_buffers():
    torch = pytest.importorskip("torch")
    ev = synth.make_mc_events(250_000, "juno_fd")
    p = np.array([[0.307, 0.022, 7.5e-5, 2.5e-3], [0.307, 0.022, 7.5e-5, -2.425e-3]])
    mc = fitcore.McEventSet(ev)
    pd = torch.tensor(p, dtype=torch.float64, device="cuda")
    od = torch.full((2, ev.n_bins), 7.0, dtype=torch.float64, device="cuda")   # cleared by the call
    mc.spectrum(2, pd, od)
    torch.cuda.synchronize()
    out = od.cpu().numpy()
    _check(ev, p, out)
    assert np.abs(out[0] - out[1]).max() > 1e-3 * out[0].max()   # the orderings differ


@pytest.mark.parametrize("geometry", ["dc_fd", "juno_fd"])
def test_zero_mixing_gives_weighted_counts(geometry):
    ev = synth.make_mc_events(123_457, geometry)
    p = (np.array([[0.0, 2.5e-3, 0.0, 7.5e-5]]) if ev.osc_mode == 0
         else np.array([[0.0, 0.0, 7.5e-5, 2.5e-3]]))
    mc = fitcore.McEventSet(ev)
    out = np.zeros((1, ev.n_bins))
    mc.spectrum(1, p, out)
    ref = np.bincount(ev.bin, weights=ev.weight.astype(np.float64), minlength=ev.n_bins)
    np.testing.assert_allclose(out[0], ref, rtol=1e-6)


@pytest.mark.parametrize("n", [0, 1, 31, 255, 256, 257, 8 * 32 * 3 + 5])
def test_ragged_event_counts(n):
    ev = synth.make_mc_events(max(n, 1) * 3 + 50, "dc_fd")
    keep = np.sort(np.random.default_rng(n).choice(len(ev.energy), size=n, replace=False))
    for f in ("energy", "core", "weight", "bin"):
        setattr(ev, f, getattr(ev, f)[keep])
    params = _sets(ev, 3, n)
    mc = fitcore.McEventSet(ev)
    out = np.full((3, ev.n_bins), -1.0)
    mc.spectrum(3, params, out)
    if n == 0:
        assert np.all(out == 0.0)
    else:
        _check(ev, params, out)


def test_single_bin_and_boundary_runs():
    """All events in one bin (every chunk adds to the same total), then bins changing inside
    every lane's run (a bin boundary every 3 events)."""
    ev = synth.make_mc_events(40_000, "dc_fd")
    ev.bin = np.zeros_like(ev.bin)
    ev.n_bins = 1
    mc = fitcore.McEventSet(ev)
    p = _sets(ev, 2, 3)
    out = np.zeros((2, 1))
    mc.spectrum(2, p, out)
    _check(ev, p, out)
    ev.bin = (np.arange(len(ev.energy)) // 3).astype(np.int32)
    ev.n_bins = int(ev.bin[-1]) + 1
    mc2 = fitcore.McEventSet(ev)
    out = np.zeros((2, ev.n_bins))
    mc2.spectrum(2, p, out)
    _check(ev, p, out)


def test_max_sets_and_limits():
    ev = synth.make_mc_events(60_000, "juno_fd")
    mc = fitcore.McEventSet(ev)
    params = _sets(ev, 64, 9)
    out = np.zeros((64, ev.n_bins))
    mc.spectrum(64, params, out)
    _check(ev, params[::9], out[::9])
    with pytest.raises(fitcore.FitError):
        mc.spectrum(65, np.tile(params[:1], (65, 1)), np.zeros((65, ev.n_bins)))


def test_full_size_sampled_bins():
    """The bench workload (8M events of the two-core far detector, 16 sets) against the oracle
    on every bin of three sets."""
    ev = synth.make_mc_events(8_000_000, "dc_fd")
    params = _sets(ev, 16, 4)
    mc = fitcore.McEventSet(ev)
    out = np.zeros((16, ev.n_bins))
    mc.spectrum(16, params, out)
    _check(ev, params[[0, 7, 15]], out[[0, 7, 15]])
