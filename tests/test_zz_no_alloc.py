"""The allocation-free evaluation entry point (fit_model_eval_noalloc) against fit_model_eval.

fit_model_eval_noalloc serves callers that cannot allocate device memory (an application
with its own fixed device budget, a plugin under another framework's allocator, a loop that
must not enter the allocator). It keeps its workspace in a fixed device array inside the
library, so the test runs it three times in a row on the same array and checks every result
against the allocating entry point. Both launch the same per-instance evaluation (one block
per parameter vector, a fixed reduction order inside the block), so the results must be
identical bit for bit, whatever grid each path uses. The file is collected last so that a
failure here cannot hide the other tests' results.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2502_15253_gb300 import fitcore, synth

pytestmark = pytest.mark.gpu

SCRATCH_FLOATS = 4 << 20        # the library's 16 MiB array


def _ws_floats(spec):
    """Per-block workspace of one evaluation, floats: (4 + 4 survival partials + cores) per
    true bin and two per reco bin of the largest detector."""
    return (8 + spec.n_cores) * spec.n_true + 2 * max(d.n_reco for d in spec.detectors)


def _cudart():
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            return C.CDLL(name)
        except OSError:
            pass
    return C.CDLL("/usr/local/cuda/lib64/libcudart.so")


def _pool_used(rt):
    """(bytes in use, high-water mark) of the current device's default memory pool, the pool
    that cudaMallocAsync draws from."""
    dev = C.c_int()
    assert rt.cudaGetDevice(C.byref(dev)) == 0
    pool = C.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(C.byref(pool), dev) == 0
    used, high = C.c_uint64(), C.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, 7, C.byref(used)) == 0    # UsedMemCurrent
    assert rt.cudaMemPoolGetAttribute(pool, 8, C.byref(high)) == 0    # UsedMemHigh
    return pool, used.value, high.value


@pytest.mark.parametrize("name", ["c2", "c1"])
def test_noalloc_eval_matches_allocating_eval_twice(name):
    """c2 needs 36,800 floats of workspace per block, so the array holds 113 slices, fewer
    than the resident blocks: the grid is capped by the array and 700 vectors run through the
    grid-stride loop. c1 (4,076 floats, 1,029 slices) runs at full occupancy."""
    torch = pytest.importorskip("torch")
    spec = synth.make_model(name)
    gm = fitcore.Model(spec)
    B = 700
    if name == "c2":
        assert SCRATCH_FLOATS // _ws_floats(spec) < 152 < B
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
    torch.cuda.synchronize()

    # The first call on a device resolves the array's address; with lazily loaded modules
    # that is also when the runtime places the library's 16 MiB array on the device. The
    # memory readings therefore bracket the calls after it.
    rt = _cudart()
    for call in range(3):
        nll = torch.full((B,), np.nan, dtype=torch.float64, device=dev)
        g = torch.full((B, spec.n_params), np.nan, dtype=torch.float32, device=dev)
        st = torch.full((B,), -7, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        pool, used0, _ = _pool_used(rt)
        assert rt.cudaMemPoolSetAttribute(pool, 8, C.byref(C.c_uint64(0))) == 0   # reset high
        free0 = torch.cuda.mem_get_info()[0]
        fitcore.fit_model_eval_noalloc(gm, B, th_d, da_d, mk_d, nll, g, st)
        torch.cuda.synchronize()
        _, used1, high1 = _pool_used(rt)
        # nothing drawn from the stream-ordered pool, nothing held in plain allocations
        assert high1 <= used0 and used1 == used0, (call, used0, used1, high1)
        if call > 0:
            assert torch.cuda.mem_get_info()[0] == free0, call
        assert np.array_equal(st.cpu().numpy(), ref_st.cpu().numpy()), call
        assert np.all(np.isfinite(nll.cpu().numpy())), call
        assert np.array_equal(nll.cpu().numpy(), ref_nll.cpu().numpy()), call
        assert np.array_equal(g.cpu().numpy(), ref_g.cpu().numpy()), call


def test_noalloc_rejects_host_buffers():
    spec = synth.make_model("c0")
    gm = fitcore.Model(spec)
    theta = spec.theta0[None].copy()
    nll = np.zeros(1)
    with pytest.raises(fitcore.FitError):
        fitcore.fit_model_eval_noalloc(gm, 1, theta, None, None, nll)
