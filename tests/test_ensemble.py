"""Checkpoint / resume of ensemble fits (host orchestration; the fit itself is replaced by a
deterministic stand-in, so this runs on the CPU). A run stopped part-way resumes from its
checkpoint, fits only what was not done, and ends with the results of an uninterrupted run."""
import os
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2502_15253_gb300 import fitcore
from paper_2502_15253_gb300.ensemble import fit_ensemble


class Stop(RuntimeError):
    pass


def _job(n=37):
    models = [SimpleNamespace(n_params=5, n_data=7), SimpleNamespace(n_params=3, n_data=4)]
    inst = np.zeros(n, fitcore.INSTANCE_DTYPE)
    inst["model"] = np.arange(n) % 2
    sizes = np.array([models[m].n_params for m in inst["model"]])
    inst["param_off"] = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    inst["data_off"] = np.arange(n) * 7
    data = np.random.default_rng(0).poisson(5.0, 7 * n).astype(np.float32)
    return models, inst, data


def _fake(log, stop_after=None):
    """Writes best[param_off + p] = 1000 i + p + data[data_off] and nll = i + 0.5 for each fitted
    instance i (identified by data_off); raises after `stop_after` calls."""
    def fit(models, sub, data, start, opts, fixed):
        if stop_after is not None and len(log) >= stop_after:
            raise Stop()
        log.append(len(sub))
        npar = max(int(r["param_off"]) + models[int(r["model"])].n_params for r in sub)
        best = np.full(npar, np.nan)
        res = np.zeros(len(sub), fitcore.RESULT_DTYPE)
        for q, r in enumerate(sub):
            i = int(r["data_off"]) // 7
            o, P = int(r["param_off"]), models[int(r["model"])].n_params
            best[o:o + P] = 1000 * i + np.arange(P) + data[int(r["data_off"])]
            res[q]["nll_min"], res[q]["iters"] = i + 0.5, i
        return best, res
    return fit


def test_resume_after_a_stop_matches_an_uninterrupted_run(tmp_path):
    models, inst, data = _job()
    ref_best, ref_res = fit_ensemble(models, inst, data, chunk=8, fit_fn=_fake([]))
    assert np.all(np.isfinite(ref_best))
    np.testing.assert_array_equal(ref_res["iters"], np.arange(len(inst)))
    ck = str(tmp_path / "ens.npz")
    log = []
    with pytest.raises(Stop):
        fit_ensemble(models, inst, data, chunk=8, checkpoint=ck, fit_fn=_fake(log, stop_after=3))
    assert log == [8, 8, 8] and os.path.exists(ck) and not os.path.exists(ck + ".tmp")
    log2 = []
    best, res = fit_ensemble(models, inst, data, chunk=8, checkpoint=ck, fit_fn=_fake(log2))
    assert log2 == [8, 5]   # only the 13 instances not done
    np.testing.assert_array_equal(best, ref_best)
    np.testing.assert_array_equal(res, ref_res)
    # a finished job is not fitted again
    log3 = []
    best, res = fit_ensemble(models, inst, data, chunk=8, checkpoint=ck, fit_fn=_fake(log3))
    assert log3 == []
    np.testing.assert_array_equal(best, ref_best)


def test_checkpoint_of_another_job_is_refused(tmp_path):
    models, inst, data = _job()
    ck = str(tmp_path / "ens.npz")
    fit_ensemble(models, inst, data, chunk=16, checkpoint=ck, fit_fn=_fake([]))
    other = data.copy()
    other[3] += 1
    with pytest.raises(ValueError, match="another job"):
        fit_ensemble(models, inst, other, chunk=16, checkpoint=ck, fit_fn=_fake([]))
    with pytest.raises(ValueError, match="another job"):
        fit_ensemble(models, inst, data, start=np.zeros(200), chunk=16, checkpoint=ck,
                     fit_fn=_fake([]))


def test_chunk_size_does_not_change_results():
    models, inst, data = _job(20)
    a = fit_ensemble(models, inst, data, chunk=1, fit_fn=_fake([]))
    b = fit_ensemble(models, inst, data, chunk=64, fit_fn=_fake([]))
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    with pytest.raises(ValueError):
        fit_ensemble(models, inst, data, chunk=0, fit_fn=_fake([]))


def test_network_weights_round_trip_on_disk(tmp_path):
    from paper_2502_15253_gb300 import warmstart
    rng = np.random.default_rng(3)
    dims = (10, 8, 2, 3)
    shapes = [(8, 10), (8, 8), (3, 8)]
    layers = [(rng.standard_normal(s).astype(np.float32), rng.standard_normal(s[0]).astype(np.float32))
              for s in shapes]
    p = str(tmp_path / "net.npz")
    warmstart.save_layers(p, dims, layers)
    d2, l2 = warmstart.load_layers(p)
    assert tuple(d2) == dims
    for (w, b), (w2, b2) in zip(layers, l2):
        np.testing.assert_array_equal(w, w2)
        np.testing.assert_array_equal(b, b2)
    with pytest.raises(ValueError):
        warmstart.save_layers(p, dims, layers[:2])
    with pytest.raises(ValueError):
        warmstart.save_layers(p, (10, 8, 2, 4), layers)
