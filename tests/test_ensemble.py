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


def _sharded_worker(rank, world, port, out_dir, ck):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank))
    import torch.distributed as dist
    from paper_2502_15253_gb300.ensemble import fit_ensemble_sharded
    dist.init_process_group("gloo", rank=rank, world_size=world)
    models, inst, data = _job()
    log = []
    best, res = fit_ensemble_sharded(models, inst, data, chunk=5, checkpoint=ck, fit_fn=_fake(log))
    np.save(os.path.join(out_dir, f"best{rank}.npy"), best)
    np.save(os.path.join(out_dir, f"res{rank}.npy"), res.view(np.uint8))
    np.save(os.path.join(out_dir, f"log{rank}.npy"), np.array(log))
    dist.destroy_process_group()


def test_sharded_ensemble_over_two_gloo_ranks(tmp_path):
    """Two ranks split the 37 instances (19 + 18), fit them with no collective, gather on the
    host, and both return the single-process result; each kept its own checkpoint."""
    torch = pytest.importorskip("torch")
    import socket
    import torch.multiprocessing as mp
    if torch.cuda.is_available():
        pytest.skip("the host-only (gloo) path is exercised where no GPU is visible")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ck = str(tmp_path / "ens.npz")
    mp.spawn(_sharded_worker, args=(2, port, str(tmp_path), ck), nprocs=2, join=True)
    models, inst, data = _job()
    ref_best, ref_res = fit_ensemble(models, inst, data, chunk=5, fit_fn=_fake([]))
    for r in range(2):
        np.testing.assert_array_equal(np.load(tmp_path / f"best{r}.npy"), ref_best)
        got = np.load(tmp_path / f"res{r}.npy").view(fitcore.RESULT_DTYPE)
        np.testing.assert_array_equal(got, ref_res)
        assert os.path.exists(ck + f".rank{r}")
    assert list(np.load(tmp_path / "log0.npy")) == [5, 5, 5, 4]
    assert list(np.load(tmp_path / "log1.npy")) == [5, 5, 5, 3]
