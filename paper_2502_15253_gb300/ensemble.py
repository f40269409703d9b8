"""Checkpointed ensemble fits and their JSON output.

Ensemble studies and parameter scans run many fits with individual settings and start
values ([S], "Structure of the framework": parallel fits; its output component writes each
converged fit as JSON). `fit_ensemble` runs the instances through the library's fit_batch in
chunks and, after every chunk, replaces one .npz checkpoint atomically; a run that stopped
(a crash, a killed job, a lost GPU) resumes from that file and fits only the instances not yet
done. This module is host orchestration only: every fit runs in the library's kernels.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np

from . import fitcore

_FORMAT = 1


def _fingerprint(models, inst, data, start, fixed) -> str:
    """Identity of a job: the instance table, the data, the start values, the held mask and the
    models' sizes. A checkpoint of another job is refused."""
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(inst).tobytes())
    for a in (data, start, fixed):
        if a is None:
            h.update(b"-")
        else:
            a = np.ascontiguousarray(a)
            h.update(str((a.dtype.str, a.shape)).encode())
            h.update(a.tobytes())
    h.update(str([(int(m.n_params), int(m.n_data)) for m in models]).encode())
    return h.hexdigest()


def _save(path, fp, done, best, res):
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        np.savez(f, format=np.int64(_FORMAT), fingerprint=np.array(fp), done=done, best=best,
                 results=res.view(np.uint8))
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def _load(path, fp, n, npar):
    with np.load(path, allow_pickle=False) as z:
        if int(z["format"]) != _FORMAT or str(z["fingerprint"]) != fp:
            raise ValueError(f"checkpoint {path} belongs to another job")
        done, best = z["done"].copy(), z["best"].copy()
        res = z["results"].copy().view(fitcore.RESULT_DTYPE)
    if done.shape != (n,) or best.shape != (npar,) or res.shape != (n,):
        raise ValueError(f"checkpoint {path} has the wrong sizes")
    return done, best, res


def fit_ensemble(models, inst, data, start=None, opts=None, fixed=None, chunk=4096,
                 checkpoint=None, fit_fn=None):
    """Fits every instance of `inst` (fitcore.INSTANCE_DTYPE) in chunks of `chunk` instances.

    data / start / fixed are laid out as for fit_batch (offsets in `inst`). With `checkpoint`
    (a file path) the finished chunks are saved after each fit_batch call, and a call that finds
    the file of the same job fits only the instances it does not list as done. Returns
    (best [flat float64, param_off layout], results [n] RESULT_DTYPE). `fit_fn(models,
    sub_inst, data, start, opts, fixed) -> (best_flat, results)` replaces fitcore.fit_numpy
    (used by tests to stop a run part-way).
    """
    inst = np.ascontiguousarray(inst, dtype=fitcore.INSTANCE_DTYPE)
    n = len(inst)
    if chunk < 1:
        raise ValueError("chunk must be >= 1")
    npar = max((int(r["param_off"]) + models[int(r["model"])].n_params for r in inst), default=0)
    fit_fn = fit_fn or (lambda m, i, d, s, o, f: fitcore.fit_numpy(m, i, d, s, o, fixed=f))
    fp = _fingerprint(models, inst, data, start, fixed)
    if checkpoint and os.path.exists(checkpoint):
        done, best, res = _load(checkpoint, fp, n, npar)
    else:
        done = np.zeros(n, bool)
        best = np.zeros(npar)
        res = np.zeros(n, fitcore.RESULT_DTYPE)
    todo = np.flatnonzero(~done)
    for a in range(0, len(todo), chunk):
        idx = todo[a:a + chunk]
        b, r = fit_fn(models, inst[idx], data, start, opts, fixed)
        for i in idx:
            o = int(inst[i]["param_off"])
            P = models[int(inst[i]["model"])].n_params
            best[o:o + P] = b[o:o + P]
        res[idx] = r
        done[idx] = True
        if checkpoint:
            _save(checkpoint, fp, done, best, res)
    return best, res


def write_results_json(path, models, inst, best, results):
    """One JSON line per instance (the library's fit_result_json record, which names the
    parameters of models created from a configuration), written atomically."""
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        for i, r in enumerate(np.asarray(results)):
            m = models[int(inst[i]["model"])]
            o = int(inst[i]["param_off"])
            f.write(fitcore.fit_result_json(m, best[o:o + m.n_params], r) + "\n")
    os.replace(tmp, path)


def shard(n_total, rank, world):
    """Contiguous share [lo, hi) of n_total instances for a rank; the first n_total % world
    ranks take one more."""
    base, rem = divmod(n_total, world)
    lo = rank * base + min(rank, rem)
    return lo, lo + base + (1 if rank < rem else 0)


def fit_ensemble_sharded(models, inst, data, start=None, opts=None, fixed=None, chunk=4096,
                         checkpoint=None, fit_fn=None, group=None):
    """fit_ensemble over the ranks of a torch.distributed process group, one GPU per rank.

    Pseudo-experiments are independent ([S]: parallel fits, with MPI across processes), so
    each rank fits a contiguous share of `inst` (its own checkpoint file `<checkpoint>.rank<r>`)
    and the results meet on the host in one all_gather of Python objects at the end: no
    collective runs during the fits. Every rank returns the whole (best, results)."""
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
    rank = dist.get_rank(group) if world > 1 else 0
    inst = np.ascontiguousarray(inst, dtype=fitcore.INSTANCE_DTYPE)
    if world == 1:
        return fit_ensemble(models, inst, data, start, opts, fixed, chunk, checkpoint, fit_fn)
    lo, hi = shard(len(inst), rank, world)
    ck = f"{checkpoint}.rank{rank}" if checkpoint else None
    b, r = fit_ensemble(models, inst[lo:hi], data, start, opts, fixed, chunk, ck, fit_fn)
    sl = [b[int(q["param_off"]):int(q["param_off"]) + models[int(q["model"])].n_params]
          for q in inst[lo:hi]]
    parts = [None] * world
    dist.all_gather_object(parts, (lo, hi, sl, r.tobytes()), group=group)
    npar = max((int(q["param_off"]) + models[int(q["model"])].n_params for q in inst), default=0)
    best = np.zeros(npar)
    res = np.zeros(len(inst), fitcore.RESULT_DTYPE)
    for plo, phi, psl, pres in parts:
        res[plo:phi] = np.frombuffer(pres, dtype=fitcore.RESULT_DTYPE)
        for i, v in zip(range(plo, phi), psl):
            o = int(inst[i]["param_off"])
            best[o:o + len(v)] = v
    return best, res
