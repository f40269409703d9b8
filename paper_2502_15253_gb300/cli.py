"""Command-line driver: configuration in, fits on the GPU, JSON records out.

The three steps follow the framework's structure ([S]): a configuration file names the model,
the library fits every pseudo-experiment, and each best fit is written as a JSON record.

  python -m paper_2502_15253_gb300.cli config --model c1 [--spline] > c1.json
  python -m paper_2502_15253_gb300.cli pseudo --config c1.json --n 64 --seed 1 --out data.npy
  python -m paper_2502_15253_gb300.cli fit --config c1.json --data data.npy --out fits.jsonl \\
      [--mask 7] [--chunk 4096] [--checkpoint fits.npz] [--no-precondition]
  python -m paper_2502_15253_gb300.cli scan --config c1.json --data data.npy --row 0 \
      --param sin2_2th13 --lo 0 --hi 0.2 --points 41 [--out scan.json]

`config` writes the JSON configuration of a synthetic model. `pseudo` draws Poisson
pseudo-data at the nominal point on the device (fit_model_expected, fit_poisson_sample).
`fit` fits each row of a [n, n_data] float32 .npy file from the nominal point and writes one
fit_result_json line per row; with --checkpoint an interrupted run resumes. Under torchrun the
rows are split over the ranks (one GPU each) and rank 0 writes the records. `scan` profiles
-2lnL in one named parameter (Eq. 7) and reports its Wilks intervals (68.27 %, 95 %) and the
goodness of fit of the best fit (Eq. 8). This module only
orchestrates: every computation runs in the library.
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

from . import ensemble, fitcore, synth


def _parser():
    p = argparse.ArgumentParser(prog="python -m paper_2502_15253_gb300.cli")
    sub = p.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("config", help="write the JSON configuration of a synthetic model")
    c.add_argument("--model", required=True, choices=["c0", "c0_tiny", "c1", "c2", "c1s", "c1_flux41"])
    c.add_argument("--spline", action="store_true", help="area-conserving spline energy correction")
    c.add_argument("--seed", type=int, default=synth.BASE_SEED)
    c.add_argument("--out", default="-")
    q = sub.add_parser("pseudo", help="Poisson pseudo-data at the nominal point (GPU)")
    q.add_argument("--config", required=True)
    q.add_argument("--n", type=int, default=16)
    q.add_argument("--seed", type=int, default=1)
    q.add_argument("--out", required=True)
    f = sub.add_parser("fit", help="fit every row of a data file (GPU)")
    f.add_argument("--config", required=True)
    f.add_argument("--data", required=True)
    f.add_argument("--out", required=True)
    f.add_argument("--mask", type=int, default=0, help="datasets in the likelihood (0 = all)")
    f.add_argument("--chunk", type=int, default=4096)
    f.add_argument("--checkpoint", default=None)
    f.add_argument("--no-precondition", action="store_true")
    s = sub.add_parser("scan", help="1-D profile likelihood of one parameter (GPU)")
    s.add_argument("--config", required=True)
    s.add_argument("--data", required=True)
    s.add_argument("--row", type=int, default=0, help="which row of the data file")
    s.add_argument("--param", required=True, help="parameter name")
    s.add_argument("--lo", type=float, required=True)
    s.add_argument("--hi", type=float, required=True)
    s.add_argument("--points", type=int, default=41)
    s.add_argument("--mask", type=int, default=0, help="datasets in the likelihood (0 = all)")
    s.add_argument("--out", default="-")
    return p


def _bins_in_mask(cfg, mask):
    """Reco bins of the datasets selected by `mask`, from the configuration."""
    dets = cfg["detectors"]
    names = {d.get("name"): k for k, d in enumerate(dets)}
    total = 0
    for k, ds in enumerate(cfg["datasets"]):
        if mask >> k & 1:
            d = ds["detector"]
            total += len(dets[names[d] if isinstance(d, str) else int(d)]["response"])
    return total


def _scan(a, model, text, scan_fn):
    """Profile of -2lnL in one parameter (Eq. 7) on a raster, its Wilks intervals at 68.27 %
    and 95 %, and the goodness of fit of the best fit (Eq. 8)."""
    names = model.param_names()
    if names is None or a.param not in names:
        raise SystemExit(f"--param {a.param!r}: not a parameter of the model")
    if a.points < 2 or not a.hi > a.lo:
        raise SystemExit("--points >= 2 and --hi > --lo are needed")
    data = _load_data(a.data, model)
    if not 0 <= a.row < len(data):
        raise SystemExit(f"--row {a.row}: the data file has {len(data)} rows")
    mask = a.mask if a.mask else (1 << model.n_datasets) - 1
    x = np.linspace(a.lo, a.hi, a.points)
    r = (scan_fn or fitcore.fit_profile_scan)(model, data[a.row], mask, [names.index(a.param)],
                                              x[:, None])
    wilks = {}
    for level in (1.0, 3.84):
        lo, hi, op = fitcore.fit_wilks_interval(x, r["dchi2"], level)
        wilks[str(level)] = {"lo": lo, "hi": hi, "open_low": bool(op & 1), "open_high": bool(op & 2)}
    _, sigma = model.params()
    dof = _bins_in_mask(json.loads(text), mask) - int(np.sum(sigma == 0))
    d = [float(v) if np.isfinite(v) else None for v in np.asarray(r["dchi2"])]   # JSON: no NaN
    return {"param": a.param, "x": x.tolist(), "dchi2": d,
            "status": [fitcore.STATUS.get(int(v), str(int(v))) for v in r["status"]],
            "nll_min": float(r["nll_min"]),
            "best": dict(zip(names, np.asarray(r["theta_best"], dtype=float).tolist())),
            "wilks": wilks,
            "gof": {"chi2": float(r["nll_min"]), "dof": dof,
                    "p": fitcore.fit_chi2_sf(float(r["nll_min"]), dof)}}


def _read_config(path):
    with open(path) as fh:
        return fh.read()


def _load_data(path, model):
    data = np.load(path)
    data = np.ascontiguousarray(np.atleast_2d(data), dtype=np.float32)
    if data.shape[1] != model.n_data:
        raise SystemExit(f"{path}: rows hold {data.shape[1]} bins, the model has {model.n_data}")
    return data


def main(argv=None, model_factory=None, fit_fn=None, write_fn=None, scan_fn=None):
    """Runs one command. model_factory(json_text) -> model, fit_fn (see ensemble.fit_ensemble),
    write_fn(path, models, inst, best, results) and scan_fn (see fitcore.fit_profile_scan)
    replace the library calls in tests."""
    a = _parser().parse_args(argv)
    if a.cmd == "config":
        text = synth.make_model(a.model, a.seed, remap=int(a.spline)).to_json()
        if a.out == "-":
            sys.stdout.write(text + "\n")
        else:
            with open(a.out, "w") as fh:
                fh.write(text + "\n")
        return 0
    make = model_factory or fitcore.Model.from_json
    text = _read_config(a.config)
    model = make(text)
    if a.cmd == "scan":
        out = json.dumps(_scan(a, model, text, scan_fn))
        if a.out == "-":
            sys.stdout.write(out + "\n")
        else:
            with open(a.out, "w") as fh:
                fh.write(out + "\n")
        return 0
    if a.cmd == "pseudo":
        if a.n < 1:
            raise SystemExit("--n must be >= 1")
        th0, _ = model.params()
        mu = np.zeros((1, model.n_data), np.float32)
        fitcore.fit_model_expected(model, 1, th0[None], mu)
        mu = np.repeat(mu, a.n, axis=0)
        out = np.zeros_like(mu)
        fitcore.fit_poisson_sample(mu.size, mu, a.seed, 0, out)
        np.save(a.out, out)
        return 0
    data = _load_data(a.data, model)
    n = len(data)
    inst = np.zeros(n, fitcore.INSTANCE_DTYPE)
    inst["mask"] = a.mask if a.mask else (1 << model.n_datasets) - 1
    inst["data_off"] = np.arange(n) * model.n_data
    inst["param_off"] = np.arange(n) * model.n_params
    th0, _ = model.params()
    start = np.tile(th0, n)
    opts = None
    if fit_fn is None:
        opts = fitcore.fit_batch_default_opts()
        opts.precondition = 0 if a.no_precondition else 1
    best, res = ensemble.fit_ensemble_sharded([model], inst, data, start=start, opts=opts,
                                              chunk=a.chunk, checkpoint=a.checkpoint,
                                              fit_fn=fit_fn)
    if _rank() == 0:
        (write_fn or ensemble.write_results_json)(a.out, [model], inst, best, res)
        bad = int(np.sum(res["status"] != 0))
        print(json.dumps({"fits": n, "not_converged": bad, "out": a.out}))
    return 0


def _rank():
    try:
        import torch.distributed as dist
        return dist.get_rank() if dist.is_available() and dist.is_initialized() else 0
    except ImportError:
        return 0


def _init_distributed():
    """Under torchrun (WORLD_SIZE > 1): one process per GPU, the instances split over the ranks
    and the results gathered on the host (ensemble.fit_ensemble_sharded)."""
    import os
    if int(os.environ.get("WORLD_SIZE", "1")) <= 1:
        return
    import torch
    import torch.distributed as dist
    if torch.cuda.is_available():
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dist.init_process_group("gloo")   # the only exchange is the host-side gather of results


if __name__ == "__main__":
    _init_distributed()
    sys.exit(main())
