"""Command-line driver (host orchestration): the configuration it writes, and the fit command's
instance table, checkpointing and output with the library calls replaced by stand-ins."""
import json
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2502_15253_gb300 import cli, fitcore, synth


def test_config_command_writes_the_model_configuration(tmp_path):
    out = tmp_path / "c1.json"
    assert cli.main(["config", "--model", "c1", "--spline", "--out", str(out)]) == 0
    cfg = json.loads(out.read_text())
    assert cfg == json.loads(synth.make_model("c1", remap=1).to_json())
    assert cfg["energy_correction"] == "spline"


def test_fit_command_fits_every_row_and_resumes(tmp_path, capsys):
    spec = synth.make_model("c0")
    cfg = tmp_path / "c0.json"
    cfg.write_text(spec.to_json())
    n = 11
    data = np.random.default_rng(0).poisson(50.0, (n, spec.n_bins)).astype(np.float32)
    np.save(tmp_path / "d.npy", data)
    model = SimpleNamespace(n_data=spec.n_bins, n_params=spec.n_params,
                            n_datasets=len(spec.datasets),
                            params=lambda: (spec.theta0.copy(), spec.prior_sigma.copy()))
    seen, written = [], {}

    def fit_fn(models, sub, d, start, opts, fixed):
        seen.append(len(sub))
        assert np.all(sub["mask"] == 1) and d.shape == (n, spec.n_bins)
        best = np.array(start, dtype=np.float64)
        res = np.zeros(len(sub), fitcore.RESULT_DTYPE)
        res["iters"] = sub["data_off"] // spec.n_bins
        return best, res

    def write_fn(path, models, inst, best, res):
        written.update(path=path, best=best.copy(), res=res.copy(), inst=inst.copy())

    argv = ["fit", "--config", str(cfg), "--data", str(tmp_path / "d.npy"), "--out",
            str(tmp_path / "f.jsonl"), "--chunk", "4", "--checkpoint", str(tmp_path / "ck.npz")]
    assert cli.main(argv, model_factory=lambda text: model, fit_fn=fit_fn, write_fn=write_fn) == 0
    assert seen == [4, 4, 3]
    assert json.loads(capsys.readouterr().out.strip().splitlines()[-1]) == {
        "fits": n, "not_converged": 0, "out": str(tmp_path / "f.jsonl")}
    np.testing.assert_array_equal(written["res"]["iters"], np.arange(n))
    np.testing.assert_array_equal(written["best"], np.tile(spec.theta0, n))
    np.testing.assert_array_equal(written["inst"]["param_off"], np.arange(n) * spec.n_params)
    # the same command again finds every instance done in its checkpoint
    seen.clear()
    assert cli.main(argv, model_factory=lambda text: model, fit_fn=fit_fn, write_fn=write_fn) == 0
    assert seen == []


def test_fit_command_rejects_data_of_another_model(tmp_path):
    spec = synth.make_model("c0")
    cfg = tmp_path / "c0.json"
    cfg.write_text(spec.to_json())
    np.save(tmp_path / "d.npy", np.zeros((2, spec.n_bins + 1), np.float32))
    model = SimpleNamespace(n_data=spec.n_bins, n_params=spec.n_params, n_datasets=1,
                            params=lambda: (spec.theta0, spec.prior_sigma))
    with pytest.raises(SystemExit, match="bins"):
        cli.main(["fit", "--config", str(cfg), "--data", str(tmp_path / "d.npy"), "--out",
                  str(tmp_path / "f.jsonl")], model_factory=lambda text: model,
                 fit_fn=lambda *a: None)


def _cli_worker(rank, world, port, d):
    import os
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    from paper_2502_15253_gb300 import cli as c
    c._init_distributed()
    spec = synth.make_model("c0")
    model = SimpleNamespace(n_data=spec.n_bins, n_params=spec.n_params, n_datasets=1,
                            params=lambda: (spec.theta0.copy(), spec.prior_sigma.copy()))

    def fit_fn(models, sub, data, start, opts, fixed):
        res = np.zeros(len(sub), fitcore.RESULT_DTYPE)
        res["iters"] = sub["data_off"] // spec.n_bins
        res["n_evals"] = rank
        return np.array(start, dtype=np.float64), res

    def write_fn(path, models, inst, best, res):
        np.save(path, res.view(np.uint8))

    c.main(["fit", "--config", os.path.join(d, "c0.json"), "--data", os.path.join(d, "d.npy"),
            "--out", os.path.join(d, f"out{rank}.npy"), "--chunk", "3"],
           model_factory=lambda text: model, fit_fn=fit_fn, write_fn=write_fn)
    dist.destroy_process_group()


def test_fit_command_under_two_gloo_ranks(tmp_path):
    """Under torchrun-style environment variables the fit command splits the rows over the
    ranks; rank 0 alone writes every row's record."""
    torch = pytest.importorskip("torch")
    import socket
    import torch.multiprocessing as mp
    if torch.cuda.is_available():
        pytest.skip("the host-only (gloo) path is exercised where no GPU is visible")
    spec = synth.make_model("c0")
    (tmp_path / "c0.json").write_text(spec.to_json())
    n = 9
    np.save(tmp_path / "d.npy", np.ones((n, spec.n_bins), np.float32))
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.spawn(_cli_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    assert not (tmp_path / "out1.npy").exists()
    res = np.load(tmp_path / "out0.npy").view(fitcore.RESULT_DTYPE)
    np.testing.assert_array_equal(res["iters"], np.arange(n))
    np.testing.assert_array_equal(res["n_evals"], [0] * 5 + [1] * 4)   # rows 0-4 on rank 0


def test_scan_command_reports_profile_intervals_and_goodness_of_fit(tmp_path, capsys):
    """The scan command with the library's profile fit replaced by a parabola of width 0.02
    around 0.09: Wilks intervals at +-1 and +-1.96 widths; the goodness of fit counts the
    bins of the selected datasets minus the parameters without a prior (c0: 40 - 2)."""
    from scipy import stats
    spec = synth.make_model("c0")
    (tmp_path / "c0.json").write_text(spec.to_json())
    np.save(tmp_path / "d.npy", np.ones((3, spec.n_bins), np.float32))
    sigma = spec.prior_sigma.copy()   # as fit_model_params reports them: sqrt(V_ii) in blocks
    for ix, cov in spec.cov_blocks:
        sigma[np.asarray(ix)] = np.sqrt(np.diag(cov))
    model = SimpleNamespace(n_data=spec.n_bins, n_params=spec.n_params, n_datasets=1,
                            params=lambda: (spec.theta0.copy(), sigma),
                            param_names=lambda: list(spec.param_names))
    calls = []

    def scan_fn(m, data, mask, idx, pts):
        calls.append((data.shape, mask, list(idx)))
        x = pts[:, 0]
        return dict(nll_min=41.0, theta_best=spec.theta0, dchi2=((x - 0.09) / 0.02) ** 2,
                    status=np.zeros(len(x), np.int32))

    fitcore.load()
    argv = ["scan", "--config", str(tmp_path / "c0.json"), "--data", str(tmp_path / "d.npy"),
            "--row", "2", "--param", "sin2_2th13", "--lo", "0.0", "--hi", "0.2", "--points", "201"]
    assert cli.main(argv, model_factory=lambda t: model, scan_fn=scan_fn) == 0
    out = json.loads(capsys.readouterr().out)
    assert calls == [((spec.n_bins,), 1, [spec.index("sin2_2th13")])]
    w1, w2 = out["wilks"]["1.0"], out["wilks"]["3.84"]
    assert w1["lo"] == pytest.approx(0.07, abs=1e-5) and w1["hi"] == pytest.approx(0.11, abs=1e-5)
    assert w2["lo"] == pytest.approx(0.09 - 0.02 * 3.84 ** 0.5, abs=1e-5)
    assert not (w1["open_low"] or w1["open_high"])
    assert out["gof"]["dof"] == 38
    assert out["gof"]["p"] == pytest.approx(stats.chi2.sf(41.0, 38), rel=1e-9)
    assert out["best"]["sin2_2th13"] == spec.theta0[0] and out["status"][0] == "converged"
    with pytest.raises(SystemExit, match="not a parameter"):
        cli.main(argv[:7] + ["--param", "nope"] + argv[9:], model_factory=lambda t: model,
                 scan_fn=scan_fn)
