"""Benchmark: batched cold-start fits of an uneven ensemble of pseudo-experiments, fits/s on one
or more GPUs.

Default workload: 8192 pseudo-experiments per rank, two thirds of the two-detector
three-dataset model (FD-I, FD-II, ND; 291 parameters; each instance fits a dataset subset drawn
from {FD-I}, {FD-II + ND}, {all three}) and one third of the 53 km ten-core model with a near
detector (460 parameters, 2000 true / 400 + 38 reco bins), true signal parameters uniform within
+-3 sigma, Poisson counts, cold start at the nominal point.

One step = one fit_batch() call over all of them: every evaluation of the expectation, -2lnL,
adjoint gradient and every L-BFGS update runs in the library's kernels. Inputs are resident in
device memory when the timed region starts; L2 is flushed (a 512 MiB write) before every timed
step. With torchrun, each rank fits its own instances (weak scaling, no collective on the data
path); the step time is the maximum over ranks and value = total fits / that time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--workload c3|c0|c1|c2]
                  [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("fits/s at |Δ(−2lnL_min)|≤1e-3 vs FP64 oracle; eval+grad/s; "
          "HBM/tensor % peak")
WORKLOADS = {
    "c3": ("uneven ensemble: 2/3 two-detector three-dataset model (FD-I, FD-II, ND; 291 params, "
           "400 true / 3x38 reco bins; fitted dataset subset drawn from {FD-I}, {FD-II+ND}, "
           "{all}) + 1/3 53 km JUNO-like model (10 cores + near detector; 460 params, 2000 true / "
           "400+38 reco bins); true signal parameters uniform within +-3 sigma, Poisson counts"),
    "c0": "single detector, one dataset: 25 params, 200 true / 40 reco bins",
    "c1": "two-detector three-dataset fit (FD-I, FD-II, ND), 291 params, 400 true / 3x38 reco bins",
    "c2": "53 km JUNO-like model: 10 cores + near detector, 460 params, 2000 true / 400+38 reco bins",
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--batch", type=int, default=8192, help="fits per rank per step")
    p.add_argument("--workload", default="c3", choices=sorted(WORKLOADS),
                   help="c3: the uneven two-model ensemble (default); c0/c1/c2: one model")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--cpu-sample", type=int, default=512,
                   help="instances of the CPU baseline (10-30 s of the FP64 oracle on 16 cores)")
    p.add_argument("--ref-sample", type=int, default=48,
                   help="instances per step of the reference arm (the FP64 oracle)")
    p.add_argument("--no-per-config", action="store_true",
                   help="skip the per-model sub-lines (c0, c1, c2 alone)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--seed", type=int, default=250215253)
    p.add_argument("--engine", default="persistent", choices=["persistent", "lockstep", "lockstep_tc"],
                   help="fit engine: one persistent launch, or one round of launches per evaluation "
                        "(lockstep_tc: the folds as tensor-core GEMMs)")
    p.add_argument("--mc-events", type=int, default=20_000_000,
                   help="simulated events of the event-reweighting measurement (0: skip)")
    p.add_argument("--no-autotune", action="store_true",
                   help="skip the launch autotuner and the CUDA-graph launch (plain defaults)")
    p.add_argument("--no-precondition", action="store_true",
                   help="fit in plain whitened coordinates (no Fisher preconditioner)")
    p.add_argument("--no-profile", action="store_true",
                   help="skip the profile-likelihood and mass-ordering scans")
    p.add_argument("--no-warm-start", action="store_true",
                   help="skip the warm-start network measurement")
    p.add_argument("--ws-samples", type=int, default=2_000_000,
                   help="training samples of the warm-start network (both geometries)")
    p.add_argument("--ws-epochs", type=int, default=12,
                   help="passes of the warm-start training over its samples")
    return p.parse_args()


# ---------------------------------------------------------------------------------------
# algorithmic work model (FP32 operations of one evaluation + gradient)
# ---------------------------------------------------------------------------------------
def flops_per_eval(spec, mask) -> float:
    """Algorithmic FP32 FLOPs of one -2lnL + gradient evaluation of one instance."""
    from paper_2502_15253_gb300 import synth
    f = 0.0
    nt = spec.n_true
    surv = 80.0 if spec.osc_mode == synth.OSC_EQ1 else 95.0   # P and its 4 partials, 2 phases
    for d, ds in enumerate(spec.datasets):
        if not (mask >> d) & 1:
            continue
        nnz = np.count_nonzero(spec.detectors[ds.det].response)
        ncore = int(np.count_nonzero(ds.weight))
        nr = spec.detectors[ds.det].n_reco
        f += nt * ncore * (surv + 2 * 6)          # survival + weighted sums of P and dP
        f += nt * 60.0                            # reweights, energy map forward + adjoint
        f += 4.0 * nnz                            # fold and its adjoint (2 FLOPs per MAC)
        f += nr * (25.0 + 6 * len(ds.backgrounds))  # backgrounds, deviance, dD/dmu
    blk = sum(len(ix) ** 2 for ix, _ in spec.cov_blocks)
    f += 2.0 * blk + 10.0 * spec.n_params        # transformation layer theta(z), J^T g
    return f


def flops_lbfgs_iter(P, m) -> float:
    """One L-BFGS iteration with m pairs: 4m + 1 dot products (2P each), the direction
    combination over 2m + 1 vectors (2P each) and ~10P of vector updates."""
    return (4.0 * m + 1) * 2.0 * P + (2.0 * m + 1) * 2.0 * P + 10.0 * P


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index),
                                          f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------------------
class Workload:
    """Instances of one benchmark workload. names[k] / specs[k] / models[k] belong to
    inst["model"] == k. Data and parameter vectors are laid out model by model (all instances of
    names[0] first), so that each model's instances form one contiguous [n, n_bins] block;
    the instance table keeps the ensemble's order."""

    def __init__(self, kind, names, specs, table, mu_of):
        self.kind, self.names, self.specs = kind, list(names), list(specs)
        self.table = table
        B = len(table)
        self.geo = np.array([self.names.index(t.model) for t in table], np.int32)
        self.inst = np.zeros(B, _fitcore().INSTANCE_DTYPE)
        self.inst["model"] = self.geo
        self.inst["mask"] = [t.mask for t in table]
        self.group = [np.flatnonzero(self.geo == k) for k in range(len(names))]
        self.data_base, self.par_base = [], []
        d0 = p0 = 0
        for k, sp in enumerate(self.specs):
            ix = self.group[k]
            self.data_base.append(d0)
            self.par_base.append(p0)
            self.inst["data_off"][ix] = d0 + np.arange(len(ix), dtype=np.int64) * sp.n_bins
            self.inst["param_off"][ix] = p0 + np.arange(len(ix), dtype=np.int64) * sp.n_params
            d0 += len(ix) * sp.n_bins
            p0 += len(ix) * sp.n_params
        self.data_len, self.par_len = d0, p0
        self.data = np.zeros(d0, np.float32)
        self.truth = np.zeros(p0)
        for k, sp in enumerate(self.specs):
            ix = self.group[k]
            if not len(ix):
                continue
            th = np.stack([table[i].theta_true for i in ix])
            mu = mu_of(k, th)
            for j, i in enumerate(ix):
                o = int(self.inst["data_off"][i])
                self.data[o:o + sp.n_bins] = synth_mod().poisson_data(mu[j], table[i].seed)
                po = int(self.inst["param_off"][i])
                self.truth[po:po + sp.n_params] = th[j]
        self.start = np.zeros(p0)
        for i, r in enumerate(self.inst):
            sp = self.specs[r["model"]]
            self.start[r["param_off"]:r["param_off"] + sp.n_params] = sp.theta0

    def __len__(self):
        return len(self.table)

    def view(self, flat, k, i_local):
        """Slice of a flat per-parameter array for the i_local-th instance of model k."""
        sp = self.specs[k]
        o = self.par_base[k] + i_local * sp.n_params
        return flat[o:o + sp.n_params]

    def data_of(self, i):
        sp = self.specs[self.geo[i]]
        o = int(self.inst["data_off"][i])
        return self.data[o:o + sp.n_bins]

    def params_of(self, flat, i):
        sp = self.specs[self.geo[i]]
        o = int(self.inst["param_off"][i])
        return flat[o:o + sp.n_params]


def _fitcore():
    from paper_2502_15253_gb300 import fitcore
    return fitcore


def synth_mod():
    from paper_2502_15253_gb300 import synth
    return synth


def draw_table(kind, B, base, remap=0):
    """(model names, specs, instance table) of a workload; instance i draws from SplitMix64(base
    + i): its model and dataset subset (c3 only), its true signal parameters (uniform within
    +-3 sigma) and its Poisson stream."""
    synth = synth_mod()
    if kind == "c3":
        names = ["c1", "c2"]
        specs = {n: synth.make_model(n, remap=remap) for n in names}
        table = synth.make_ensemble(B, specs, base=base)
    else:
        names = [kind]
        specs = {kind: synth.make_model(kind, remap=remap)}
        sp = specs[kind]
        table = []
        for i in range(B):
            s = synth.instance_seed(i, base)
            rng = np.random.default_rng(s)
            table.append(synth.Instance(kind, sp.all_mask(), synth.draw_theta_true(sp, rng), s))
    return names, [specs[n] for n in names], table


def make_workload(kind, B, seed, rank, remap=0):
    """The workload's B instances of this rank (instances rank*B .. rank*B + B - 1 of the seeded
    table) with the library's models; expectations from the library, Poisson counts from
    numpy's PCG64 stream of each instance's seed."""
    fitcore = _fitcore()
    names, specs, table = draw_table(kind, B, seed + rank * B, remap)
    models = [fitcore.Model(sp) for sp in specs]

    def mu_of(k, th):
        mu, st = fitcore.expected_numpy(models[k], th)
        assert np.all(st == 0)
        return mu

    w = Workload(kind, names, specs, table, mu_of)
    w.models = models
    return w


def make_workload_oracle(kind, B, seed):
    """The same instance table with the oracle's models and expectations (reference arm)."""
    import oracle
    names, specs, table = draw_table(kind, B, seed)
    oms = [oracle.OracleModel(sp) for sp in specs]

    def mu_of(k, th):
        return np.stack([oms[k].expected(t) for t in th])

    w = Workload(kind, names, specs, table, mu_of)
    w.oms = oms
    return w


def config_of(args, world, B):
    """The workload description shared by both arms' JSON lines."""
    return {"workload": WORKLOADS[args.workload], "instances_per_rank": B,
            "start": "nominal (cold)", "l2": "flushed (512 MiB write) before each step",
            "parallelism": f"instances sharded over {world} GPU(s), no collective"}


_COLL_DEVICE = "cpu"


def dist_setup(args):
    """Rank layout from the torchrun environment; NCCL with one GPU per rank when CUDA is
    present, gloo on the host otherwise (the path has no collective on its data; only the
    barrier and the max of the step times cross ranks)."""
    global _COLL_DEVICE
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
            _COLL_DEVICE = "cuda"
        else:
            dist.init_process_group("gloo")
            _COLL_DEVICE = "cpu"
        pg = dist
    return world, rank, local, pg


def shard_range(n_total, rank, world):
    """Contiguous share of n_total units for a rank (the first n_total % world ranks get +1),
    the same split as the library's sharded ensembles."""
    from paper_2502_15253_gb300.ensemble import shard
    return shard(n_total, rank, world)


def max_over_ranks(x, pg):
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=_COLL_DEVICE)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg):
    if pg is not None:
        pg.barrier()


def cpu_baseline(w, n, threads=None):
    """The FP64 oracle (dense BFGS, OpenMP over instances) on the host cores, fitting the first n
    instances of workload w from the same cold start."""
    import oracle
    oms = [oracle.OracleModel(sp) for sp in w.specs]
    threads = threads or os.cpu_count() or 1
    ds = [w.data_of(i).astype(np.float64) for i in range(n)]
    starts = [w.specs[w.geo[i]].theta0 for i in range(n)]
    t0 = time.perf_counter()
    r = oracle.fit_many(oms, [int(g) for g in w.geo[:n]], ds, [int(m) for m in w.inst["mask"][:n]],
                        starts, edm_tol=1e-10, n_threads=threads)
    dt = time.perf_counter() - t0
    cnt = {nm: int(np.sum(w.geo[:n] == k)) for k, nm in enumerate(w.names)}
    return {"value": n / dt, "unit": "fits/s", "cores": threads if oracle.openmp_enabled() else 1,
            "kind": "oracle", "sample": f"first {n} instances of the same workload "
            f"({', '.join(f'{v} {k}' for k, v in cnt.items())}), cold start, FP64 dense BFGS "
            f"(EDM < 1e-10), {dt:.1f} s", "s": dt,
            "_r": r, "_oms": oms, "_ds": ds}


def certify(cpu, w, gpu_best, gpu_nll):
    """Parity of the GPU minima on the oracle's sample: |d(-2lnL_min)| per instance and per
    model; an instance beyond 1e-3 is certified when the oracle restarted at the GPU point stays
    there (another minimum of the FP64 likelihood) and counted apart."""
    r, oms, ds = cpu.pop("_r"), cpu.pop("_oms"), cpu.pop("_ds")
    n = len(ds)
    dn = gpu_nll[:n] - r["nll"]
    d = np.abs(dn)
    other = np.flatnonzero(d > 1e-3)
    cert = 0
    for i in other:
        th = w.params_of(gpu_best, i)
        om = oms[w.geo[i]]
        m = int(w.inst["mask"][i])
        rr = om.fit(ds[i], mask=m, start=th)
        cert += int(rr["status"] == 0 and abs(rr["nll"] - om.nll(th, ds[i], mask=m)) <= 1e-4)
    cpu["parity_max_abs_dnll"] = float(d.max()) if n else None
    cpu["parity_frac_within_1e-3"] = float(np.mean(d <= 1e-3)) if n else None
    cpu["parity_other_minima"] = int(len(other))
    cpu["parity_other_minima_certified"] = int(cert)
    cpu["parity_other_minima_gpu_lower"] = int(np.sum(dn[other] < 0))
    cpu["oracle_converged_frac"] = float(np.mean(r["status"] == 0)) if n else None
    per = {}
    for k, nm in enumerate(w.names):
        ix = np.flatnonzero(w.geo[:n] == k)
        if len(ix):
            per[nm] = {"n": int(len(ix)), "frac_within_1e-3": float(np.mean(d[ix] <= 1e-3)),
                       "max_abs_dnll": float(d[ix].max()),
                       "oracle_iters_per_fit": float(np.mean(r["iters"][ix]))}
    cpu["parity_per_model"] = per
    return cpu


def mlp_flops_per_sample(dims, train):
    """Multiply-adds x 2 of the network's products per sample: forward; training adds the
    weight gradients (same count) and the input gradients of every layer but the first."""
    fwd = [2 * i * o for i, o in zip(dims[:-1], dims[1:])]
    return sum(fwd) * 2 + sum(fwd[1:]) if train else sum(fwd)


def r2_per_target(pred, truth, names):
    """Coefficient of determination of pred against truth, per column."""
    out = {}
    for j, nm in enumerate(names):
        v = np.var(truth[:, j])
        out[nm] = float(1.0 - np.mean((pred[:, j] - truth[:, j]) ** 2) / v) if v > 0 else None
    return out


def warm_start_measurement(args, w, data_d, cold_res, cold_best, opts, stream, flush, pg, world):
    """Warm start (not in the paper): train the network on device-drawn samples of both
    geometries, time one bf16 training step on the tensor cores, the TF32 fold of a training
    batch, and fits of the benchmark's pseudo-experiments (held out: the training samples come
    from the device generator) from the predicted starts, per model, against the cold fits."""
    import torch
    from paper_2502_15253_gb300 import fitcore, synth, warmstart

    dev = data_d.device
    B = len(w)
    by_name = dict(zip(w.names, w.models))
    specs_by_name = dict(zip(w.names, w.specs))
    tr_specs = [specs_by_name.get(n) or synth.make_model(n) for n in ("c1", "c2")]
    tr_models = [by_name.get(n) or fitcore.Model(s) for n, s in zip(("c1", "c2"), tr_specs)]
    net = warmstart.network(seed=3)
    batch = 4096
    n_steps = max(2, args.ws_samples // batch)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    losses = warmstart.train(net, tr_models, tr_specs, n_steps=n_steps, batch=batch,
                             lr=1e-3, stream=stream, epochs=args.ws_epochs)
    ev1.record(stream)
    torch.cuda.synchronize()
    train_s = ev0.elapsed_time(ev1) / 1e3

    # one training step alone (bf16 GEMMs, fused epilogues, AdamW) on a resident batch
    dims = [warmstart.N_IN] + [warmstart.N_HIDDEN] * warmstart.N_HIDDEN_LAYERS + [warmstart.N_OUT]
    tb = 16384
    x = torch.randn((tb, warmstart.N_IN), dtype=torch.float32, device=dev)
    y = torch.randn((tb, warmstart.N_OUT), dtype=torch.float32, device=dev)
    probe = warmstart.network(seed=4)
    for _ in range(3):
        probe.train_step(tb, x, y, 1e-4, 0.0, None, stream)
    reps = 20
    ev0.record(stream)
    for _ in range(reps):
        probe.train_step(tb, x, y, 1e-4, 0.0, None, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    step_ms = ev0.elapsed_time(ev1) / reps
    peaks = read_peaks()
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    mlp_tflops = mlp_flops_per_sample(dims, True) * tb / (step_ms / 1e3) / 1e12

    # TF32 fold of a 53 km training batch: V [B x 2000] times R^T for both detectors
    spec2, model2 = tr_specs[1], tr_models[1]
    fb = 8192
    th2 = torch.zeros((fb, spec2.n_params), dtype=torch.float64, device=dev)
    fitcore.fit_warmstart_draw(model2, warmstart.geometry(spec2), fb, 11, 0, th2, None, stream)
    mu2 = torch.zeros((fb, spec2.n_bins), dtype=torch.float32, device=dev)
    for _ in range(3):
        fitcore.fit_model_expected_tc(model2, fb, th2, mu2, None, 0, stream)
    ev0.record(stream)
    for _ in range(5):
        fitcore.fit_model_expected_tc(model2, fb, th2, mu2, None, 0, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    fold_ms = ev0.elapsed_time(ev1) / 5
    n_t = spec2.n_true
    fold_flops = 2.0 * fb * n_t * sum(spec2.detectors[d.det].n_reco for d in spec2.datasets)
    tf32_peak = bf16_peak * 1.1 / 2.25
    del th2, mu2

    # the fold's tensor-core GEMM alone at the same shape: V [fb x N_t'] (FP32 read as TF32)
    # times the far detector's response [400 x N_t']^T
    ldk = (n_t + 3) // 4 * 4
    Va = torch.rand((fb, ldk), dtype=torch.float32, device=dev)
    Rb = torch.rand((400, ldk), dtype=torch.float32, device=dev)
    Cc = torch.empty((fb, 400), dtype=torch.float32, device=dev)
    for _ in range(3):
        fitcore.fit_tc_gemm(1, fb, 400, n_t, Va, ldk, Rb, ldk, 0, Cc, 400, stream=stream)
    ev0.record(stream)
    for _ in range(10):
        fitcore.fit_tc_gemm(1, fb, 400, n_t, Va, ldk, Rb, ldk, 0, Cc, 400, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    gemm_ms = ev0.elapsed_time(ev1) / 10
    gemm_tflops = 2.0 * fb * 400 * n_t / (gemm_ms / 1e3) / 1e12
    del Va, Rb, Cc

    # warm fits of the benchmark's pseudo-experiments: starts predicted per model
    starts = torch.from_numpy(w.start.copy()).to(dev)
    masks_d = torch.from_numpy(w.inst["mask"].astype(np.int32)).to(dev)
    flush.fill_(0.5)

    def predict(mode="network"):
        for k, (nm, sp, m) in enumerate(zip(w.names, w.specs, w.models)):
            ix = w.group[k]
            if not len(ix):
                continue
            n = len(ix)
            dv = data_d[w.data_base[k]:w.data_base[k] + n * sp.n_bins].view(n, sp.n_bins)
            sv = starts[w.par_base[k]:w.par_base[k] + n * sp.n_params].view(n, sp.n_params)
            mk = masks_d[torch.from_numpy(ix).to(dev)].contiguous()
            if mode == "linear":
                fitcore.fit_linear_start(m, n, dv, mk, sv, stream)
            else:
                warmstart.predict_starts(net, m, sp, n, dv, mk, sv, stream)

    def run_mode(mode):
        """Fits from the starts of `mode`: one-time set-up (the linearised rows of each model
        and dataset subset), start computation + fits and the fits alone over three steps."""
        best_v = torch.zeros_like(cold_best)
        res_v = torch.zeros(B * fitcore.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        predict(mode)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        fitcore.fit_batch(w.models, w.inst, data_d, starts, best_v, res_v, opts, stream)
        torch.cuda.synchronize()
        ev3 = torch.cuda.Event(enable_timing=True)
        tt, fo = [], []
        for r in range(3):
            flush.fill_(0.75 + r)
            ev0.record(stream)
            predict(mode)
            ev3.record(stream)
            fitcore.fit_batch(w.models, w.inst, data_d, starts, best_v, res_v, opts, stream)
            ev1.record(stream)
            torch.cuda.synchronize()
            tt.append(ev0.elapsed_time(ev1))
            fo.append(ev3.elapsed_time(ev1))
        ms_t = max_over_ranks(float(np.mean(tt)), pg)
        ms_f = max_over_ranks(float(np.mean(fo)), pg)
        rv = np.frombuffer(res_v.cpu().numpy().tobytes(), dtype=fitcore.RESULT_DTYPE)
        sm = np.abs(rv["nll_min"] - cold_res["nll_min"]) <= 1e-3
        return {"fits_per_s": world * B / (ms_t / 1e3), "fits_per_s_fits_alone": world * B / (ms_f / 1e3),
                "start_ms": ms_t - ms_f, "first_call_s": setup_s,
                "same_minimum_as_cold_frac": float(sm.mean()),
                "converged_frac": float(np.mean(rv["status"] == 0)),
                "per_model": {nm: {"evals_per_fit": float(rv["n_evals"][w.group[k]].mean()),
                                   "evals_per_fit_cold": float(cold_res["n_evals"][w.group[k]].mean()),
                                   "iters_per_fit": float(rv["iters"][w.group[k]].mean()),
                                   "same_minimum_as_cold_frac": float(sm[w.group[k]].mean())}
                              for k, nm in enumerate(w.names) if len(w.group[k])}}

    best_w = torch.zeros_like(cold_best)
    res_w = torch.zeros(B * fitcore.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    predict()
    fitcore.fit_batch(w.models, w.inst, data_d, starts, best_w, res_w, opts, stream)  # warm-up
    torch.cuda.synchronize()
    ev2 = torch.cuda.Event(enable_timing=True)
    tot, fit_only = [], []
    for r in range(3):   # inference + fits, and the fits alone, over three steps
        flush.fill_(0.25 + r)
        ev0.record(stream)
        predict()
        ev2.record(stream)
        fitcore.fit_batch(w.models, w.inst, data_d, starts, best_w, res_w, opts, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        tot.append(ev0.elapsed_time(ev1))
        fit_only.append(ev2.elapsed_time(ev1))
    warm_ms = max_over_ranks(float(np.mean(tot)), pg)
    warm_fit_ms = max_over_ranks(float(np.mean(fit_only)), pg)
    rw = np.frombuffer(res_w.cpu().numpy().tobytes(), dtype=fitcore.RESULT_DTYPE)
    same = np.abs(rw["nll_min"] - cold_res["nll_min"]) <= 1e-3
    st_h = starts.cpu().numpy()
    cb_h = cold_best.cpu().numpy()
    per = {}
    for k, nm in enumerate(w.names):
        ix = w.group[k]
        if not len(ix):
            continue
        g = warmstart.geometry(w.specs[k])
        tix = list(g.target_idx)[:g.n_targets]
        tnames = [w.specs[k].param_names[j] for j in tix]
        pred = np.stack([w.params_of(st_h, i)[tix] for i in ix])
        fit = np.stack([w.params_of(cb_h, i)[tix] for i in ix])
        tru = np.stack([w.params_of(w.truth, i)[tix] for i in ix])
        per[nm] = {"n": int(len(ix)),
                   "iters_per_fit_warm": float(rw["iters"][ix].mean()),
                   "iters_per_fit_cold": float(cold_res["iters"][ix].mean()),
                   "evals_per_fit_warm": float(rw["n_evals"][ix].mean()),
                   "evals_per_fit_cold": float(cold_res["n_evals"][ix].mean()),
                   "same_minimum_as_cold_frac": float(same[ix].mean()),
                   "converged_frac_warm": float(np.mean(rw["status"][ix] == 0)),
                   "rms_error_in_widths_network": {nm: float(np.sqrt(np.mean(((pred[:, j] - fit[:, j])
                                                                               / g.target_scale[j]) ** 2)))
                                                   for j, nm in enumerate(tnames)},
                   "rms_error_in_widths_nominal": {nm: float(np.sqrt(np.mean(((w.specs[k].theta0[tix[j]]
                                                                               - fit[:, j])
                                                                              / g.target_scale[j]) ** 2)))
                                                   for j, nm in enumerate(tnames)},
                   "r2_network_vs_cold_fit": r2_per_target(pred, fit, tnames),
                   "r2_network_vs_truth": r2_per_target(pred, tru, tnames),
                   "r2_cold_fit_vs_truth": r2_per_target(fit, tru, tnames)}
    lin = run_mode("linear")
    return {
        "note": "not in the paper: start points from the linearised best fit of every parameter "
                "(one Gauss-Newton step from theta0) with the network's corrections on its 12 "
                "targets; every fit still runs to the same EDM tolerance. The held-out set is the "
                "benchmark's own instances. The network is trained on where a fit ends (the "
                "linearised best fit from each training sample's drawn point) minus the start from "
                "theta0; r2_network_vs_cold_fit compares the combined start of those 12 parameters "
                "with the cold best fit (1 = the best any start of these 12 can do), null where a "
                "target does not vary",
        "train_samples": n_steps * batch, "train_epochs": args.ws_epochs, "train_s": train_s,
        "train_samples_per_s": args.ws_epochs * n_steps * batch / train_s,
        "train_loss_first_last": [float(losses[:2].mean()), float(losses[-20:].mean())],
        "mlp_train_step": {"batch": tb, "ms": step_ms, "achieved": mlp_tflops,
                           "unit": "TFLOP/s", "peak": bf16_peak, "frac": mlp_tflops / bf16_peak,
                           "bound": "tensor", "dtype": "bf16",
                           "flops_per_sample": mlp_flops_per_sample(dims, True)},
        "fold_tf32_53km": {"batch": fb, "ms": fold_ms, "achieved": fold_flops / fold_ms / 1e9,
                           "unit": "TFLOP/s", "peak": tf32_peak,
                           "frac": fold_flops / fold_ms / 1e9 / tf32_peak,
                           "peak_note": "measured bf16 burst x 1.1/2.25 (nominal tf32/bf16)",
                           "timed": "whole fit_model_expected_tc call (spectra, GEMMs, epilogue)"},
        "fold_gemm_tf32_alone": {"M": fb, "N": 400, "K": n_t, "ms": gemm_ms, "achieved": gemm_tflops,
                                 "unit": "TFLOP/s", "peak": tf32_peak, "frac": gemm_tflops / tf32_peak,
                                 "bound": "tensor", "kernel": "tc_gemm_kernel<TF32>"},
        "fits_per_s_warm": world * B / (warm_ms / 1e3),
        "warm_ms_incl_inference": warm_ms,
        "fits_per_s_warm_fits_alone": world * B / (warm_fit_ms / 1e3),
        "inference_ms": warm_ms - warm_fit_ms,
        "iters_per_fit_warm": float(rw["iters"].mean()),
        "iters_per_fit_cold": float(cold_res["iters"].mean()),
        "same_minimum_as_cold_frac": float(same.mean()),
        "converged_frac_warm": float(np.mean(rw["status"] == 0)),
        "per_model": per,
        "linear_start_alone": dict(lin, note="the warm start without the network: every parameter "
                                             "at the linearised best fit (one Gauss-Newton step of -2lnL "
                                             "from theta0 with the expected Hessian; fit_linear_start, "
                                             "split-TF32 tensor-core GEMMs per model and dataset subset)"),
    }


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except Exception:
            return {}
    return {}


# DRAM bytes (read + write) per fit of the fit kernel by workload, from ncu captures of the current
# kernel on a smaller launch of the same workload (traffic grows with the fits)
FIT_DRAM_BYTES_PER_FIT = {
    "c3": {"per_fit": (42.005760e6 + 331.655168e6) / 760,
           "note": "DRAM read+write bytes per fit of an ncu capture of this kernel on 760 fits of "
                   "the same recipe (42.0 MB read, 331.7 MB written), scaled to the launch"},
}

# DRAM bytes (read + write) per event of mc_spectrum_kernel for one parameter set, from an ncu
# capture of 11,904,680 events (154.81 MB read, 3.62 MB written); traffic grows with the events
MC_DRAM_BYTES_PER_EVENT = (154.811136e6 + 3.620096e6) / 11_904_680


def event_reweighting_measurement(args, stream, pg, world):
    """Event-level reweighting (the loop the paper moves to the GPU): oscillated spectra of
    args.mc_events simulated events of the two-core far detector (13 bytes an event, resident,
    larger than L2) for one parameter set (HBM-bound) and for 16 sets in one pass."""
    import torch
    from paper_2502_15253_gb300 import fitcore, synth

    ev = synth.make_mc_events(args.mc_events, "dc_fd", seed=args.seed + 7)
    n = len(ev.energy)
    mc = fitcore.McEventSet(ev)
    dev = torch.device("cuda", torch.cuda.current_device())
    peaks = {}
    peak_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peak_path):
        peaks = json.load(open(peak_path))
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    out = {"note": "per-event survival weights summed per reco bin (Eq. 1), FP32 with "
                   "float-pair phases, FP64 bin sums",
           "workload": f"two-core far detector, {n} events sorted by reco bin, 38 bins",
           "bytes_per_event": 13}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rng = np.random.default_rng(args.seed)
    for B in (1, 16):
        prm = np.tile(ev.osc_nominal, (B, 1)) * rng.uniform(0.8, 1.2, (B, 4))
        pd = torch.tensor(prm, dtype=torch.float64, device=dev)
        od = torch.zeros((B, ev.n_bins), dtype=torch.float64, device=dev)
        for _ in range(3):
            mc.spectrum(B, pd, od, stream)
        reps = 20
        barrier(pg)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            mc.spectrum(B, pd, od, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1) / reps, pg)
        r = {"sets": B, "ms": ms, "events_per_s": world * n / (ms / 1e3),
             "event_sets_per_s": world * n * B / (ms / 1e3)}
        if B == 1:
            gbs = 13.0 * n / (ms / 1e3) / 1e9
            r["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                             "frac": gbs / hbm_peak, "traffic": MC_DRAM_BYTES_PER_EVENT * n,
                             "traffic_note": "DRAM read+write bytes per event of an ncu capture "
                                             "of this kernel (11.9M events, one set), scaled",
                             "kernel": "mc_spectrum_kernel",
                             "peak_note": "measured copy bandwidth (hbm_gbs)"}
        out[f"sets_{B}"] = r
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        m = min(n, 2_000_000)
        sub = synth.McEvents(energy=ev.energy[:m], core=ev.core[:m], weight=ev.weight[:m],
                             bin=ev.bin[:m], n_bins=ev.n_bins, core_L=ev.core_L,
                             osc_mode=ev.osc_mode, osc_nominal=ev.osc_nominal)
        t0 = time.perf_counter()
        oracle.event_spectrum(sub, ev.osc_nominal)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": m / dt, "unit": "events/s", "cores": 1, "kind": "oracle",
                               "sample": f"first {m} events, one parameter set, FP64"}
    mc.close()
    return out


def profile_measurement(args, pg, world):
    """Profile likelihood (Eq. 7): a 32 x 32 raster of constrained fits of the three-dataset
    model in (sin^2 2th13, dm2_ee) on the first pseudo-experiment, one launch, with its 1-D
    Wilks interval and goodness of fit; and the mass-ordering profiles of the 53 km model
    (dm2_31 > 0 and < 0: Eq. 10 with +phi and -phi) on its normal-ordering Asimov data."""
    import torch
    from paper_2502_15253_gb300 import fitcore, synth

    w = make_workload("c1", 1, args.seed, 0)
    spec, model = w.specs[0], w.models[0]
    D = spec.n_bins
    data = np.ascontiguousarray(w.data[:D])
    mask = spec.all_mask()
    i13, idm = spec.index("sin2_2th13"), spec.index("dm2_ee")
    a = np.linspace(0.05, 0.13, 32)
    b = np.linspace(2.3e-3, 2.7e-3, 32)
    pts = np.array([[x, y] for x in a for y in b])
    fitcore.fit_profile_scan(model, data, mask, [i13, idm], pts[:16])   # warm-up
    barrier(pg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fitcore.fit_profile_scan(model, data, mask, [i13, idm], pts)
    dt = max_over_ranks(time.perf_counter() - t0, pg)
    g1 = np.linspace(0.0, 0.2, 81)
    r1 = fitcore.fit_profile_scan(model, data, mask, [i13], g1)
    lo, hi, op = fitcore.fit_wilks_interval(g1, r1["dchi2"], 1.0)
    # goodness of fit: chi^2 with (bins - free parameters without any prior) degrees of freedom
    in_block = np.zeros(spec.n_params, bool)
    for ix, _ in spec.cov_blocks:
        in_block[np.asarray(ix)] = True
    dof = D - int(np.sum((spec.prior_sigma == 0) & ~in_block))
    out = {"raster": "32 x 32 in sin^2 2th13 [0.05, 0.13] x dm2_ee [2.3e-3, 2.7e-3], plus the "
                     "unconstrained fit, one launch",
           "fits": len(pts) + 1, "s": dt, "raster_points_per_s": world * len(pts) / dt,
           "converged_frac": float(np.mean(r["status"] == 0)),
           "wilks_1sigma_sin2_2th13": [lo, hi], "wilks_open": int(op),
           "gof_p": fitcore.fit_chi2_sf(r1["nll_min"], dof), "gof_dof": dof}
    spec2 = synth.make_model("c2")
    m2 = fitcore.Model(spec2)
    asimov, _ = fitcore.expected_numpy(m2, spec2.theta0[None, :])
    i31 = spec2.index("dm2_31")
    no = np.linspace(2.44e-3, 2.56e-3, 25)
    io = -np.linspace(2.40e-3, 2.52e-3, 25)
    st_io = spec2.theta0.copy()
    st_io[i31] = io[12]
    # warm-up (builds the model's preconditioner once, outside the timing)
    fitcore.fit_profile_scan(m2, asimov[0], spec2.all_mask(), [i31], no[:2])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r_no = fitcore.fit_profile_scan(m2, asimov[0], spec2.all_mask(), [i31], no)
    r_io = fitcore.fit_profile_scan(m2, asimov[0], spec2.all_mask(), [i31], io, start=st_io)
    dt2 = max_over_ranks(time.perf_counter() - t0, pg)
    nll0 = min(r_no["nll_min"], r_io["nll_min"])
    d_no = r_no["dchi2"] + r_no["nll_min"] - nll0
    d_io = r_io["dchi2"] + r_io["nll_min"] - nll0

    def ee(th):   # Eq. 2, magnitudes
        s12 = th[spec2.index("sin2_th12")]
        d21, d31 = th[spec2.index("dm2_21")], th[i31]
        return (1 - s12) * abs(d31) + s12 * abs(d31 - d21)

    k_no, k_io = int(np.argmin(d_no)), int(np.argmin(d_io))
    out["mass_ordering"] = {
        "model": "53 km ten-core far + near detector, Asimov data of the normal ordering",
        "points": len(no) + len(io), "s": dt2,
        "dchi2_inverted_min": float(d_io[k_io]),
        "best_dm2_ee_normal": ee(r_no["theta"][k_no]), "best_dm2_ee_inverted": ee(r_io["theta"][k_io]),
        "converged_frac": float(np.mean(np.concatenate([r_no["status"], r_io["status"]]) == 0))}

    # 3+1 raster ("Sterile neutrino searches"): sin^2 2th14 x dm2_41 over the paper's mass
    # range on null-hypothesis Asimov data of the three-dataset model; Wilks' 95 % level for
    # two parameters (5.99) gives the excluded region
    spec3 = synth.make_model("c1s")
    m3 = fitcore.Model(spec3)
    null, _ = fitcore.expected_numpy(m3, spec3.theta0[None, :])
    i14, i41 = spec3.index("sin2_2th14"), spec3.index("dm2_41")
    s14 = np.linspace(0.0, 0.2, 21)
    dm41 = np.geomspace(5e-4, 0.5, 31)
    pts3 = np.array([[a, b] for a in s14 for b in dm41])
    fitcore.fit_profile_scan(m3, null[0], spec3.all_mask(), [i14, i41], pts3[:2])   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r3 = fitcore.fit_profile_scan(m3, null[0], spec3.all_mask(), [i14, i41], pts3)
    dt3 = max_over_ranks(time.perf_counter() - t0, pg)
    d3 = r3["dchi2"].reshape(len(s14), len(dm41))
    excl = d3 > 5.99
    limit = [float(s14[np.argmax(excl[:, j])]) if excl[:, j].any() else None for j in range(len(dm41))]
    out["sterile_raster"] = {
        "model": "three-dataset model with the exact 3+1 survival, null Asimov data",
        "raster": "21 sin^2 2th14 in [0, 0.2] x 31 dm2_41 log-spaced in [5e-4, 0.5] eV^2",
        "fits": len(pts3) + 1, "s": dt3, "raster_points_per_s": world * len(pts3) / dt3,
        "converged_frac": float(np.mean(r3["status"] == 0)),
        "stalled_frac": float(np.mean(r3["status"] == 7)),
        "excluded_95cl_frac": float(excl.mean()),
        "sin2_2th14_limit_at_dm2_41": {f"{dm41[j]:.3g}": limit[j] for j in (0, 10, 15, 20, 30)}}
    return out


def spline_measurement(args, stream, flush, pg, world):
    """The three-dataset fits with the area-conserving spline energy correction (the paper's
    smoother remap) instead of the overlap rule: same pseudo-experiment recipe and timing."""
    import torch
    from paper_2502_15253_gb300 import fitcore

    B = args.batch
    w = make_workload("c1", B, args.seed, 0, remap=1)
    model, inst = w.models[0], w.inst
    dev = torch.device("cuda", torch.cuda.current_device())
    data_d = torch.from_numpy(w.data).to(dev)
    best_d = torch.zeros(w.par_len, dtype=torch.float64, device=dev)
    res_d = torch.zeros(B * fitcore.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    opts = fitcore.fit_batch_default_opts()
    for _ in range(max(1, args.warmup)):
        fitcore.fit_batch([model], inst, data_d, None, best_d, res_d, opts, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for i in range(max(1, args.steps)):
        flush.fill_(float(i))
        barrier(pg)
        e0.record(stream)
        fitcore.fit_batch([model], inst, data_d, None, best_d, res_d, opts, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = max_over_ranks(float(np.mean(ms)), pg)
    res = np.frombuffer(res_d.cpu().numpy().tobytes(), dtype=fitcore.RESULT_DTYPE)
    return {"note": "energy correction by the area-conserving spline (C1 in a0, a1, a2) instead "
                    "of fractional bin overlap; same recipe, 8192 pseudo-experiments",
            "fits_per_s": world * B / (t / 1e3), "ms_per_step": t,
            "iters_per_fit": float(res["iters"].mean()), "evals_per_fit": float(res["n_evals"].mean()),
            "converged_frac": float(np.mean(res["status"] == 0))}


def run_ours(args):
    import torch
    from paper_2502_15253_gb300 import fitcore

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    B = args.batch
    w = make_workload(args.workload, B, args.seed, rank)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    data_d = torch.from_numpy(w.data).to(dev)
    best_d = torch.zeros(w.par_len, dtype=torch.float64, device=dev)
    res_d = torch.zeros(B * fitcore.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    opts = fitcore.fit_batch_default_opts()
    opts.engine = {"persistent": 0, "lockstep": 1, "lockstep_tc": 2}[args.engine]
    opts.precondition = 0 if args.no_precondition else 1
    tuned = None
    if opts.engine == 0 and not args.no_autotune:
        # launch shape picked by the library's autotuner on a sample of the workload (outside
        # the timing, like the models' one-time set-up), then launched through a CUDA graph
        # (timed on the whole workload: on an uneven mix a sample's tail is not the batch's)
        opts = fitcore.fit_batch_autotune(w.models, w.inst, data_d, None, len(w), opts, stream)
        opts.use_graph = 1
        tuned = {"threads": int(opts.threads), "blocks_per_sm": int(opts.blocks_per_sm),
                 "cuda_graph": True, "tuned_on": f"all {len(w)} instances"}

    def step():
        fitcore.fit_batch(w.models, w.inst, data_d, None, best_d, res_d, opts, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    fitcore.fit_kernel_launches()

    clocks = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ
                          else local)
    clocks.start()
    barrier(pg)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))                       # evict L2 before every timed step
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    wall = time.perf_counter() - wall0
    launches = fitcore.fit_kernel_launches()
    ms_steps = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(float(np.mean(ms_steps)), pg)
    clk = clocks.stop()

    res = np.frombuffer(res_d.cpu().numpy().tobytes(), dtype=fitcore.RESULT_DTYPE)
    evals = int(res["n_evals"].sum())
    iters = int(res["iters"].sum())
    conv = float(np.mean(res["status"] == 0))
    fits_per_s = world * B / (ms / 1e3)
    evals_per_s = world * evals / (ms / 1e3)
    per_model = {}
    for k, nm in enumerate(w.names):
        ix = w.group[k]
        if len(ix):
            per_model[nm] = {"n": int(len(ix)), "params": w.specs[k].n_params,
                             "iters_per_fit": float(res["iters"][ix].mean()),
                             "evals_per_fit": float(res["n_evals"][ix].mean()),
                             "converged_frac": float(np.mean(res["status"][ix] == 0))}
    if w.kind == "c3":
        ix = w.group[0]
        per_model["c1"]["dataset_subsets"] = {
            nm: int(np.sum(w.inst["mask"][ix] == m)) for nm, m in
            (("FD-I", 0b001), ("FD-II+ND", 0b110), ("all", 0b111))}

    # roofline of the fit kernel. Bytes: the L-BFGS state a minimiser iteration reads and
    # writes (2 m P floats of history read with m = 10, 2 P floats written) per instance.
    peaks = read_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    alg_bytes = 0.0
    alg_flops = 0.0
    for k, sp in enumerate(w.specs):
        ix = w.group[k]
        P = sp.n_params
        alg_bytes += float(res["iters"][ix].sum()) * (2 * 10 * P * 4 + 2 * P * 4)
        for i in ix:
            f_eval = flops_per_eval(sp, int(w.inst["mask"][i]))
            if opts.precondition:
                f_eval += 8.0 * P * min(32, sp.n_bins, P)
            alg_flops += res["n_evals"][i] * f_eval + res["iters"][i] * flops_lbfgs_iter(P, opts.history)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = sm_count * 128 * 2 * sm_max * 1e6 / 1e12
    gbs = alg_bytes / (ms / 1e3) / 1e9
    tflops = alg_flops / (ms / 1e3) / 1e12
    traffic = FIT_DRAM_BYTES_PER_FIT.get(w.kind)

    # end-to-end through the public API with host buffers (pinned), copies inside the timing;
    # the one-time set-up (models created from their descriptions, the first fit_batch call
    # building each model's preconditioner) is timed once and reported beside it
    data_pin = torch.from_numpy(w.data).pin_memory()
    best_pin = torch.zeros(w.par_len, dtype=torch.float64).pin_memory()
    res_pin = torch.zeros(B * fitcore.RESULT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    torch.cuda.synchronize()
    barrier(pg)
    t0 = time.perf_counter()
    fresh = [fitcore.Model(sp) for sp in w.specs]
    fitcore.fit_batch(fresh, w.inst, data_pin, None, best_pin, res_pin, opts, stream)
    first_s = max_over_ranks(time.perf_counter() - t0, pg)
    e2e_t = []
    for i in range(max(1, min(args.steps, 3))):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        barrier(pg)
        t0 = time.perf_counter()
        fitcore.fit_batch(fresh, w.inst, data_pin, None, best_pin, res_pin, opts, stream)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(float(np.mean(e2e_t)), pg)
    for m in fresh:
        m.close()
    h2d = w.data.nbytes + w.inst.nbytes
    d2h = best_pin.numel() * 8 + res_pin.numel()

    ws = None
    if not args.no_warm_start and w.kind in ("c3", "c1", "c2"):
        ws = warm_start_measurement(args, w, data_d, res, best_d, opts, stream, flush, pg, world)

    per_cfg = None
    if not args.no_per_config:
        per_cfg = per_config_measurement(args, stream, flush, pg, world, rank)

    spl = None
    if not args.no_profile:
        spl = spline_measurement(args, stream, flush, pg, world)

    prof = None
    if not args.no_profile:
        prof = profile_measurement(args, pg, world)

    mc = None
    if args.mc_events > 0:
        mc = event_reweighting_measurement(args, stream, pg, world)

    out = None
    if rank == 0:
        cpu = None
        frac_ok = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = certify(cpu_baseline(w, min(args.cpu_sample, B)), w, best_d.cpu().numpy(),
                          res["nll_min"])
            frac_ok = cpu["parity_frac_within_1e-3"]
        value = fits_per_s * frac_ok if frac_ok is not None else fits_per_s
        cfg = config_of(args, world, B)
        cfg.update({"engine": args.engine, "launch": tuned,
                    "minimiser": "L-BFGS (32 pairs)" + (", Fisher-preconditioned coordinates"
                                                       if opts.precondition else "")})
        out = {
            "metric": METRIC, "value": value, "unit": "fits/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": cfg, "fits_per_step": world * B,
            "value_note": ("fits/s x the fraction of the oracle-checked sample within 1e-3 of "
                           "the oracle's -2lnL_min" if frac_ok is not None else
                           "all fits/s (no oracle sample in this run)"),
            "fits_per_s_all": fits_per_s, "frac_within_1e-3": frac_ok,
            "evals_per_s": evals_per_s, "iters_per_fit": iters / B, "evals_per_fit": evals / B,
            "converged_frac": conv, "per_model": per_model,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": gbs / hbm_peak,
                         "traffic": traffic["per_fit"] * B if traffic else None,
                         "traffic_note": traffic["note"] if traffic else
                         "no ncu capture of the current kernel on this workload",
                         "kernel": "fit_kernel",
                         "algorithmic": "L-BFGS state per minimiser iteration and instance: "
                                        "2 m P floats read (m = 10) + 2 P floats written",
                         "peak_note": "measured copy bandwidth (hbm_gbs)",
                         "alu_model": {"achieved": tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                                       "frac": tflops / peak_tflops,
                                       "peak_note": f"FP32 FMA: {sm_count} SMs x 128 lanes x 2 x "
                                                    f"{sm_max:.0f} MHz"}},
            "e2e": {"value": world * B / e2e_s, "unit": "fits/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "setup_s": max(0.0, first_s - e2e_s),
                    "setup_note": "one-time: models created from their descriptions and each "
                                  "model's preconditioner built (first fit_batch call minus a "
                                  "plain call)",
                    "value_incl_setup_one_step": world * B / first_s},
            "gpu_launches": int(launches // max(1, args.steps)) * args.steps,
            "clocks": clk, "wall_s": wall,
            "cpu_baseline": cpu,
            "per_config": per_cfg,
            "warm_start": ws,
            "profile_likelihood": prof,
            "spline_energy_correction": spl,
            "event_reweighting": mc,
        }
        print(json.dumps(out))
    if pg is not None:
        pg.destroy_process_group()
    return out


def run_reference(args):
    """Reference arm: the FP64 oracle (dense BFGS, OpenMP over instances) timed on the host cores
    on the same workload; each step fits a bounded sample (the first --ref-sample instances of
    the same seeded table) from the same cold start."""
    world, rank, _, pg = dist_setup(args)
    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return
    import oracle
    n = max(4, args.ref_sample)
    w = make_workload_oracle(args.workload, n, args.seed)
    threads = os.cpu_count() or 1
    ds = [w.data_of(i).astype(np.float64) for i in range(n)]
    geo = [int(g) for g in w.geo]
    masks = [int(m) for m in w.inst["mask"]]
    starts = [w.specs[g].theta0 for g in geo]
    for _ in range(args.warmup):
        oracle.fit_many(w.oms, geo[:2], ds[:2], masks[:2], starts[:2], n_threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.fit_many(w.oms, geo, ds, masks, starts, n_threads=threads)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    val = n / (ms / 1e3)
    cores = threads if oracle.openmp_enabled() else 1
    cfg = config_of(args, 1, args.batch)
    cnt = {nm: int(np.sum(w.geo == k)) for k, nm in enumerate(w.names)}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "fits/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg, "fits_per_step": n,
        "cpu_baseline": {"value": val, "unit": "fits/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {n} instances of the workload per step "
                                   f"({', '.join(f'{v} {k}' for k, v in cnt.items())}) on "
                                   f"{cores} host threads"},
        "e2e": {"value": val, "unit": "fits/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    if pg is not None:
        pg.destroy_process_group()


def time_fit_steps(w, data_d, best_d, res_d, opts, stream, flush, warmup, steps, pg):
    """Mean device time (ms, max over ranks) of fit_batch over the whole workload."""
    import torch
    from paper_2502_15253_gb300 import fitcore
    for _ in range(warmup):
        fitcore.fit_batch(w.models, w.inst, data_d, None, best_d, res_d, opts, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for i in range(steps):
        flush.fill_(float(i))
        barrier(pg)
        e0.record(stream)
        fitcore.fit_batch(w.models, w.inst, data_d, None, best_d, res_d, opts, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return max_over_ranks(float(np.mean(ms)), pg)


# oracle samples of the per-model lines (about 2-6 s each on 16 Grace cores)
PER_CONFIG_ORACLE_SAMPLE = {"c0": 256, "c1": 256, "c2": 48}


def per_config_measurement(args, stream, flush, pg, world, rank):
    """Each model alone: fits/s of args.batch cold-start fits (one fit_batch call), evaluations
    (-2lnL + gradient) per second of fit_model_eval on args.batch parameter vectors, and the
    oracle's all-core fits/s, one-core evaluations/s and parity on a bounded sample."""
    import torch
    from paper_2502_15253_gb300 import fitcore
    import oracle
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {}
    for kind in ("c0", "c1", "c2"):
        B = args.batch
        w = make_workload(kind, B, args.seed, rank)
        sp, model = w.specs[0], w.models[0]
        data_d = torch.from_numpy(w.data).to(dev)
        best_d = torch.zeros(w.par_len, dtype=torch.float64, device=dev)
        res_d = torch.zeros(B * fitcore.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        opts = fitcore.fit_batch_default_opts()
        if not args.no_autotune:
            opts = fitcore.fit_batch_autotune(w.models, w.inst, data_d, None, len(w), opts, stream)
            opts.use_graph = 1
        ms = time_fit_steps(w, data_d, best_d, res_d, opts, stream, flush, 2, 3, pg)
        res = np.frombuffer(res_d.cpu().numpy().tobytes(), dtype=fitcore.RESULT_DTYPE)
        # evaluations of the truth points against their own pseudo-data
        th = torch.from_numpy(w.truth).to(dev).view(B, sp.n_params)
        dv = data_d.view(B, sp.n_bins)
        nll = torch.zeros(B, dtype=torch.float64, device=dev)
        grad = torch.zeros((B, sp.n_params), dtype=torch.float32, device=dev)
        for _ in range(3):
            fitcore.fit_model_eval(model, B, th, dv, None, nll, grad, None, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        flush.fill_(1.0)
        barrier(pg)
        e0.record(stream)
        for _ in range(reps):
            fitcore.fit_model_eval(model, B, th, dv, None, nll, grad, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(e0.elapsed_time(e1) / reps, pg)
        # the same roofline models as the headline line: L-BFGS state bytes per iteration
        # against the copy bandwidth, the FP32 work model against the FMA peak
        peaks = read_peaks()
        hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        alu_peak = sm_count * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
        P = sp.n_params
        f_eval = flops_per_eval(sp, sp.all_mask()) + 8.0 * P * min(32, sp.n_bins, P)
        fit_bytes = float(res["iters"].sum()) * (2 * 10 * P * 4 + 2 * P * 4)
        fit_flops = float(res["n_evals"].sum()) * f_eval + float(res["iters"].sum()) * flops_lbfgs_iter(P, 32)
        r = {"workload": WORKLOADS[kind], "fits": world * B,
             "fits_per_s": world * B / (ms / 1e3), "ms_per_step": ms,
             "fit_roofline": {"hbm_frac": fit_bytes / (ms / 1e3) / 1e9 / hbm_peak,
                              "alu_frac": fit_flops / (ms / 1e3) / 1e12 / alu_peak},
             "eval_alu_frac": flops_per_eval(sp, sp.all_mask()) * B / (ems / 1e3) / 1e12 / alu_peak,
             "iters_per_fit": float(res["iters"].mean()), "evals_per_fit": float(res["n_evals"].mean()),
             "converged_frac": float(np.mean(res["status"] == 0)),
             "eval_grad_per_s": world * B / (ems / 1e3), "eval_batch": B, "eval_ms": ems}
        if kind == "c2":
            # the same fits on engine 2, whose rounds fold the spectra of all active fits on the
            # tensor cores (split-TF32 GEMMs F = V R^T, G R); minima compared with the default's
            o2 = fitcore.fit_batch_default_opts()
            o2.engine = 2
            best2 = torch.zeros_like(best_d)
            res2_d = torch.zeros_like(res_d)
            ms2 = time_fit_steps(w, data_d, best2, res2_d, o2, stream, flush, 1, 2, pg)
            res2 = np.frombuffer(res2_d.cpu().numpy().tobytes(), dtype=fitcore.RESULT_DTYPE)
            r["engine2_tensor_core_fold"] = {
                "note": "lockstep rounds over all active fits with the response fold and its adjoint as "
                        "split-TF32 tcgen05 GEMMs (tensor pipe share of its device time in "
                        "profiles/lockstep_tc_c2_fits.md)",
                "fits_per_s": world * B / (ms2 / 1e3), "ms_per_step": ms2,
                "evals_per_fit": float(res2["n_evals"].mean()),
                "same_minimum_as_default_frac": float(np.mean(np.abs(res2["nll_min"] - res["nll_min"]) <= 1e-3)),
                "converged_frac": float(np.mean(res2["status"] == 0))}
            del best2, res2_d
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            n = min(PER_CONFIG_ORACLE_SAMPLE[kind], B)
            cpu = certify(cpu_baseline(w, n), w, best_d.cpu().numpy(), res["nll_min"])
            om = oracle.OracleModel(sp)
            k = 0
            t0 = time.perf_counter()
            while k < 200 and (k < 3 or time.perf_counter() - t0 < 1.0):
                om.nll(w.truth[k % B * sp.n_params:(k % B + 1) * sp.n_params],
                       w.data_of(k % B).astype(np.float64), grad=True)
                k += 1
            cpu["oracle_eval_grad_per_s_1core"] = k / (time.perf_counter() - t0)
            r["cpu_baseline"] = cpu
        out[kind] = r
        del data_d, best_d, res_d, th, nll, grad
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
