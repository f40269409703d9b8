"""Benchmark: batched cold-start fits of the two-detector, three-dataset model (FD-I, FD-II, ND;
291 parameters), fits/s on one or more GPUs.

One step = one fit_batch() call that fits B Poisson pseudo-experiments from the nominal start:
every evaluation of the expectation, -2lnL, adjoint gradient and every L-BFGS update runs in
the persistent fit kernel. Inputs are resident in device memory when the timed region starts;
L2 is flushed (a 512 MiB write) before every timed step. With torchrun, each rank fits its own
B instances (weak scaling, no collective on the data path); the step time is the maximum over
ranks and value = total fits / that time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--impl ours|reference]
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
WORKLOAD = "two-detector three-dataset fit (FD-I, FD-II, ND), 291 params, 400 true / 3x38 reco bins"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--batch", type=int, default=8192, help="fits per rank per step")
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--cpu-sample", type=int, default=2560,
                   help="instances of the CPU baseline (about 10 s of the FP64 oracle on 16 cores)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--seed", type=int, default=250215253)
    p.add_argument("--engine", default="persistent", choices=["persistent", "lockstep"],
                   help="fit engine: one persistent launch, or one round of launches per evaluation")
    p.add_argument("--mc-events", type=int, default=20_000_000,
                   help="simulated events of the event-reweighting measurement (0: skip)")
    p.add_argument("--no-precondition", action="store_true",
                   help="fit in plain whitened coordinates (no Fisher preconditioner)")
    p.add_argument("--no-profile", action="store_true",
                   help="skip the profile-likelihood and mass-ordering scans")
    p.add_argument("--no-warm-start", action="store_true",
                   help="skip the warm-start network measurement")
    p.add_argument("--ws-samples", type=int, default=2_000_000,
                   help="training samples of the warm-start network (both geometries)")
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
def make_workload(B, seed, rank, remap=0):
    """B pseudo-experiments of the C1 model: true (sin^2 2th13, dm2_ee) drawn within +-3 sigma,
    expectation from the library, Poisson counts from numpy's PCG64 (seeded per instance).
    remap=1: the same model with the area-conserving spline energy correction."""
    from paper_2502_15253_gb300 import fitcore, synth
    spec = synth.make_model("c1", remap=remap)
    model = fitcore.Model(spec)
    rng = np.random.default_rng(seed + 7919 * rank)
    truths = np.stack([synth.draw_theta_true(spec, rng) for _ in range(B)])
    mu, st = fitcore.expected_numpy(model, truths)
    assert np.all(st == 0)
    data = np.random.default_rng(seed + 1 + 7919 * rank).poisson(mu.astype(np.float64))
    data = data.astype(np.float32)
    inst = np.zeros(B, fitcore.INSTANCE_DTYPE)
    inst["model"] = 0
    inst["mask"] = spec.all_mask()
    inst["data_off"] = np.arange(B, dtype=np.int64) * spec.n_bins
    inst["param_off"] = np.arange(B, dtype=np.int64) * spec.n_params
    return spec, model, data, inst


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


def cpu_baseline(spec, data, inst, n, threads=None):
    """The FP64 oracle (dense BFGS) on the host cores, on the first n instances."""
    import oracle
    om = oracle.OracleModel(spec)
    threads = threads or os.cpu_count() or 1
    P, D = spec.n_params, spec.n_bins
    flat = np.asarray(data).reshape(-1)
    ds = [flat[i * D:(i + 1) * D].astype(np.float64) for i in range(n)]
    starts = [spec.theta0] * n
    t0 = time.perf_counter()
    r = oracle.fit_many([om], [0] * n, ds, [int(inst["mask"][i]) for i in range(n)], starts,
                        edm_tol=1e-10, n_threads=threads)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "fits/s", "cores": threads if oracle.openmp_enabled() else 1,
            "kind": "oracle", "sample": f"{n} instances of the same workload, cold start, "
            f"FP64 dense BFGS (EDM < 1e-10), {dt:.1f} s", "nll": r["nll"], "iters": r["iters"],
            "status": r["status"], "om": om, "data": ds}


def certify_other_minima(cpu, gpu_best, gpu_nll, P):
    """Instances whose GPU minimum is not the oracle's: is the GPU point an oracle minimum?
    (the oracle restarted there stays within 1e-4 in -2lnL)"""
    om, ds = cpu.pop("om"), cpu.pop("data")
    cpu_nll = cpu.pop("nll")
    cpu.pop("iters")
    cpu.pop("status")
    d = np.abs(gpu_nll[:len(cpu_nll)] - cpu_nll)
    other = np.flatnonzero(d > 1e-3)
    cert = 0
    for i in other:
        th = gpu_best[i * P:(i + 1) * P]
        r = om.fit(ds[i], start=th)
        cert += int(r["status"] == 0 and abs(r["nll"] - om.nll(th, ds[i])) <= 1e-4)
    cpu["parity_max_abs_dnll"] = float(d.max())
    cpu["parity_frac_within_1e-3"] = float(np.mean(d <= 1e-3))
    cpu["parity_other_minima"] = int(len(other))
    cpu["parity_other_minima_certified"] = int(cert)


def mlp_flops_per_sample(dims, train):
    """Multiply-adds x 2 of the network's products per sample: forward; training adds the
    weight gradients (same count) and the input gradients of every layer but the first."""
    fwd = [2 * i * o for i, o in zip(dims[:-1], dims[1:])]
    return sum(fwd) * 2 + sum(fwd[1:]) if train else sum(fwd)


def warm_start_measurement(args, spec, model, inst, data_d, cold_res, cold_best, opts, stream,
                           flush, pg, world):
    """Warm start (not in the paper): train the network on device-drawn samples of both
    geometries, time one bf16 training step on the tensor cores, the TF32 fold of a training
    batch, and fits of the benchmark's pseudo-experiments from the predicted starts."""
    import torch
    from paper_2502_15253_gb300 import fitcore, synth, warmstart

    dev = data_d.device
    B, P = len(inst), spec.n_params
    spec2 = synth.make_model("c2")
    model2 = fitcore.Model(spec2)
    net = warmstart.network(seed=3)
    batch = 4096
    n_steps = max(2, args.ws_samples // batch)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    losses = warmstart.train(net, [model, model2], [spec, spec2], n_steps=n_steps, batch=batch,
                             lr=1e-3, stream=stream)
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
    peaks = {}
    peak_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peak_path):
        peaks = json.load(open(peak_path))
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    mlp_tflops = mlp_flops_per_sample(dims, True) * tb / (step_ms / 1e3) / 1e12

    # TF32 fold of a 53 km training batch: V [B x 2000] times R^T for both detectors
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

    # warm fits of the benchmark's pseudo-experiments
    starts = torch.zeros((B, P), dtype=torch.float64, device=dev)
    flush.fill_(0.5)
    ev0.record(stream)
    warmstart.predict_starts(net, model, spec, B, data_d.view(B, -1), None, starts, stream)
    best_w = torch.zeros_like(cold_best)
    res_w = torch.zeros(B * fitcore.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    fitcore.fit_batch([model], inst, data_d, starts.view(-1), best_w, res_w, opts, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    warm_ms = max_over_ranks(ev0.elapsed_time(ev1), pg)
    rw = np.frombuffer(res_w.cpu().numpy().tobytes(), dtype=fitcore.RESULT_DTYPE)
    same = np.abs(rw["nll_min"] - cold_res["nll_min"]) <= 1e-3
    return {
        "note": "not in the paper: a network proposes start points; every fit still runs to "
                "the same EDM tolerance",
        "train_samples": n_steps * batch, "train_s": train_s,
        "train_samples_per_s": n_steps * batch / train_s,
        "train_loss_first_last": [float(losses[:2].mean()), float(losses[-20:].mean())],
        "mlp_train_step": {"batch": tb, "ms": step_ms, "achieved": mlp_tflops,
                           "unit": "TFLOP/s", "peak": bf16_peak, "frac": mlp_tflops / bf16_peak,
                           "bound": "tensor", "dtype": "bf16",
                           "flops_per_sample": mlp_flops_per_sample(dims, True)},
        "fold_tf32_53km": {"batch": fb, "ms": fold_ms, "achieved": fold_flops / fold_ms / 1e9,
                           "unit": "TFLOP/s", "peak": tf32_peak,
                           "frac": fold_flops / fold_ms / 1e9 / tf32_peak,
                           "peak_note": "measured bf16 burst x 1.1/2.25 (nominal tf32/bf16)",
                           "timed": "whole fit_model_expected_tc call (spectra, GEMMs, epilogue); "
                                    "the spectra kernel (survival at 2000 bins x 10 cores per "
                                    "instance and detector) dominates"},
        "fold_gemm_tf32_alone": {"M": fb, "N": 400, "K": n_t, "ms": gemm_ms, "achieved": gemm_tflops,
                                 "unit": "TFLOP/s", "peak": tf32_peak, "frac": gemm_tflops / tf32_peak,
                                 "bound": "tensor", "kernel": "tc_gemm_kernel<TF32>"},
        "fits_per_s_warm": world * B / (warm_ms / 1e3),
        "warm_ms_incl_inference": warm_ms,
        "iters_per_fit_warm": float(rw["iters"].mean()),
        "iters_per_fit_cold": float(cold_res["iters"].mean()),
        "same_minimum_as_cold_frac": float(same.mean()),
        "converged_frac_warm": float(np.mean(rw["status"] == 0)),
    }


# DRAM bytes (read + write) per fit of fit_kernel on the three-dataset model, from an ncu
# capture of one 760-fit launch of the preconditioned build (the default; 4.39 MB read,
# 14.58 MB written, mostly the workspace write-back); traffic grows with the fits. The plain
# build's capture (7.30 MB, 47.86 MB) predates later changes of the kernel, so a run with
# --no-precondition reports no traffic.
FIT_DRAM_BYTES_PER_FIT = (4.394240e6 + 14.576896e6) / 760

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


def profile_measurement(args, spec, model, data_h, pg, world):
    """Profile likelihood (Eq. 7): a 32 x 32 raster of constrained fits of the three-dataset
    model in (sin^2 2th13, dm2_ee) on the first pseudo-experiment, one launch, with its 1-D
    Wilks interval and goodness of fit; and the mass-ordering profiles of the 53 km model
    (dm2_31 > 0 and < 0: Eq. 10 with +phi and -phi) on its normal-ordering Asimov data."""
    import torch
    from paper_2502_15253_gb300 import fitcore, synth

    D = spec.n_bins
    data = np.ascontiguousarray(data_h[:D])
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
    spec, model, data_h, inst = make_workload(B, args.seed, 0, remap=1)
    dev = torch.device("cuda", torch.cuda.current_device())
    data_d = torch.from_numpy(data_h).to(dev)
    best_d = torch.zeros(B * spec.n_params, dtype=torch.float64, device=dev)
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


def run_reference(args):
    """Reference arm: the FP64 oracle timed on the host cores on the same workload."""
    world, rank, _, pg = dist_setup(args)
    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return
    from paper_2502_15253_gb300 import synth
    import oracle
    spec = synth.make_model("c1")
    om = oracle.OracleModel(spec)
    rng = np.random.default_rng(args.seed)
    n = max(8, min(args.cpu_sample, 64))
    truths = [synth.draw_theta_true(spec, rng) for _ in range(n)]
    ds = [synth.poisson_data(om.expected(t), args.seed + i) for i, t in enumerate(truths)]
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.fit_many([om], [0] * 2, ds[:2], [spec.all_mask()] * 2, [spec.theta0] * 2,
                        n_threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.fit_many([om], [0] * n, ds, [spec.all_mask()] * n, [spec.theta0] * n,
                        n_threads=threads)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    val = n / (ms / 1e3)
    cores = threads if oracle.openmp_enabled() else 1
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "fits/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "fits_per_step": n, "start": "nominal (cold)"},
        "cpu_baseline": {"value": val, "unit": "fits/s", "cores": cores, "kind": "oracle",
                         "sample": f"{n} instances per step on {cores} host threads"},
        "e2e": {"value": val, "unit": "fits/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    if pg is not None:
        pg.destroy_process_group()


def run_ours(args):
    import torch
    from paper_2502_15253_gb300 import fitcore

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    B = args.batch
    spec, model, data_h, inst = make_workload(B, args.seed, rank)
    P, D = spec.n_params, spec.n_bins
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    data_d = torch.from_numpy(data_h).to(dev)
    best_d = torch.zeros(B * P, dtype=torch.float64, device=dev)
    res_d = torch.zeros(B * fitcore.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    opts = fitcore.fit_batch_default_opts()
    opts.engine = 1 if args.engine == "lockstep" else 0
    opts.precondition = 0 if args.no_precondition else 1

    def step():
        fitcore.fit_batch([model], inst, data_d, None, best_d, res_d, opts, stream)

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
    value = world * B / (ms / 1e3)
    evals_per_s = world * evals / (ms / 1e3)

    # roofline of the fit kernel: FP32 ALU peak from unit counts and the maximum SM clock;
    # with the Fisher preconditioner each evaluation also applies T twice (Q^T x and Q u:
    # 2 P r multiply-adds each, r = min(32, bins, P))
    f_eval = flops_per_eval(spec, spec.all_mask())
    if opts.precondition:
        f_eval += 8.0 * P * min(32, D, P)
    alg_flops = evals * f_eval + iters * flops_lbfgs_iter(P, opts.history)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    sm_max = 2070.0
    if os.path.exists(peak_path):
        try:
            sm_max = float(json.load(open(peak_path)).get("sm_max_mhz", sm_max))
        except Exception:
            pass
    peak_tflops = sm_count * 128 * 2 * sm_max * 1e6 / 1e12
    achieved = alg_flops / (ms / 1e3) / 1e12

    # end-to-end through the public API with host buffers (pinned), copies inside the timing
    data_pin = torch.from_numpy(data_h).pin_memory()
    best_pin = torch.zeros(B * P, dtype=torch.float64).pin_memory()
    res_pin = torch.zeros(B * fitcore.RESULT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    fitcore.fit_batch([model], inst, data_pin, None, best_pin, res_pin, opts, stream)
    barrier(pg)
    e2e_t = []
    for i in range(max(1, min(args.steps, 3))):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fitcore.fit_batch([model], inst, data_pin, None, best_pin, res_pin, opts, stream)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(float(np.mean(e2e_t)), pg)
    h2d = data_h.nbytes + inst.nbytes
    d2h = best_pin.numel() * 8 + res_pin.numel()

    ws = None
    if not args.no_warm_start:
        ws = warm_start_measurement(args, spec, model, inst, data_d, res, best_d, opts, stream,
                                    flush, pg, world)

    spl = None
    if not args.no_profile:
        spl = spline_measurement(args, stream, flush, pg, world)

    prof = None
    if not args.no_profile:
        prof = profile_measurement(args, spec, model, data_h, pg, world)

    mc = None
    if args.mc_events > 0:
        mc = event_reweighting_measurement(args, stream, pg, world)

    out = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(spec, data_h, inst, min(args.cpu_sample, B))
            certify_other_minima(cpu, best_d.cpu().numpy(), res["nll_min"], P)
        out = {
            "metric": METRIC, "value": value, "unit": "fits/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "fits_per_step": world * B, "fits_per_rank": B,
                       "engine": args.engine,
                       "minimiser": "L-BFGS (32 pairs)" + (", Fisher-preconditioned coordinates"
                                                          if opts.precondition else ""),
                       "start": "nominal (cold)", "l2": "flushed (512 MiB write) before each step",
                       "parallelism": f"instances sharded over {world} GPU(s), no collective"},
            "evals_per_s": evals_per_s, "iters_per_fit": iters / B, "evals_per_fit": evals / B,
            "converged_frac": conv,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops,
                         "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                         "traffic": FIT_DRAM_BYTES_PER_FIT * B if opts.precondition else None,
                         "traffic_note": ("DRAM read+write bytes per fit of an ncu capture of "
                                          "this kernel (760 fits), scaled to the launch"
                                          if opts.precondition else
                                          "no capture of the current plain build"),
                         "kernel": "fit_kernel",
                         "peak_note": f"FP32 FMA: {sm_count} SMs x 128 lanes x 2 x {sm_max:.0f} MHz"},
            "e2e": {"value": world * B / e2e_s, "unit": "fits/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches // max(1, args.steps)) * args.steps,
            "clocks": clk, "wall_s": wall,
            "cpu_baseline": cpu,
            "warm_start": ws,
            "profile_likelihood": prof,
            "spline_energy_correction": spl,
            "event_reweighting": mc,
        }
        print(json.dumps(out))
    if pg is not None:
        pg.destroy_process_group()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
