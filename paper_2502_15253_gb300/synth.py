"""Seeded synthetic inputs for the forward-folding likelihood fit.

This module builds the *inputs* of the method and nothing else: energy grids, detector
response matrices, un-oscillated signal spectra, background templates, the parameter table
(nominal values, Gaussian prior widths, minimiser step scales), prior covariance blocks,
ensemble instance tables and Poisson draws around an expectation that the caller supplies.
It evaluates no part of the expectation, the likelihood or its gradient, so both the FP64
oracle and the CUDA library can take their inputs from here without sharing any arithmetic
of the method.

The three geometries follow the paper's two case studies:

* ``c0`` - one detector, one reactor at 1050 m (the Double Chooz far detector, section "Experimental context").
* ``c1`` - the Double Chooz three-dataset layout FD-I, FD-II, ND with two cores, 38 reco bins
  per dataset (Eq. 9) and the nuisance families listed in section "Likelihood
  implementation for Double Chooz within the framework" (flux/shape bins,
  Li-9, accidental and fast-neutron backgrounds, quadratic energy response, efficiencies).
* ``c2`` - the medium-baseline (JUNO-like) study of section "Application to medium
  baseline reactor measurements": a far detector 52-53.5 km from
  ten cores, a near detector at the Double Chooz near baseline, 3 %/sqrt(E) resolution.

Every number the paper does not fix (bin counts, templates, prior widths, event counts) is a
stated synthetic choice; nothing here is taken from the experiments' data.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from math import erf, sqrt

import numpy as np

BASE_SEED = 250215253

# Survival-probability parameterisations understood by both implementations.
OSC_EQ1 = 0        # Eq. 1: (sin^2 2th13, dm2_ee, sin^2 2th12, dm2_21)
OSC_VACUUM3 = 1    # exact 3-flavour vacuum: (sin^2 th12, sin^2 th13, dm2_21, dm2_31); the sign of dm2_31 is the ordering
OSC_STERILE4 = 2   # exact 3+1 vacuum: the four above, then (sin^2 2th14, dm2_41)

PROMPT_SHIFT_MEV = 0.782   # E_vis = E_nu - 0.782 MeV (IBD kinematics, neutron recoil neglected)
RESPONSE_EPS0 = 0.9        # nominal detection efficiency folded into the response
RESPONSE_NSIGMA = 7.0      # response entries of reco bins beyond +-7 sigma are exactly zero


def splitmix64(x: int) -> int:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014), used to derive per-instance seeds."""
    x = (x + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


def instance_seed(i: int, base: int = BASE_SEED) -> int:
    return splitmix64(base + i)


# ----------------------------------------------------------------------------------------
# Model description
# ----------------------------------------------------------------------------------------
@dataclass
class Background:
    name: str
    template: np.ndarray          # [N_r] expected counts at nominal rate and shape
    rate_idx: int                 # parameter index of the rate multiplier, -1 = fixed at 1
    shape_idx: np.ndarray         # [N_r] int32 parameter index of (1 + delta_j), -1 = none


@dataclass
class Detector:
    name: str
    reco_edges: np.ndarray        # [N_r + 1] MeV
    response: np.ndarray          # [N_r, N_t] probability true bin k -> reco bin j (incl. eps0)

    @property
    def n_reco(self) -> int:
        return self.response.shape[0]


@dataclass
class Dataset:
    name: str
    det: int                      # detector index
    t: np.ndarray                 # [N_t] un-oscillated expected signal counts per true bin
    baseline: np.ndarray          # [C] reactor-detector distance per core, m
    weight: np.ndarray            # [C] flux share per core at nominal power (sums to 1)
    norm_idx: int                 # signal normalisation parameter, -1 = fixed at 1
    eff_idx: int                  # detection efficiency parameter, -1 = fixed at 1
    escale_idx: np.ndarray        # [3] int32 indices of (a0, a1, a2); -1 = nominal (0, 1, 0)
    shape_idx: np.ndarray         # [N_t] int32 index of the true-space shape reweight, -1 = none
    backgrounds: list = field(default_factory=list)


@dataclass
class ModelSpec:
    name: str
    param_names: list
    theta0: np.ndarray            # [P] nominal values (prior means)
    prior_sigma: np.ndarray       # [P] Gaussian prior width, 0 = no individual prior
    scale: np.ndarray             # [P] minimiser step scale (the "transformation layer" unit)
    cov_blocks: list              # [(idx int32[m], cov float64[m, m])], prior mean theta0[idx]
    osc_mode: int
    osc_idx: np.ndarray           # [4] ([6] for OSC_STERILE4) int32 parameter index or -1
    osc_val: np.ndarray           # [4] ([6]) value used when osc_idx == -1
    core_power_idx: np.ndarray    # [C] int32 parameter index of each core's power, -1 = fixed 1
    n_true: int
    e_lo: float
    e_hi: float
    detectors: list
    datasets: list
    remap: int = 0                # energy correction: 0 overlap length, 1 area-conserving spline
    # Eq. 6 priors on b = A theta[idx]: [(idx int32[k], A float64[m, k], b0 float64[m],
    # V float64[m, m])]; the measured values b0 with covariance V
    map_priors: list = field(default_factory=list)

    @property
    def n_params(self) -> int:
        return len(self.theta0)

    @property
    def n_cores(self) -> int:
        return len(self.core_power_idx)

    @property
    def true_edges(self) -> np.ndarray:
        return np.linspace(self.e_lo, self.e_hi, self.n_true + 1)

    def reco_sizes(self) -> list:
        return [self.detectors[d.det].n_reco for d in self.datasets]

    @property
    def n_bins(self) -> int:
        """Total number of reco bins over all datasets (length of a data vector)."""
        return int(sum(self.reco_sizes()))

    def data_offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.reco_sizes())]).astype(np.int64)

    def all_mask(self) -> int:
        return (1 << len(self.datasets)) - 1

    def index(self, name: str) -> int:
        return self.param_names.index(name)

    def to_config(self) -> dict:
        """The JSON configuration of this model (the schema fit_model_create_json reads):
        parameters by name, held entries as null, survival constants as numbers."""
        names = list(self.param_names)

        def ref(i):
            return None if int(i) < 0 else names[int(i)]

        def refs(a):
            return [ref(i) for i in np.asarray(a).ravel()]

        def nums(a):
            return [float(x) for x in np.asarray(a, dtype=np.float64).ravel()]

        formula = {OSC_EQ1: "eq1", OSC_VACUUM3: "vacuum3", OSC_STERILE4: "sterile4"}[self.osc_mode]
        return {
            "name": self.name,
            "parameters": [{"name": n, "value": float(v), "sigma": float(s), "scale": float(c)}
                           for n, v, s, c in zip(names, self.theta0, self.prior_sigma, self.scale)],
            "covariances": [{"params": refs(ix), "cov": [nums(r) for r in np.asarray(cv)]}
                            for ix, cv in self.cov_blocks]
                           + [{"params": refs(ix), "map": [nums(r) for r in np.asarray(A)],
                               "mean": nums(b0), "cov": [nums(r) for r in np.asarray(V)]}
                              for ix, A, b0, V in self.map_priors],
            "oscillation": {"formula": formula,
                            "params": [names[int(i)] if int(i) >= 0 else float(v)
                                       for i, v in zip(self.osc_idx, self.osc_val)]},
            "true_grid": {"bins": int(self.n_true), "e_lo": float(self.e_lo), "e_hi": float(self.e_hi)},
            "energy_correction": "spline" if int(self.remap) == 1 else "overlap",
            "core_powers": refs(self.core_power_idx),
            "detectors": [{"name": dt.name, "reco_edges": nums(dt.reco_edges),
                           "response": [nums(r) for r in dt.response]}
                          for dt in self.detectors],
            "datasets": [{"name": x.name, "detector": self.detectors[x.det].name,
                          "t": nums(x.t), "baseline": nums(x.baseline), "weight": nums(x.weight),
                          "norm": ref(x.norm_idx), "efficiency": ref(x.eff_idx),
                          "escale": refs(x.escale_idx), "shape": refs(x.shape_idx),
                          "backgrounds": [{"name": b.name, "template": nums(b.template),
                                           "rate": ref(b.rate_idx), "shape": refs(b.shape_idx)}
                                          for b in x.backgrounds]}
                         for x in self.datasets],
        }

    def to_json(self) -> str:
        import json
        return json.dumps(self.to_config())

    @classmethod
    def from_config(cls, cfg) -> "ModelSpec":
        """The description held by a JSON configuration (a dict or its text) in the schema of
        fit_model_create_json: names resolved (namespaces flattened to "ns.name"), held
        entries as -1. Priors given through a linear map (b = A theta) are kept as they are
        written (map_priors): the map, the measured values and their covariance."""
        import json
        if isinstance(cfg, (str, bytes)):
            cfg = json.loads(cfg)
        names, th0, sig, scl = [], [], [], []

        def add(entries, prefix):
            for e in entries:
                if "namespace" in e:
                    add(e["parameters"], prefix + e["namespace"] + ".")
                    continue
                names.append(prefix + e["name"])
                th0.append(float(e["value"]))
                sig.append(float(e.get("sigma", 0.0)))
                scl.append(float(e.get("scale", 0.0)))

        add(cfg["parameters"], "")
        index = {n: i for i, n in enumerate(names)}
        if len(index) != len(names):
            raise ValueError("duplicate parameter names")

        def ref(v):
            if v is None:
                return -1
            return index[v] if isinstance(v, str) else int(v)

        def refs(vs):
            return np.array([ref(v) for v in vs], np.int32)

        cov_blocks, map_priors = [], []
        for b in cfg.get("covariances", []):
            if "map" in b:
                map_priors.append((refs(b["params"]), np.array(b["map"], np.float64),
                                   np.array(b["mean"], np.float64), np.array(b["cov"], np.float64)))
                continue
            cov_blocks.append((refs(b["params"]), np.array(b["cov"], np.float64)))
        osc = cfg["oscillation"]
        mode = {"eq1": OSC_EQ1, "vacuum3": OSC_VACUUM3, "sterile4": OSC_STERILE4}[osc["formula"]]
        osc_idx = np.array([ref(e) if isinstance(e, str) else -1 for e in osc["params"]], np.int32)
        osc_val = np.array([th0[index[e]] if isinstance(e, str) else float(e) for e in osc["params"]])
        grid = cfg["true_grid"]
        n_true = int(grid["bins"])
        dets, det_index = [], {}
        for k, d in enumerate(cfg["detectors"]):
            resp = np.array(d["response"], np.float64).reshape(-1, n_true)
            edges = np.array(d.get("reco_edges", np.arange(len(resp) + 1)), np.float64)
            dets.append(Detector(d.get("name", f"det{k}"), edges, resp))
            det_index[dets[-1].name] = k
        datasets = []
        for k, d in enumerate(cfg["datasets"]):
            det = det_index[d["detector"]] if isinstance(d["detector"], str) else int(d["detector"])
            nr = dets[det].n_reco
            bkgs = [Background(b.get("name", f"bkg{j}"), np.array(b["template"], np.float64),
                               ref(b.get("rate")), refs(b.get("shape", [None] * nr)))
                    for j, b in enumerate(d.get("backgrounds", []))]
            datasets.append(Dataset(d.get("name", f"ds{k}"), det, np.array(d["t"], np.float64),
                                    np.array(d["baseline"], np.float64),
                                    np.array(d["weight"], np.float64), ref(d.get("norm")),
                                    ref(d.get("efficiency")),
                                    refs(d.get("escale", [None] * 3)),
                                    refs(d.get("shape", [None] * n_true)), bkgs))
        remap = 1 if cfg.get("energy_correction", "overlap") == "spline" else 0
        return cls(cfg.get("name", "config"), names, np.array(th0), np.array(sig), np.array(scl),
                   cov_blocks, mode, osc_idx, osc_val, refs(cfg["core_powers"]), n_true,
                   float(grid["e_lo"]), float(grid["e_hi"]), dets, datasets, remap, map_priors)


# ----------------------------------------------------------------------------------------
# Building blocks
# ----------------------------------------------------------------------------------------
def _ncdf(x: np.ndarray) -> np.ndarray:
    return 0.5 * (1.0 + np.vectorize(erf)(np.asarray(x, dtype=np.float64) / sqrt(2.0)))


def gaussian_response(true_edges, reco_edges, resolution, shift=PROMPT_SHIFT_MEV,
                      eps0=RESPONSE_EPS0, nsigma=RESPONSE_NSIGMA):
    """Response matrix R[j, k] for a Gaussian smearing of E_vis = E_k - shift.

    sigma_k = resolution * sqrt(E_vis_k); the Gaussian is integrated over each reco bin and
    multiplied by eps0. Reco bins lying entirely beyond +-nsigma are set to exactly zero, so
    the matrix is banded with explicit zeros (the dropped mass is below 3e-12 per column).
    """
    true_edges = np.asarray(true_edges, np.float64)
    reco_edges = np.asarray(reco_edges, np.float64)
    ec = 0.5 * (true_edges[:-1] + true_edges[1:])
    evis = ec - shift
    sig = resolution * np.sqrt(np.maximum(evis, 1e-3))
    lo = (reco_edges[:-1, None] - evis[None, :]) / sig[None, :]
    hi = (reco_edges[1:, None] - evis[None, :]) / sig[None, :]
    r = eps0 * (_ncdf(hi) - _ncdf(lo))
    outside = (hi < -nsigma) | (lo > nsigma)
    r[outside] = 0.0
    return r


def flux_xsec(e):
    """Flux x cross-section shape of the synthetic reactor spectrum, E^2 exp(-0.8 E)."""
    return e * e * np.exp(-0.8 * e)


SPECTRUM_TAPER_MEV = 0.25   # smooth ramp to zero at both ends of the true grid


def _taper(e, lo, hi, width):
    """C1 ramp (smoothstep) that is 0 at the grid ends and 1 beyond width from them."""
    x = np.clip(np.minimum(e - lo, hi - e) / width, 0.0, 1.0)
    return x * x * (3.0 - 2.0 * x)


def signal_spectrum(true_edges, n_events, taper=SPECTRUM_TAPER_MEV):
    """Un-oscillated expected counts per true bin, normalised to n_events in total.

    The flux x cross-section shape is multiplied by a smooth ramp that vanishes at both grid
    ends (the IBD threshold at the low end, the end of the simulated range at the high end),
    so that the energy correction never moves content of finite density across a grid end:
    the expectation then has no crease in (a0, a1, a2) at the nominal energy scale.
    """
    ec = 0.5 * (true_edges[:-1] + true_edges[1:])
    w = flux_xsec(ec) * _taper(ec, true_edges[0], true_edges[-1], taper) * np.diff(true_edges)
    return n_events * w / w.sum()


def shape_correlation(n, rng, rho=0.5, mix=0.1):
    """Random SPD correlation: unit-diagonal normalisation of T + mix * G G^T / n.

    T_ij = rho^|i-j| (AR(1), SPD) and G is an n x n standard normal matrix from rng.
    """
    i = np.arange(n)
    t = rho ** np.abs(i[:, None] - i[None, :])
    g = rng.standard_normal((n, n))
    c = t + mix * (g @ g.T) / n
    d = np.sqrt(np.diag(c))
    return c / d[:, None] / d[None, :]


def _template_flat(reco_edges, total):
    w = np.diff(reco_edges)
    return total * w / w.sum()


def _template_exp(reco_edges, total, slope):
    a, b = reco_edges[:-1], reco_edges[1:]
    w = (np.exp(-slope * a) - np.exp(-slope * b)) / slope
    return total * w / w.sum()


def _template_gauss(reco_edges, total, mean, sigma):
    w = _ncdf((reco_edges[1:] - mean) / sigma) - _ncdf((reco_edges[:-1] - mean) / sigma)
    return total * w / w.sum()


def _group_of(true_edges, group_edges, shift):
    """Index of the group (bin of group_edges) containing E_vis of each true-bin centre."""
    ec = 0.5 * (true_edges[:-1] + true_edges[1:]) - shift
    g = np.searchsorted(group_edges, ec, side="right") - 1
    return np.clip(g, 0, len(group_edges) - 2)


class _Params:
    """Parameter table builder. A parameter without a prior gets a minimiser step scale of
    about its posterior width on Asimov data (measured once with the FP64 fit and written
    here as configuration), so that its whitened curvature is close to that of the
    prior-dominated bulk (~2); the Li-9 rates keep 0.1 (whitened curvature ~6) because a
    smaller scale made their weakly determined direction flatter."""

    def __init__(self):
        self.names, self.theta0, self.sigma, self.scale = [], [], [], []

    def add(self, name, theta0, sigma=0.0, scale=None):
        self.names.append(name)
        self.theta0.append(float(theta0))
        self.sigma.append(float(sigma))
        self.scale.append(float(scale if scale is not None else sigma))
        assert self.scale[-1] > 0, name
        return len(self.names) - 1

    def add_block(self, prefix, n, theta0, sigma):
        return np.array([self.add(f"{prefix}[{i}]", theta0, 0.0, sigma) for i in range(n)],
                        dtype=np.int32)

    def arrays(self):
        return (list(self.names), np.array(self.theta0), np.array(self.sigma),
                np.array(self.scale))


def _core_weights(baselines):
    inv = 1.0 / np.asarray(baselines, np.float64) ** 2
    return inv / inv.sum()


# ----------------------------------------------------------------------------------------
# Configurations
# ----------------------------------------------------------------------------------------
def make_c0(seed=BASE_SEED, tiny=False):
    """Single detector, one core at 1050 m, 2-flavour Eq. 1, ~25 parameters.

    200 true bins 1.8-10 MeV, 40 reco bins 1-8 MeV, 8 %/sqrt(E) resolution, 30k un-oscillated
    signal events, flat / exponential / 2.2 MeV-peak backgrounds with rate priors, energy
    scale (a0, a1, a2) with priors, 16 true-space shape reweights with a correlated prior.
    With ``tiny=True`` only (sin^2 2th13, dm2_ee) remain as parameters (all nuisances fixed).
    """
    rng = np.random.default_rng(seed)
    n_true, e_lo, e_hi = 200, 1.8, 10.0
    tedges = np.linspace(e_lo, e_hi, n_true + 1)
    redges = np.linspace(1.0, 8.0, 41)
    p = _Params()
    i_s13 = p.add("sin2_2th13", 0.09, 0.0, 0.04)
    i_dm = p.add("dm2_ee", 2.5e-3, 0.0 if tiny else 1e-4, 1e-4)
    if tiny:
        i_norm, rates, esc, shp = -1, [-1, -1, -1], np.array([-1, -1, -1], np.int32), None
    else:
        i_norm = p.add("norm", 1.0, 0.0, 0.025)
        rates = [p.add("bkg_flat_rate", 1.0, 0.10), p.add("bkg_exp_rate", 1.0, 0.20),
                 p.add("bkg_peak_rate", 1.0, 0.10)]
        esc = np.array([p.add("a0", 0.0, 0.01), p.add("a1", 1.0, 0.005), p.add("a2", 0.0, 0.001)],
                       np.int32)
        shp = p.add_block("shape", 16, 1.0, 0.02)
    names, th0, sig, scl = p.arrays()
    cov_blocks = []
    if shp is not None:
        cov_blocks.append((shp, 0.02 ** 2 * shape_correlation(16, rng)))
        gidx = _group_of(tedges, np.linspace(e_lo, e_hi, 17), 0.0)
        shape_idx = shp[gidx].astype(np.int32)
    else:
        shape_idx = np.full(n_true, -1, np.int32)
    det = Detector("D", redges, gaussian_response(tedges, redges, 0.08))
    bk = [Background("flat", _template_flat(redges, 300.0), rates[0], np.full(40, -1, np.int32)),
          Background("exp", _template_exp(redges, 600.0, 1.0), rates[1], np.full(40, -1, np.int32)),
          Background("peak", _template_gauss(redges, 150.0, 2.2, 0.15), rates[2],
                     np.full(40, -1, np.int32))]
    ds = Dataset("D", 0, signal_spectrum(tedges, 30000.0), np.array([1050.0]), np.array([1.0]),
                 i_norm, -1, esc, shape_idx, bk)
    return ModelSpec("c0_tiny" if tiny else "c0", names, th0, sig, scl, cov_blocks, OSC_EQ1,
                     np.array([i_s13, i_dm, -1, -1], np.int32), np.array([0.09, 2.5e-3, 0.0, 7.53e-5]),
                     np.array([-1], np.int32), n_true, e_lo, e_hi, [det], [ds])


def make_c1(seed=BASE_SEED, sterile=False, flux41=False):
    """Double Chooz-like FD-I / FD-II / ND with two cores, 38 reco bins each, ~291 parameters.

    Oscillation: full Eq. 1 with sin^2 2th12 and dm2_21 as constrained nuisances. With
    sterile=True ("c1s", the 3+1 search): the exact 3+1 vacuum survival with sin^2 th12,
    dm2_21 and dm2_31 constrained, sin^2 th13 free, and the two new parameters sin^2 2th14
    (nominal 0) and dm2_41 (nominal 0.1 eV^2) free; everything else as c1. With flux41=True
    ("c1_flux41"): the signal shape parameters on the uniform 41-bin flux grid of 0.25 MeV over
    1-11.25 MeV (prompt energy) instead of the 38 reco bins, 3 x 41 parameters correlated
    between the datasets as c1's plus an uncorrelated 41 x 41 deviation per dataset. Per dataset:
    efficiency (correlated prior), energy scale (a0, a1, a2), 38 signal shape reweights
    (joint 114 x 114 prior, FD-I/FD-II correlation 0.9). Backgrounds: Li-9 (shape shared by
    all datasets, rate shared by FD-I/FD-II, rates free), accidentals (per-dataset shape and
    rate with prior) and fast neutrons (fixed shape, FD / ND rates with prior). Core powers
    carry a 0.8 % prior.
    """
    rng = np.random.default_rng(seed + 1)
    n_true, e_lo, e_hi = 400, 1.8, 10.0
    tedges = np.linspace(e_lo, e_hi, n_true + 1)
    redges = np.linspace(1.0, 8.6, 39)
    nr = 38
    p = _Params()
    if sterile:
        osc = np.array([p.add("sin2_th12", 0.307, 0.013), p.add("sin2_th13", 0.0231, 0.0, 0.004),
                        p.add("dm2_21", 7.53e-5, 0.18e-5), p.add("dm2_31", 2.5e-3, 1e-4),
                        p.add("sin2_2th14", 0.0, 0.0, 0.01), p.add("dm2_41", 0.1, 0.0, 0.002)],
                       np.int32)
        osc_val = np.array([0.307, 0.0231, 7.53e-5, 2.5e-3, 0.0, 0.1])
    else:
        osc = np.array([p.add("sin2_2th13", 0.09, 0.0, 0.016), p.add("dm2_ee", 2.5e-3, 1e-4),
                        p.add("sin2_2th12", 0.851, 0.02), p.add("dm2_21", 7.53e-5, 0.18e-5)],
                       np.int32)
        osc_val = np.array([0.09, 2.5e-3, 0.851, 7.53e-5])
    eff = p.add_block("eff", 3, 1.0, 0.01)
    esc = [np.array([p.add(f"a0[{d}]", 0.0, 0.01), p.add(f"a1[{d}]", 1.0, 0.005),
                     p.add(f"a2[{d}]", 0.0, 0.001)], np.int32) for d in range(3)]
    r_li9_fd = p.add("li9_rate_fd", 1.0, 0.0, 0.1)
    r_li9_nd = p.add("li9_rate_nd", 1.0, 0.0, 0.1)
    r_acc = [p.add(f"acc_rate[{d}]", 1.0, 0.10) for d in range(3)]
    r_fn_fd = p.add("fn_rate_fd", 1.0, 0.15)
    r_fn_nd = p.add("fn_rate_nd", 1.0, 0.15)
    ng = 41 if flux41 else nr          # signal shape groups per dataset
    shp = p.add_block("shape", 3 * ng, 1.0, 0.02)
    li9 = p.add_block("li9_shape", nr, 0.0, 0.1)
    acc = [p.add_block(f"acc_shape{d}", nr, 0.0, 0.05) for d in range(3)]
    pw = np.array([p.add("power[0]", 1.0, 0.008), p.add("power[1]", 1.0, 0.008)], np.int32)
    names, th0, sig, scl = p.arrays()

    k = np.array([[1.0, 0.9, 0.8], [0.9, 1.0, 0.8], [0.8, 0.8, 1.0]])
    c_shape = shape_correlation(ng, rng)
    cov_shape = 0.02 ** 2 * np.kron(k, c_shape)
    if flux41:   # plus an uncorrelated deviation per dataset (own generator: c1 stays as is)
        rng_u = np.random.default_rng(seed + 11)
        cov_shape = cov_shape + 0.01 ** 2 * np.kron(np.eye(3), shape_correlation(41, rng_u))
    cov_blocks = [
        (eff, 0.01 ** 2 * np.array([[1.0, 0.5, 0.5], [0.5, 1.0, 0.5], [0.5, 0.5, 1.0]])),
        (shp, cov_shape),
        (li9, 0.1 ** 2 * shape_correlation(nr, rng)),
    ] + [(acc[d], 0.05 ** 2 * shape_correlation(nr, rng)) for d in range(3)]

    gidx = _group_of(tedges, redges, PROMPT_SHIFT_MEV)
    gshape = _group_of(tedges, np.linspace(1.0, 11.25, 42), PROMPT_SHIFT_MEV) if flux41 else gidx
    resp = gaussian_response(tedges, redges, 0.08)
    dets = [Detector("FD", redges, resp), Detector("ND", redges, resp.copy())]
    none_r = np.full(nr, -1, np.int32)
    spec = [("FD-I", 0, 20000.0, [950.0, 1150.0], (300.0, 150.0, 200.0), r_li9_fd, r_fn_fd),
            ("FD-II", 0, 40000.0, [950.0, 1150.0], (600.0, 100.0, 400.0), r_li9_fd, r_fn_fd),
            ("ND", 1, 150000.0, [300.0, 500.0], (1500.0, 500.0, 2500.0), r_li9_nd, r_fn_nd)]
    datasets = []
    for d, (nm, det, nev, base, (nli, nacc, nfn), rli, rfn) in enumerate(spec):
        bk = [Background("li9", _template_gauss(redges, nli, 4.5, 2.0), rli, li9.copy()),
              Background("acc", _template_exp(redges, nacc, 2.0), r_acc[d], acc[d].copy()),
              Background("fn", _template_flat(redges, nfn), rfn, none_r.copy())]
        base = np.array(base)
        datasets.append(Dataset(nm, det, signal_spectrum(tedges, nev), base, _core_weights(base),
                                -1, int(eff[d]), esc[d], shp[d * ng + gshape].astype(np.int32), bk))
    return ModelSpec("c1s" if sterile else ("c1_flux41" if flux41 else "c1"), names, th0, sig, scl, cov_blocks,
                     OSC_STERILE4 if sterile else OSC_EQ1, osc, osc_val, pw, n_true, e_lo, e_hi,
                     dets, datasets)


def make_c2(seed=BASE_SEED):
    """Medium-baseline far detector (10 cores, 52-53.5 km) plus a near detector, ~460 params.

    Exact 3-flavour vacuum survival (normal ordering), 2000 true bins 1.8-8 MeV, 3 %/sqrt(E)
    resolution into 400 (FD) and 38 (ND) reco bins, 100k (FD) and 200k (ND) un-oscillated
    events, no backgrounds. Nuisances: core powers (0.8 %), free FD / ND normalisations,
    quadratic energy scale per detector, 400 + 38 shape reweights with correlated priors.
    """
    rng = np.random.default_rng(seed + 2)
    n_true, e_lo, e_hi = 2000, 1.8, 8.0
    tedges = np.linspace(e_lo, e_hi, n_true + 1)
    fd_edges = np.linspace(1.018, 7.218, 401)
    nd_edges = np.linspace(1.018, 7.218, 39)
    p = _Params()
    i_s12 = p.add("sin2_th12", 0.307, 0.013)
    i_s13 = p.add("sin2_th13", 0.022, 0.0007)
    i_dm21 = p.add("dm2_21", 7.5e-5, 0.2e-5)
    i_dm31 = p.add("dm2_31", 2.5e-3, 0.0, 1e-5)
    pw = np.array([p.add(f"power[{c}]", 1.0, 0.008) for c in range(10)], np.int32)
    norm = [p.add("norm_fd", 1.0, 0.0, 0.005), p.add("norm_nd", 1.0, 0.0, 0.003)]
    esc = [np.array([p.add(f"a0[{d}]", 0.0, 0.01), p.add(f"a1[{d}]", 1.0, 0.005),
                     p.add(f"a2[{d}]", 0.0, 0.001)], np.int32) for d in range(2)]
    shp_fd = p.add_block("shape_fd", 400, 1.0, 0.02)
    shp_nd = p.add_block("shape_nd", 38, 1.0, 0.02)
    names, th0, sig, scl = p.arrays()
    cov_blocks = [(shp_fd, 0.02 ** 2 * shape_correlation(400, rng)),
                  (shp_nd, 0.02 ** 2 * shape_correlation(38, rng))]
    dets = [Detector("FD", fd_edges, gaussian_response(tedges, fd_edges, 0.03)),
            Detector("ND", nd_edges, gaussian_response(tedges, nd_edges, 0.03))]
    fd_base = np.linspace(52000.0, 53500.0, 10)
    nd_base = np.linspace(400.0, 550.0, 10)
    g_fd = _group_of(tedges, fd_edges, PROMPT_SHIFT_MEV)
    g_nd = _group_of(tedges, nd_edges, PROMPT_SHIFT_MEV)
    datasets = [
        Dataset("FD", 0, signal_spectrum(tedges, 100000.0), fd_base, _core_weights(fd_base),
                norm[0], -1, esc[0], shp_fd[g_fd].astype(np.int32), []),
        Dataset("ND", 1, signal_spectrum(tedges, 200000.0), nd_base, _core_weights(nd_base),
                norm[1], -1, esc[1], shp_nd[g_nd].astype(np.int32), []),
    ]
    return ModelSpec("c2", names, th0, sig, scl, cov_blocks, OSC_VACUUM3,
                     np.array([i_s12, i_s13, i_dm21, i_dm31], np.int32),
                     np.array([0.307, 0.022, 7.5e-5, 2.5e-3]), pw, n_true, e_lo, e_hi, dets,
                     datasets)


def make_model(name: str, seed: int = BASE_SEED, remap: int = 0) -> ModelSpec:
    """The named model; remap=1 selects the area-conserving spline energy correction."""
    if remap:
        spec = make_model(name, seed)
        spec.remap = int(remap)
        return spec
    if name == "c0":
        return make_c0(seed)
    if name == "c0_tiny":
        return make_c0(seed, tiny=True)
    if name == "c1":
        return make_c1(seed)
    if name == "c1s":
        return make_c1(seed, sterile=True)
    if name == "c1_flux41":
        return make_c1(seed, flux41=True)
    if name == "c2":
        return make_c2(seed)
    raise ValueError(f"unknown model {name!r}")


# ----------------------------------------------------------------------------------------
# Instances and pseudo-data
# ----------------------------------------------------------------------------------------
# Widths used to draw the true signal parameters of ensemble instances (+-3 sigma, uniform).
TRUE_DRAW_SIGMA = {
    "c0": {"sin2_2th13": 0.02, "dm2_ee": 1e-4},
    "c1": {"sin2_2th13": 0.016, "dm2_ee": 1e-4},
    "c2": {"sin2_th13": 0.0007, "dm2_31": 1e-5},
}
# Dataset masks drawn for C1 instances of an ensemble: {FD-I}, {FD-II, ND}, {all three}.
C1_MASKS = (0b001, 0b110, 0b111)


@dataclass
class Instance:
    model: str        # model key ("c0", "c1", "c2")
    mask: int         # bit d set = dataset d enters the likelihood
    theta_true: np.ndarray
    seed: int


def draw_theta_true(spec: ModelSpec, rng) -> np.ndarray:
    th = spec.theta0.copy()
    for nm, s in TRUE_DRAW_SIGMA[spec.name.split("_")[0]].items():
        if nm in spec.param_names:
            th[spec.index(nm)] += rng.uniform(-3.0, 3.0) * s
    return th


def make_ensemble(n: int, specs: dict, frac_c2: float = 1.0 / 3.0, base: int = BASE_SEED,
                  models=("c1", "c2")) -> list:
    """Instance table of an uneven ensemble: a share frac_c2 of models[1], the rest models[0].

    Instance i draws from SplitMix64(base + i): which model, which dataset mask (C1 only) and
    the true signal parameters (uniform within +-3 sigma of nominal).
    """
    out = []
    for i in range(n):
        s = instance_seed(i, base)
        rng = np.random.default_rng(s)
        m = models[1] if (len(models) > 1 and rng.uniform() < frac_c2) else models[0]
        spec = specs[m]
        mask = int(C1_MASKS[rng.integers(3)]) if m == "c1" else spec.all_mask()
        out.append(Instance(m, mask, draw_theta_true(spec, rng), s))
    return out


def poisson_data(mu: np.ndarray, seed: int) -> np.ndarray:
    """Poisson pseudo-data around the expectation mu (numpy PCG64 stream of this seed)."""
    rng = np.random.default_rng(seed)
    return rng.poisson(np.maximum(np.asarray(mu, np.float64), 0.0)).astype(np.float64)


# ----------------------------------------------------------------------------------------
# Monte Carlo events (event-level reweighting of the signal)
# ----------------------------------------------------------------------------------------
@dataclass
class McEvents:
    """Simulated signal events of one detector, sorted by reco bin.

    energy: true neutrino energy (float32, MeV); core: index of the emitting core (uint8);
    weight: expected events represented by each (float32); bin: reco bin (int32,
    non-decreasing); core_L: baseline of each core (m); osc_mode / osc_nominal: survival
    formula and its nominal parameters (same conventions as ModelSpec)."""
    energy: np.ndarray
    core: np.ndarray
    weight: np.ndarray
    bin: np.ndarray
    n_bins: int
    core_L: np.ndarray
    osc_mode: int
    osc_nominal: np.ndarray


def make_mc_events(n_events: int, geometry: str = "dc_fd", seed: int = BASE_SEED) -> McEvents:
    """n_events simulated events drawn from the synthetic flux x cross-section (with its end
    ramps) over 1.8-10 MeV, a core per event in proportion to L^-2, prompt energy E - 0.782 MeV
    smeared by the detector's Gaussian resolution, kept inside the reco range, sorted by reco
    bin. geometry "dc_fd": the two-core far detector at 950 / 1150 m, 8 %/sqrt(E), 38 bins over
    1.0-8.6 MeV, 40k expected events, Eq. 1 survival; "juno_fd": ten cores at 52.0-53.5 km,
    3 %/sqrt(E), 400 bins over 1.018-7.218 MeV, 100k expected events, exact 3-flavour
    survival."""
    rng = np.random.default_rng(seed + 101)
    if geometry == "dc_fd":
        L = np.array([950.0, 1150.0])
        res, redges, n_exp = 0.08, np.linspace(1.0, 8.6, 39), 40_000.0
        mode, nominal = OSC_EQ1, np.array([0.09, 2.5e-3, 0.851, 7.53e-5])
    elif geometry == "juno_fd":
        L = np.linspace(52_000.0, 53_500.0, 10)
        res, redges, n_exp = 0.03, np.linspace(1.018, 7.218, 401), 100_000.0
        mode, nominal = OSC_VACUUM3, np.array([0.307, 0.022, 7.5e-5, 2.5e-3])
    else:
        raise ValueError(geometry)
    e_lo, e_hi = 1.8, 10.0
    grid = np.linspace(e_lo, e_hi, 20_001)
    mid = 0.5 * (grid[:-1] + grid[1:])
    dens = flux_xsec(mid) * _taper(mid, e_lo, e_hi, SPECTRUM_TAPER_MEV)
    cdf = np.concatenate([[0.0], np.cumsum(dens)])
    cdf /= cdf[-1]
    u = rng.random(n_events)
    cell = np.clip(np.searchsorted(cdf, u, side="right") - 1, 0, len(mid) - 1)
    frac = (u - cdf[cell]) / np.maximum(cdf[cell + 1] - cdf[cell], 1e-300)
    e_true = grid[cell] + frac * (grid[cell + 1] - grid[cell])
    w_core = L ** -2.0
    core = rng.choice(len(L), size=n_events, p=w_core / w_core.sum()).astype(np.uint8)
    evis = np.maximum(e_true - PROMPT_SHIFT_MEV, 1e-3)
    e_rec = evis + res * np.sqrt(evis) * rng.standard_normal(n_events)
    b = np.floor((e_rec - redges[0]) / (redges[1] - redges[0])).astype(np.int64)
    keep = (b >= 0) & (b < len(redges) - 1)
    order = np.argsort(b[keep], kind="stable")
    weight = np.full(int(keep.sum()), RESPONSE_EPS0 * n_exp / n_events, np.float32)
    return McEvents(energy=e_true[keep][order].astype(np.float32), core=core[keep][order],
                    weight=weight, bin=b[keep][order].astype(np.int32), n_bins=len(redges) - 1,
                    core_L=L, osc_mode=mode, osc_nominal=nominal)
