"""Warm-start network configuration: which inputs each geometry fills and which parameters the
twelve outputs predict (argument tables only; training, inference and the fits run in the
library's kernels).

Inputs (438 slots): the far + near spectra of the 53 km geometry fill all 438; the three
38-bin datasets of the 1 km geometry fill slots 0-113 and slot 114 carries a one-hot marking
that geometry. Outputs (12, standardised by each parameter's width): 1 km geometry - the two
oscillation parameters, the nine energy-scale coefficients and the far-detector Li-9 rate;
53 km geometry - the four oscillation parameters, the six energy-scale coefficients and the two
normalisations. The oscillation parameters of interest are drawn uniformly within +-3.5 widths
of nominal for training, every other parameter from its prior.
"""
from __future__ import annotations

import numpy as np

from . import fitcore, synth

N_IN, N_HIDDEN, N_HIDDEN_LAYERS, N_OUT = 438, 512, 3, 12
UNIFORM_WIDTHS = 3.5

_TARGETS = {
    "c1": ["sin2_2th13", "dm2_ee"] + [f"a{k}[{d}]" for d in range(3) for k in range(3)]
          + ["li9_rate_fd"],
    "c2": ["sin2_th12", "sin2_th13", "dm2_21", "dm2_31"]
          + [f"a{k}[{d}]" for d in range(2) for k in range(3)] + ["norm_fd", "norm_nd"],
}
_LAYOUT = {"c1": (0, 114), "c2": (0, -1)}


def param_width(spec, i: int) -> float:
    """Prior width of parameter i (a covariance block's diagonal, an individual prior, or for a
    free parameter the width its true value is drawn with, else its step scale)."""
    for idx, cov in spec.cov_blocks:
        hit = np.flatnonzero(np.asarray(idx) == i)
        if hit.size:
            return float(np.sqrt(cov[hit[0], hit[0]]))
    if spec.prior_sigma[i] > 0:
        return float(spec.prior_sigma[i])
    draw = synth.TRUE_DRAW_SIGMA.get(spec.name.split("_")[0], {})
    nm = spec.param_names[i]
    return float(draw.get(nm, spec.scale[i]))


def geometry(spec) -> fitcore.fit_warmstart_geom:
    key = spec.name.split("_")[0]
    slot0, onehot = _LAYOUT[key]
    tidx = [spec.index(n) for n in _TARGETS[key]]
    tscl = [param_width(spec, i) for i in tidx]
    draw = synth.TRUE_DRAW_SIGMA.get(key, {})
    uidx = [spec.index(n) for n in draw if n in spec.param_names]
    uhalf = [UNIFORM_WIDTHS * draw[spec.param_names[i]] for i in uidx]
    masks = synth.C1_MASKS if key == "c1" else ()
    return fitcore.make_geom(slot0, onehot, tidx, tscl, uidx, uhalf, masks)


def network(seed: int = 0) -> fitcore.Mlp:
    return fitcore.Mlp(N_IN, N_HIDDEN, N_HIDDEN_LAYERS, N_OUT, seed=seed)


def train(net, models, specs, n_steps, batch=4096, lr=1e-3, weight_decay=1e-4, seed=1,
          stream=None):
    """Trains on fresh device-drawn samples of every geometry in turn; returns the losses."""
    geoms = [geometry(s) for s in specs]
    losses = np.zeros(n_steps)
    fitcore.fit_warmstart_train(net, models, geoms, n_steps, batch, lr, weight_decay, seed,
                                losses, stream)
    return losses


def predict_starts(net, model, spec, B, data, masks, theta_out, stream=None):
    """Start points theta_out [B x P] (device) for the device spectra data [B x n_data]."""
    g = geometry(spec)
    n = g.n_targets
    fitcore.fit_warmstart_predict(net, model, B, data, masks, g.slot0, g.onehot_slot,
                                  list(g.target_idx)[:n], list(g.target_scale)[:n], theta_out,
                                  stream)
