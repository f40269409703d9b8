"""Warm-start network configuration: which inputs each geometry fills and which parameters the
twelve outputs predict (argument tables only; training, inference and the fits run in the
library's kernels).

Inputs (438 slots): the far + near spectra of the 53 km geometry fill all 438; the three
38-bin datasets of the 1 km geometry fill slots 0-113 and slot 114 carries a one-hot marking
that geometry. Outputs (12, standardised by each parameter's width): 1 km geometry - the two
oscillation parameters, the nine energy-scale coefficients and the far-detector Li-9 rate;
53 km geometry - the four oscillation parameters, the six energy-scale coefficients and the two
normalisations. The oscillation parameters of interest are drawn uniformly within +-3.5 widths
of nominal for training, every other parameter from its prior. The network is trained to
predict where a fit of the spectrum ends: the drawn point moved by one Gauss-Newton step of
-2lnL with the expected Hessian at the nominal point, the mass splittings' columns of the
Jacobian taken at the drawn point (fit_warmstart_train).
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
          stream=None, epochs=1):
    """Trains on device-drawn samples of every geometry in turn; returns the losses. Each epoch
    is one fit_warmstart_train call of n_steps steps under the same seed, so every epoch sees
    the same n_steps x batch samples (the generator is counter-based) with its own cosine
    learning-rate cycle; the optimiser's moments carry over."""
    geoms = [geometry(s) for s in specs]
    out = []
    for _ in range(max(1, int(epochs))):
        losses = np.zeros(n_steps)
        fitcore.fit_warmstart_train(net, models, geoms, n_steps, batch, lr, weight_decay, seed,
                                    losses, stream)
        out.append(losses)
    return np.concatenate(out)


def predict_starts(net, model, spec, B, data, masks, theta_out, stream=None):
    """Start points theta_out [B x P] (device) for the device spectra data [B x n_data]: the
    linearised best fit of every parameter, the network's corrections on its targets."""
    g = geometry(spec)
    n = g.n_targets
    fitcore.fit_warmstart_predict(net, model, B, data, masks, g.slot0, g.onehot_slot,
                                  list(g.target_idx)[:n], list(g.target_scale)[:n], theta_out,
                                  stream)


# ---- weights on disk ------------------------------------------------------------------------
def save_layers(path, dims, layers):
    """Writes a network's FP32 master weights: dims = (n_in, n_hidden, n_hidden_layers, n_out),
    layers = [(w [out x in], b [out]), ...]. One .npz (w0, b0, w1, ...) with the dimensions as a
    JSON string, replaced atomically. The optimiser moments are not kept (a resumed training
    starts them at zero)."""
    import json
    import os
    n_in, n_hidden, n_hl, n_out = (int(x) for x in dims)
    shapes = [(n_hidden if l < n_hl else n_out, n_in if l == 0 else n_hidden) for l in range(n_hl + 1)]
    if len(layers) != len(shapes):
        raise ValueError(f"expected {len(shapes)} layers")
    arrays = {}
    for l, ((w, b), (o, i)) in enumerate(zip(layers, shapes)):
        w = np.ascontiguousarray(w, dtype=np.float32)
        b = np.ascontiguousarray(b, dtype=np.float32)
        if w.shape != (o, i) or b.shape != (o,):
            raise ValueError(f"layer {l}: expected w {(o, i)} and b {(o,)}")
        arrays[f"w{l}"], arrays[f"b{l}"] = w, b
    meta = json.dumps({"n_in": n_in, "n_hidden": n_hidden, "n_hidden_layers": n_hl, "n_out": n_out})
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        np.savez(f, meta=np.array(meta), **arrays)
    os.replace(tmp, path)


def load_layers(path):
    """(dims, layers) as written by save_layers, shapes checked against the dimensions."""
    import json
    with np.load(path, allow_pickle=False) as z:
        m = json.loads(str(z["meta"]))
        dims = (m["n_in"], m["n_hidden"], m["n_hidden_layers"], m["n_out"])
        layers = [(z[f"w{l}"].copy(), z[f"b{l}"].copy()) for l in range(dims[2] + 1)]
    n_in, n_hidden, n_hl, n_out = dims
    for l, (w, b) in enumerate(layers):
        o, i = (n_hidden if l < n_hl else n_out), (n_in if l == 0 else n_hidden)
        if w.shape != (o, i) or b.shape != (o,) or w.dtype != np.float32:
            raise ValueError(f"{path}: layer {l} does not match the dimensions")
    return dims, layers


def save_network(net: fitcore.Mlp, path):
    """Copies the device weights of `net` to `path` (fit_mlp_get_layer per layer)."""
    dims = (net.n_in, net.n_hidden, net.n_layers - 1, net.n_out)
    save_layers(path, dims, [net.get_layer(l)[:2] for l in range(net.n_layers)])


def load_network(path, seed: int = 0) -> fitcore.Mlp:
    """A device network with the weights stored at `path` (fit_mlp_create, fit_mlp_set_layer)."""
    dims, layers = load_layers(path)
    net = fitcore.Mlp(*dims, seed=seed)
    for l, (w, b) in enumerate(layers):
        net.set_layer(l, w, b)
    return net
