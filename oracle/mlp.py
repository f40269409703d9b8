"""Plain FP64 reference of the warm-start network - TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this module. The network (not part of the paper; it only proposes start points for the
variable-metric fit) is x -> [Linear, GELU] x H -> Linear with GELU(x) = x Phi(x) (the erf
form), trained on the mean squared error with AdamW (Loshchilov & Hutter, decoupled weight
decay; Adam moments with bias correction, Kingma & Ba). Weights are [out x in] row-major.

Parity status: forward and gradient pinned (GELU against the normal CDF, a 0-hidden-layer
network against the least-squares closed form, central finite differences of the loss);
AdamW pinned (first step is lr * (sign(g) + wd * w) up to eps; moment recursion by hand on
two steps).
"""
from __future__ import annotations

import math

import numpy as np


def gelu(x):
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


def _erf(x):
    return np.vectorize(math.erf, otypes=[np.float64])(x) if np.ndim(x) else math.erf(float(x))


def forward(weights, x):
    """weights: list of (W [out x in], b [out]); returns (output, list of pre-activations,
    list of layer inputs)."""
    a = np.asarray(x, dtype=np.float64)
    pres, ins = [], []
    for li, (W, b) in enumerate(weights):
        ins.append(a)
        z = a @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        if li + 1 < len(weights):
            pres.append(z)
            a = gelu(z)
        else:
            a = z
    return a, pres, ins


def loss_and_grads(weights, x, target):
    """Mean squared error over all B x n_out entries and its gradients per layer."""
    out, pres, ins = forward(weights, x)
    t = np.asarray(target, dtype=np.float64)
    r = out - t
    loss = float(np.mean(r * r))
    d = 2.0 * r / r.size
    grads = [None] * len(weights)
    for li in range(len(weights) - 1, -1, -1):
        W = np.asarray(weights[li][0], np.float64)
        grads[li] = (d.T @ ins[li], d.sum(axis=0))
        if li > 0:
            d = (d @ W) * gelu_grad(pres[li - 1])
    return loss, grads


def adamw_step(w, g, m, v, step, lr, wd, b1=0.9, b2=0.999, eps=1e-8, decay=True):
    """One AdamW update of array w with gradient g; returns (w, m, v). step counts from 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    upd = mh / (np.sqrt(vh) + eps)
    if decay:
        upd = upd + wd * w
    return w - lr * upd, m, v
