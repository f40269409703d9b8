"""Fits the polynomial that the event kernel uses for sin^2(pi r), |r| <= 1/2.

p(u) = u (c0 + c1 u + ... + c7 u^7), u = r^2, chosen to minimise the largest absolute error
over u in [0, 0.2501] by Lawson's iteratively reweighted least squares (C. L. Lawson, 1961:
the weights of a least-squares fit are multiplied by the current errors until the fit
equi-oscillates). The factor u makes p(0) = 0 exactly. In FP64 the fit is within 5e-13 of
sin^2; evaluated by Horner's rule in FP32 with fused multiply-adds its error is below 1.8e-7,
i.e. set by the FP32 rounding of values near 1, not by the fit.

Run: python sin2pi_fit.py  (prints the coefficients as float32 literals and both errors)."""
import numpy as np


def fit(deg=7, u_max=0.2501, n=4000, iters=200):
    t = np.cos(np.pi * (np.arange(n) + 0.5) / n)
    u = (t + 1) / 2 * u_max
    f = np.sin(np.pi * np.sqrt(u)) ** 2
    A = np.stack([u ** (k + 1) for k in range(deg + 1)], 1)
    w = np.full(n, 1.0 / n)
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(A * sw[:, None], f * sw, rcond=None)
        w = w * np.abs(A @ c - f)
        w /= w.sum()
    return c, float(np.abs(A @ c - f).max())


def f32_error(c32):
    r = np.linspace(-0.5, 0.5, 2_000_001).astype(np.float32)
    u = (r * r).astype(np.float32)
    q = np.full_like(u, c32[-1])
    for k in range(len(c32) - 2, -1, -1):
        q = (q.astype(np.float64) * u + c32[k]).astype(np.float32)
    p = (u.astype(np.float64) * q).astype(np.float32)
    return float(np.abs(p - np.sin(np.pi * r.astype(np.float64)) ** 2).max())


if __name__ == "__main__":
    c, err = fit()
    c32 = c.astype(np.float32)
    print("coefficients:", ", ".join(f"{float(x):.9g}f" for x in c32))
    print(f"fit error (FP64) {err:.3g}, FP32 Horner error {f32_error(c32):.3g}")
