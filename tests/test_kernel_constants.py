"""Constants the kernels carry, checked on the host against the mathematics they stand for."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_sin2pi_polynomial_of_the_event_kernel():
    """The degree-7 polynomial in r^2 that the event and batched-expectation kernels evaluate
    for sin^2(pi r) is within 2e-7 of the exact value over |r| <= 1/2 when evaluated as the
    kernels do (FP32 Horner with fused multiply-adds), and its leading coefficient is pi^2
    rounded to FP32."""
    src = open(os.path.join(ROOT, "paper_2502_15253_gb300", "csrc", "dev_model.cuh")).read()
    body = src[src.index("float sin2pi(float r)"):]
    body = body[:body.index("return u * q;")]
    first = float(re.search(r"float q = (-?[\d.e+-]+)f;", body).group(1))
    rest = [float(x) for x in re.findall(r"q = fmaf\(q, u, (-?[\d.e+-]+)f\);", body)]
    c = np.array([first] + rest, dtype=np.float32)   # highest degree first
    assert len(c) == 8
    assert c[-1] == np.float32(np.pi ** 2)
    r = np.linspace(-0.5, 0.5, 1_000_001).astype(np.float32)
    u = (r * r).astype(np.float32)
    q = np.full_like(u, c[0])
    for k in c[1:]:
        q = (q.astype(np.float64) * u + k).astype(np.float32)   # one rounding per fma
    p = (u.astype(np.float64) * q).astype(np.float32)
    err = np.abs(p.astype(np.float64) - np.sin(np.pi * r.astype(np.float64)) ** 2)
    assert err.max() < 2e-7
    assert p[len(r) // 2] == 0.0
