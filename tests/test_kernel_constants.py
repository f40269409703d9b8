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


def test_gelu_normal_cdf_of_the_gemm_epilogue():
    """The GEMM epilogue's normal CDF (erfc from the Abramowitz & Stegun 7.1.26 rational form,
    the tail formed without cancellation) read from the source and evaluated in FP32 as the
    kernel does: Phi within 3.5e-7 of the exact value everywhere (the form's own error is
    1.5e-7 / 2; FP32 rounding of 1 - erfc/2 adds the rest), relatively close in the left
    tail down to Phi = 1e-6 (2e-3) and down to 1e-12 (1e-2), so GELU(x) = x Phi(x) and its
    derivative Phi(x) + x phi(x) carry no error that their bf16 rounding (2^-8) would not hide."""
    from scipy.special import ndtr
    src = open(os.path.join(ROOT, "paper_2502_15253_gb300", "csrc", "gemm_tc.cu")).read()
    body = src[src.index("void phi_pair(float x"):]
    body = body[:body.index("cdf = x < 0.f")]
    p = float(re.search(r"fmaf\((-?[\d.]+)f, z, 1.f\)", body).group(1))
    poly = re.search(r"const float q = t \* (.*?);\n", body, re.S).group(1)
    nums = [float(x) for x in re.findall(r"(-?\d+\.\d+)f", poly)]
    # Horner from the innermost: a5, a4, a3, a2, a1
    a5, a4, a3, a2, a1 = nums
    assert (p, a1, a2, a3, a4, a5) == (0.3275911, 0.254829592, -0.284496736, 1.421413741, -1.453152027, 1.061405429)
    f = np.float32
    x = np.linspace(-9.0, 9.0, 2_000_001).astype(f)
    z = (np.abs(x) * f(0.70710678118654752)).astype(f)
    t = (f(1.0) / (f(p) * z + f(1.0))).astype(f)
    q = f(a5)
    for a in (a4, a3, a2, a1):
        q = (q * t + f(a)).astype(f)
    q = (t * q).astype(f)
    e = np.exp((f(-0.5) * x * x).astype(np.float64)).astype(f)
    h = (f(0.5) * q * e).astype(f)
    cdf = np.where(x < 0, h, f(1.0) - h).astype(np.float64)
    exact = ndtr(x.astype(np.float64))
    assert np.max(np.abs(cdf - exact)) < 3.5e-7
    for floor, bound in ((1e-6, 2e-3), (1e-12, 1e-2)):
        m = (x < 0) & (exact > floor)
        assert np.max(np.abs(cdf[m] / exact[m] - 1.0)) < bound
