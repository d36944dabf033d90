"""The GELU of the network kernels evaluates erf by a polynomial fit (the
coefficients kErfFit in tamp_mlp.cu).  Evaluated here the way the kernel
does -- FP32 clamp, FP32 Horner in t = 2 x^2 / 3.2^2 - 1 -- it must stay
within 1e-5 of the double-precision erf everywhere, and the GELU built on it
within 2.5e-5 (absolute) of the exact GELU, far below the BF16 rounding of
the activations (2^-9 relative)."""
import os
import re

import numpy as np
from scipy.special import erf

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2411_11833_b300", "csrc",
                   "tamp_mlp.cu")


def _coefficients():
    body = open(SRC).read()
    body = body[body.index("kErfFit[11] = {"):]
    body = body[body.index("{") + 1:body.index("}")]
    return [np.float32(v.strip().rstrip("f")) for v in body.split(",") if v.strip()]   # highest degree first


def _erf_fit(x):
    c = _coefficients()
    x = np.asarray(x, dtype=np.float32)
    xc = np.minimum(np.maximum(x, np.float32(-3.2)), np.float32(3.2))
    t = (xc * xc * np.float32(2.0 / (3.2 * 3.2)) - np.float32(1.0)).astype(np.float32)
    p = c[0]
    for ck in c[1:]:
        p = (p * t + ck).astype(np.float32)
    return (xc * p).astype(np.float32)


def test_erf_fit_against_double_precision_erf():
    assert len(_coefficients()) == 11
    x = np.linspace(-8.0, 8.0, 400001).astype(np.float32)
    assert np.abs(_erf_fit(x).astype(np.float64) - erf(x.astype(np.float64))).max() <= 1e-5


def test_gelu_on_the_fit_against_exact_gelu():
    z = np.linspace(-12.0, 12.0, 600001).astype(np.float32)
    h = np.float32(0.5) * z
    g = h + h * _erf_fit(z * np.float32(0.70710678118654752))
    zd = z.astype(np.float64)
    exact = 0.5 * zd * (1.0 + erf(zd / np.sqrt(2.0)))
    assert np.abs(g.astype(np.float64) - exact).max() <= 2.5e-5
