"""The GELU of the network kernels evaluates the normal CDF Phi by a
polynomial fit (the coefficients kPhiFit in tamp_mlp.cu): Phi(z) = sat(1/2 +
z p(z^2)), p of degree 8 fitted on |z| <= 2.9 sqrt 2, sat the saturation to
[0, 1] of the last FMA, which gives Phi = 1 or 0 beyond the fitted range.
Evaluated here the way the kernel does -- FP32 Horner in s = z^2, the last
step saturated -- it must stay within 2.5e-5 of the double-precision Phi
everywhere (including where p overflows), the GELU built on it (z Phi(z))
within 1e-5 of the exact GELU on |z| <= 2 (where most pre-activations lie),
4.5e-5 on |z| <= 4 and 1e-4 everywhere, and its derivative (Phi(z) + z
phi(z)) within 2.5e-5.  What sets the bar is the BF16 rounding (2^-9 relative:
1e-3 at an activation of 0.5) of the activations the kernels store: the fit's
errors stay an order below it."""
import os

import numpy as np
from scipy.special import erf

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2411_11833_b300", "csrc",
                   "tamp_mlp.cu")


def _coefficients():
    body = open(SRC).read()
    body = body[body.index("kPhiFit[9] = {"):]
    body = body[body.index("{") + 1:body.index("}")]
    return [np.float32(v.strip().rstrip("f")) for v in body.split(",") if v.strip()]   # highest degree first


def _phi_fit(z):
    c = _coefficients()
    z = np.asarray(z, dtype=np.float32)
    with np.errstate(over="ignore", invalid="ignore"):
        s = (z * z).astype(np.float32)
        p = np.full_like(z, c[0])
        for ck in c[1:]:
            p = (p * s + ck).astype(np.float32)
        w = (z.astype(np.float64) * p.astype(np.float64) + 0.5)      # one rounding, as the FMA
    return np.clip(np.nan_to_num(w, nan=0.0, posinf=1.0, neginf=0.0), 0.0, 1.0).astype(np.float32)


def _phi(zd):
    return 0.5 * (1.0 + erf(zd / np.sqrt(2.0)))


def _grid():
    return np.concatenate([np.linspace(-12.0, 12.0, 600001), np.geomspace(12.0, 1e30, 2000),
                           -np.geomspace(12.0, 1e30, 2000)]).astype(np.float32)


def test_phi_fit_against_double_precision_phi():
    assert len(_coefficients()) == 9
    z = _grid()
    assert np.abs(_phi_fit(z).astype(np.float64) - _phi(z.astype(np.float64))).max() <= 2.5e-5


def test_saturation_beyond_the_fitted_range():
    z = np.linspace(4.2, 1e4, 200001).astype(np.float32)
    assert (_phi_fit(z) == 1.0).all() and (_phi_fit(-z) == 0.0).all()


def test_gelu_on_the_fit_against_exact_gelu():
    z = np.linspace(-12.0, 12.0, 600001).astype(np.float32)
    g = (z * _phi_fit(z)).astype(np.float64)
    zd = z.astype(np.float64)
    err = np.abs(g - zd * _phi(zd))
    assert err[np.abs(zd) <= 2.0].max() <= 1e-5
    assert err[np.abs(zd) <= 4.0].max() <= 4.5e-5
    assert err.max() <= 1e-4


def test_gelu_derivative_on_the_fit():
    z = np.linspace(-12.0, 12.0, 600001).astype(np.float32)
    zd = z.astype(np.float64)
    pdf = np.exp(-0.5 * zd * zd) / np.sqrt(2.0 * np.pi)
    d = _phi_fit(z).astype(np.float64) + zd * pdf
    assert np.abs(d - (_phi(zd) + zd * pdf)).max() <= 2.5e-5
