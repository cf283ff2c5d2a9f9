"""Host-side checks of constants that the CUDA kernels hard-code.

The BF16 path's GELU uses erf from Abramowitz & Stegun, Handbook of
Mathematical Functions, formula 7.1.28 (|error| <= 3e-7 for u >= 0).  The
coefficients are read from the kernels' shared header and the formula is checked
against that published bound, so a mistyped coefficient fails here.
"""
import os
import re

import numpy as np
from scipy.special import erf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2605_13807_gb300", "csrc", "psr_bf16_math.cuh")


def _gelu_fit():
    src = open(SRC).read()
    vals = {k: float(v) for k, v in re.findall(r"#define PSR_GELU_(G\d) ([0-9.eE+-]+)f", src)}
    assert sorted(vals) == ["G1", "G3", "G5"]
    return vals["G1"], vals["G3"], vals["G5"]


def _coeffs():
    src = open(SRC).read()
    vals = {int(k): float(v) for k, v in re.findall(r"#define PSR_AS7128_A(\d) ([0-9.eE+-]+)f", src)}
    assert sorted(vals) == [1, 2, 3, 4, 5, 6]
    return [vals[i] for i in range(1, 7)]


def test_as7128_erf_meets_its_published_bound():
    a = _coeffs()
    u = np.linspace(0.0, 8.0, 200001)
    poly = 1.0 + sum(a[k] * u ** (k + 1) for k in range(6))
    approx = 1.0 - poly ** -16
    assert np.max(np.abs(approx - erf(u))) <= 3.0e-7


def test_gelu_from_as7128_is_close_to_exact_gelu():
    a = _coeffs()
    x = np.linspace(-12.0, 12.0, 240001)
    u = np.abs(x) / np.sqrt(2.0)
    poly = 1.0 + sum(a[k] * u ** (k + 1) for k in range(6))
    e = 1.0 - poly ** -16
    gelu = 0.5 * x * (1.0 + np.sign(x) * e)
    exact = 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))
    assert np.max(np.abs(gelu - exact)) <= 3.0e-7 * 0.5 * 12.0


def test_fitted_tanh_gelu_error_is_far_below_bf16_rounding():
    """The layer-0/1 GELU form (outputs rounded to BF16 at once) stays within
    3e-5 of the exact GELU in FP32 arithmetic; a 2^-11 relative error in tanh
    adds at most 2.5e-4 |x|, under the BF16 rounding step (2^-8 |x|) of an
    activation of the same magnitude."""
    g1, g3, g5 = (np.float32(v) for v in _gelu_fit())
    x = np.linspace(-16.0, 16.0, 320001).astype(np.float32)
    s = np.minimum(x * x, np.float32(36.0))
    arg = x * ((g5 * s + g3) * s + g1)
    t = np.tanh(arg.astype(np.float64))
    exact = 0.5 * x.astype(np.float64) * (1.0 + erf(x.astype(np.float64) / np.sqrt(2.0)))
    approx = 0.5 * x * (1.0 + t.astype(np.float32))
    assert np.max(np.abs(approx - exact)) <= 3.0e-5
    for sgn in (1.0, -1.0):
        tt = t * (1.0 + sgn * 2.0 ** -10.987)
        worst = np.abs(0.5 * x * (1.0 + tt) - exact)
        assert np.all(worst <= 2.5e-4 * np.abs(x) + 3.0e-5)
