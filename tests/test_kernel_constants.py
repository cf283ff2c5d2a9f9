"""Host-side checks of constants that the CUDA kernels hard-code.

The BF16 path's GELU uses erf from Abramowitz & Stegun, Handbook of
Mathematical Functions, formula 7.1.28 (|error| <= 3e-7 for u >= 0).  The
coefficients are read from the kernel source and the formula is checked
against that published bound, so a mistyped coefficient fails here.
"""
import os
import re

import numpy as np
from scipy.special import erf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2605_13807_gb300", "csrc", "psr_fwd_bf16.cu")


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
