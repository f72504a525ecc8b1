"""The emulator kernels' GELU evaluates erf by the rational approximation of
Abramowitz & Stegun 7.1.26 (absolute error at most 1.5e-7).  This test reads
the constants from the kernel source and checks that bound in float64 against
scipy's erf, so a mistyped digit in the kernel fails here rather than as a
small bias in the emulator."""
import math
import os
import re

import numpy as np
from scipy.special import erf

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2605_21149_gb300", "csrc", "emu.cu")


def _kernel_constants():
    text = open(SRC).read()
    body = text[text.index("float two_phi_f(float z)"):]
    body = body[:body.index("}")]
    # the literals with at least five decimals, in source order: 1/sqrt(2),
    # p, then the Horner chain a5, a4, a3, a2, a1 (1.0f, 0.5f, 2.0f skipped)
    nums = [float(x) for x in re.findall(r"-?\d+\.\d{5,}", body)]
    inv_sqrt2, p, a5, a4, a3, a2, a1 = nums
    return inv_sqrt2, p, (a1, a2, a3, a4, a5)


def test_erf_approximation_bound():
    inv_sqrt2, p, a = _kernel_constants()
    assert abs(inv_sqrt2 - 1 / math.sqrt(2)) < 1e-15
    x = np.linspace(0.0, 8.0, 400001)
    t = 1.0 / (1.0 + p * x)
    poly = sum(ak * t ** (k + 1) for k, ak in enumerate(a))
    approx = 1.0 - poly * np.exp(-x * x)
    assert np.abs(approx - erf(x)).max() <= 1.5e-7


def test_gelu_form_matches_definition():
    """GELU(z) = z (1 + erf(z / sqrt 2)) / 2 with 1 + erf = 2 - Q (z >= 0) or
    Q (z < 0): the odd extension of the approximation, checked on both signs."""
    inv_sqrt2, p, a = _kernel_constants()
    z = np.linspace(-9.0, 9.0, 180001)
    x = np.abs(z) * inv_sqrt2
    t = 1.0 / (1.0 + p * x)
    q = sum(ak * t ** (k + 1) for k, ak in enumerate(a)) * np.exp(-0.5 * z * z)
    two_phi = np.where(z >= 0, 2.0 - q, q)
    gelu = 0.5 * z * two_phi
    ref = 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))
    assert np.abs(gelu - ref).max() <= 0.5 * 9.0 * 1.5e-7
