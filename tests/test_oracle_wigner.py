"""Pins for the oracle's Wigner d-matrix (App. A.3 conventions)."""
import math
import os

import numpy as np
import pytest
import scipy.special as sp

from oracle import wigner

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "wigner_d_closed_forms.txt")


def _golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#"):
                continue
            j, mp, m, b, v = line.split()
            rows.append((int(j), int(mp), int(m), float(b), float(v)))
    return rows


def test_closed_forms_textbook():
    """Eigen-definition and factorial sum both reproduce the textbook j=1,2 table."""
    for j, mp, m, b, v in _golden():
        D = wigner.d_matrix_columns(j, [m], [b])[0, mp + j, 0]
        assert abs(D - v) < 4e-15
        assert abs(wigner.d_factorial(j, mp, m, b) - v) < 4e-15


@pytest.mark.parametrize("l", [2, 5, 9, 14])
def test_eigen_vs_factorial(l):
    betas = np.array([0.05, 0.7, 1.5707963, 2.4, 3.1])
    cols = [-2, -1, 0, 1, 2]
    D = wigner.d_matrix_columns(l, cols, betas)
    for ib, b in enumerate(betas):
        for mp in range(-l, l + 1):
            for jc, m in enumerate(cols):
                assert abs(D[ib, mp + l, jc] - wigner.d_factorial(l, mp, m, b)) < 1e-12


@pytest.mark.parametrize("l", [3, 30, 95])
def test_unitarity_and_legendre(l):
    """sum_m' d_{m' s}^2 = 1; d^l_{m0} = sqrt((l-m)!/(l+m)!) P_l^m (Condon-Shortley);
    d^l_{00} = P_l."""
    betas = np.linspace(0.01, 3.13, 7)
    D = wigner.d_matrix_columns(l, [-2, 0, 2], betas)
    assert np.allclose(np.sum(D ** 2, axis=1), 1.0, atol=1e-12, rtol=0)
    # scipy's spherical Legendre: sqrt((2l+1)/4pi (l-m)!/(l+m)!) P_l^m(cos b), CS phase included
    for m in range(0, l + 1, max(1, l // 7)):
        ref = sp.sph_legendre_p(l, m, betas) * math.sqrt(4 * math.pi / (2 * l + 1))
        assert np.allclose(D[:, m + l, 1], ref, atol=1e-12, rtol=0)
    assert np.allclose(D[:, l, 1], sp.eval_legendre(l, np.cos(betas)), atol=1e-12)


def test_symmetries():
    """d_{m's} = (-1)^(m'-s) d_{s m'} = d_{-s,-m'} for the columns used by spin-2."""
    l, b = 11, 0.9
    D = wigner.d_matrix_columns(l, list(range(-l, l + 1)), [b])[0]
    for mp in range(-l, l + 1):
        for s in (-2, 0, 2):
            v = D[mp + l, s + l]
            assert abs(v - (-1) ** (mp - s) * D[s + l, mp + l]) < 1e-13
            assert abs(v - D[-s + l, -mp + l]) < 1e-13
