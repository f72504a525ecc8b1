"""Small Wigner d-matrix (oracle; test infrastructure only).

Convention (the one App. A.2 builds on, Eq. spin_y_def):
    d^l_{m'm}(beta) = <l m'| exp(-i beta J_y) |l m>,
with J_+|l m> = sqrt((l-m)(l+m+1)) |l m+1> and J_y = (J_+ - J_-)/(2i).
This reproduces the textbook (Wigner) factorial sum, implemented separately in
`d_factorial` for pins on small l.

`d_matrix_columns` evaluates the definition directly: J_y is Hermitian with
eigenvalues -l..l, so exp(-i beta J_y) = U diag(exp(-i beta mu)) U^H from one
eigendecomposition per l (numpy.linalg.eigh).  Stable for every beta, no
recurrence, no closed-form start value.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def _jy(l: int) -> np.ndarray:
    """J_y in the basis m = -l..l (index m + l)."""
    dim = 2 * l + 1
    jp = np.zeros((dim, dim))
    for m in range(-l, l):
        jp[m + 1 + l, m + l] = math.sqrt((l - m) * (l + m + 1))
    return (jp - jp.T) / 2j


def d_matrix_columns(l: int, cols, beta) -> np.ndarray:
    """d^l_{m', s}(beta) for m' = -l..l and s in `cols`.

    Returns an array of shape (len(beta), 2l+1, len(cols)) (real).  Columns
    with |s| > l are zero.
    """
    beta = np.atleast_1d(np.asarray(beta, dtype=np.float64))
    dim = 2 * l + 1
    out = np.zeros((beta.size, dim, len(cols)))
    if l == 0:
        for j, s in enumerate(cols):
            if s == 0:
                out[:, 0, j] = 1.0
        return out
    mu, U = np.linalg.eigh(_jy(l))
    # phases exp(-i beta mu) : (nb, dim)
    ph = np.exp(-1j * np.outer(beta, mu))
    for j, s in enumerate(cols):
        if abs(s) > l:
            continue
        # column s of U diag(ph) U^H  =  U (ph * conj(U[s, :]))
        v = ph * np.conj(U[s + l, :])[None, :]
        col = v @ U.T  # (nb, dim): sum_k U[m', k] v[k]
        out[:, :, j] = col.real
    return out


def d_factorial(l: int, mp: int, m: int, beta: float) -> float:
    """Textbook Wigner factorial sum for d^l_{mp, m}(beta) (small l only).

    d = sum_k (-1)^(mp - m + k) sqrt((l+mp)!(l-mp)!(l+m)!(l-m)!)
          / ((l+m-k)! k! (mp-m+k)! (l-mp-k)!)
          * cos(beta/2)^(2l+m-mp-2k) * sin(beta/2)^(mp-m+2k)
    The rational coefficients are exact (Fraction); cancellation makes it
    unsuitable beyond l ~ 20 in double precision.
    """
    if abs(mp) > l or abs(m) > l:
        return 0.0
    c, s = math.cos(beta / 2.0), math.sin(beta / 2.0)
    f = math.factorial
    pref = math.sqrt(f(l + mp) * f(l - mp) * f(l + m) * f(l - m))
    total = 0.0
    for k in range(0, 2 * l + 1):
        a, b, cc, d = l + m - k, k, mp - m + k, l - mp - k
        if min(a, b, cc, d) < 0:
            continue
        coef = Fraction((-1) ** (mp - m + k), f(a) * f(b) * f(cc) * f(d))
        total += float(coef) * c ** (2 * l + m - mp - 2 * k) * s ** (mp - m + 2 * k)
    return pref * total
