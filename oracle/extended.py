"""Decorrelated normalisation in extended precision (oracle; test
infrastructure only).

Eq. decorrelated sets C_decorr = F^-1/2 q with the symmetric inverse square
root F^-1/2 = U Xi^-1/2 U^T of the Fisher matrix.  In float64 that map loses
about eps kappa(F) / 2 in relative accuracy (its relative condition number is
kappa(F) / 2), which at kappa ~ 1e9 is far above the 1e-10 the other outputs
reach.  To measure how far a float64 result really is from the exact F^-1/2 q
of the same (F, q), this module evaluates it in numpy's long double (80-bit
extended on x86-64, IEEE binary128 on AArch64): a float64 eigendecomposition
gives the starting point X0 ~ F^-1/2, and the coupled Newton-Schulz iteration
for the matrix square root (Higham, Functions of Matrices, 2008, Sect. 6.3)

    T = (3 I - Z Y) / 2,   Y <- Y T,   Z <- T Z,     Y0 = F X0, Z0 = X0,

converges quadratically to Z = F^-1/2 (and Y = F^1/2) from any start with
||I - Z0 Y0|| < 1; it is the stable coupled form of Newton's method for
X F X = I.  F and q are taken as exact.  Every eigenvalue must be above the
1e-12 relative cut of Eq. decorrelated (no component is dropped), which holds
for every Fisher matrix of the workloads here.
"""
from __future__ import annotations

import numpy as np

LD = np.longdouble


def inv_sqrt_extended(F: np.ndarray, iters: int = 8, cut: float = 1e-12):
    """F^-1/2 of a symmetric positive-definite float64 matrix, in long double.

    Returns (Z, residual) with residual = max |I - Z F Z| after the last step.
    """
    F = np.asarray(F, dtype=np.float64)
    F = 0.5 * (F + F.T)
    xi, U = np.linalg.eigh(F)
    if xi.min() < cut * xi.max() or xi.min() <= 0:
        raise ValueError("F has eigenvalues below the decorrelation cut")
    X0 = (U * (1.0 / np.sqrt(xi))) @ U.T
    n = F.shape[0]
    I = np.eye(n, dtype=LD)
    Fl = F.astype(LD)
    Z = X0.astype(LD)
    Z = (Z + Z.T) / 2
    Y = Fl @ Z
    res = None
    for _ in range(iters):
        T = (3 * I - Z @ Y) / 2
        Y, Z = Y @ T, T @ Z
        R = I - Z @ Fl @ Z
        r = float(np.abs(R).max())
        if res is not None and r >= res:
            res = min(res, r)
            break
        res = r
    return (Z + Z.T) / 2, res


def decorrelated_extended(F: np.ndarray, q: np.ndarray):
    """C_decorr = F^-1/2 q (Eq. decorrelated) in long double, F and q exact."""
    Z, _ = inv_sqrt_extended(F)
    return Z @ np.asarray(q, dtype=np.float64).astype(LD)
