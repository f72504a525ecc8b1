"""Real harmonic matrix Y (pixels x modes), transfer folded in (oracle).

Paper basis (Sect. 2.3.1, Eqs. addition_theorem, S_factored, real_ylm; App. A.1
Eqs. V_spin2, V_multifield; App. A.2 Eqs. spin_y_def, EB_from_spin):

    sY_lm(theta, phi) = sqrt((2l+1)/(4 pi)) d^l_{m,-s}(theta) e^{i m phi}
    E_lm = -(2Y_lm + -2Y_lm)/2 ,   B_lm = +i (2Y_lm - -2Y_lm)/2

A spin-2 field with a_{+-2,lm} = -(a^E_lm +- i a^B_lm) has
    Q = sum_lm [a^E E_lm - a^B B_lm],   U = sum_lm [a^E B_lm + a^B E_lm].
All of a^T, a^E, a^B, Y_lm, E_lm, B_lm obey x_{l,-m} = (-1)^m x*_{lm}, so the
m and -m terms pair into 2 Re(a_m x_m).  With real coefficients
r_m = sqrt(2) Re a_m and s_m = -sqrt(2) Im a_m (m > 0; a_0 real), which have
<r^X r^Y> = <s^X s^Y> = C^XY and <r s> = 0, the real basis functions are

    column     T rows           Q rows                U rows
    T cos m    sqrt2 Re Y_lm    .                     .
    T sin m    sqrt2 Im Y_lm    .                     .
    E cos m    .                sqrt2 Re E_lm         sqrt2 Re B_lm
    E sin m    .                sqrt2 Im E_lm         sqrt2 Im B_lm
    B cos m    .               -sqrt2 Re B_lm         sqrt2 Re E_lm
    B sin m    .               -sqrt2 Im B_lm         sqrt2 Im E_lm
(m = 0: the same without sqrt2, the sin column absent).  Then
S = Y Lambda Y^T with Lambda the 3x3 (T,E,B) spectrum block repeated over the
2l+1 real modes of each l (Eq. Lambda_TEB), and each column is multiplied by
its field's transfer function T_l = B_l p_l (the W_l = B_l^2 p_l^2 of
Eq. signal_cov split symmetrically over the two factors).

Column layout (shared interface with the library, no arithmetic): component
major over the fields present (T, then E, then B), then l = lmin..lmax, then
within l: index 0 for m = 0, 2m-1 for cos m, 2m for sin m.
Row layout: T pixels, then Q pixels, then U pixels.
"""
from __future__ import annotations

import math

import numpy as np

from .wigner import d_matrix_columns


def mode_offset(l: int, lmin: int) -> int:
    return l * l - lmin * lmin


def theta_functions(l: int, theta: np.ndarray):
    """lam_lm, F1_lm, F2_lm for m = 0..l at each theta.

    lam = sqrt((2l+1)/4pi) d^l_{m0}         (spin-0, 0Y_lm = lam e^{imphi})
    F1  = -sqrt((2l+1)/4pi) (d^l_{m,-2} + d^l_{m,2}) / 2   (E_lm = F1 e^{imphi})
    F2  = +sqrt((2l+1)/4pi) (d^l_{m,-2} - d^l_{m,2}) / 2   (B_lm = i F2 e^{imphi})
    Shapes (ntheta, l+1).
    """
    nrm = math.sqrt((2 * l + 1) / (4.0 * math.pi))
    # evaluate once per distinct colatitude (HEALPix rings share theta)
    ut, inv = np.unique(np.asarray(theta, dtype=np.float64), return_inverse=True)
    d = d_matrix_columns(l, [-2, 0, 2], ut)  # (nt, 2l+1, 3), first index m = -l..l
    dm = d[inv.reshape(-1), l:, :]  # m = 0..l
    lam = nrm * dm[:, :, 1]
    F1 = -0.5 * nrm * (dm[:, :, 0] + dm[:, :, 2])
    F2 = 0.5 * nrm * (dm[:, :, 0] - dm[:, :, 2])
    return lam, F1, F2


def build_Y(lmin: int, lmax: int, theta_T, phi_T, theta_P, phi_P,
            transfer_T, transfer_P, has_T: bool, has_P: bool) -> np.ndarray:
    """Dense Y (n x k) as documented in the module docstring."""
    theta_T = np.asarray(theta_T, dtype=np.float64)
    phi_T = np.asarray(phi_T, dtype=np.float64)
    theta_P = np.asarray(theta_P, dtype=np.float64)
    phi_P = np.asarray(phi_P, dtype=np.float64)
    nT = theta_T.size if has_T else 0
    nP = theta_P.size if has_P else 0
    k0 = (lmax + 1) ** 2 - lmin ** 2
    ncomp = (1 if has_T else 0) + (2 if has_P else 0)
    Y = np.zeros((nT + 2 * nP, ncomp * k0))
    s2 = math.sqrt(2.0)
    cT = 0
    cE = k0 if has_T else 0
    cB = cE + k0
    for l in range(lmin, lmax + 1):
        off = mode_offset(l, lmin)
        ms = np.arange(0, l + 1)
        if has_T:
            lam, _, _ = theta_functions(l, theta_T)
            cosm = np.cos(np.outer(phi_T, ms))
            sinm = np.sin(np.outer(phi_T, ms))
            t = transfer_T[l]
            Y[:nT, cT + off] = t * lam[:, 0]
            for m in range(1, l + 1):
                Y[:nT, cT + off + 2 * m - 1] = t * s2 * lam[:, m] * cosm[:, m]
                Y[:nT, cT + off + 2 * m] = t * s2 * lam[:, m] * sinm[:, m]
        if has_P:
            _, F1, F2 = theta_functions(l, theta_P)
            cosm = np.cos(np.outer(phi_P, ms))
            sinm = np.sin(np.outer(phi_P, ms))
            t = transfer_P[l]
            q0, u0 = nT, nT + nP
            # Re E = F1 cos, Im E = F1 sin, Re B = -F2 sin, Im B = F2 cos
            reE, imE = F1 * cosm, F1 * sinm
            reB, imB = -F2 * sinm, F2 * cosm
            # m = 0
            Y[q0:q0 + nP, cE + off] = t * reE[:, 0]
            Y[u0:u0 + nP, cE + off] = t * reB[:, 0]
            Y[q0:q0 + nP, cB + off] = -t * reB[:, 0]
            Y[u0:u0 + nP, cB + off] = t * reE[:, 0]
            for m in range(1, l + 1):
                ic, is_ = off + 2 * m - 1, off + 2 * m
                Y[q0:q0 + nP, cE + ic] = t * s2 * reE[:, m]
                Y[u0:u0 + nP, cE + ic] = t * s2 * reB[:, m]
                Y[q0:q0 + nP, cE + is_] = t * s2 * imE[:, m]
                Y[u0:u0 + nP, cE + is_] = t * s2 * imB[:, m]
                Y[q0:q0 + nP, cB + ic] = -t * s2 * reB[:, m]
                Y[u0:u0 + nP, cB + ic] = t * s2 * reE[:, m]
                Y[q0:q0 + nP, cB + is_] = -t * s2 * imB[:, m]
                Y[u0:u0 + nP, cB + is_] = t * s2 * imE[:, m]
    return Y


def build_Y_for(w) -> np.ndarray:
    """Y for a synthetic workload description (attributes as in synth.Workload)."""
    return build_Y(w.lmin, w.lmax, w.theta_T, w.phi_T, w.theta_P, w.phi_P,
                   w.transfer_T, w.transfer_P, w.has_T, w.has_P)
