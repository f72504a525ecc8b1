"""Dense pixel-space brute force for tiny inputs (oracle; test infrastructure only).

Nothing here uses the real harmonic basis of oracle.harmonic.  The pixel
covariance derivatives P_a = dS/dC_a are built two independent ways:

* spin-0 x spin-0 by the Legendre sum of Eq. P_ell,
      (P_l)_pp' = (2l+1)/(4 pi) W_l P_l(cos theta_pp'),
  with P_l from Bonnet's recurrence and W_l = T_l^2;
* every field combination (T, Q, U) by synthesising the pixel response to
  each independent real Gaussian variable of the complex harmonic
  coefficients, straight from App. A.2: a^X_{l,-m} = (-1)^m conj(a^X_{lm})
  with a_{lm} = (x + i y)/sqrt2 (m > 0) and a_{l0} = x, each of x, y having
  variance C_l^XY against the same variable of field Y;
      T       = sum_m a^T_lm Y_lm,
      Q + i U = sum_m a_{2,lm} 2Y_lm,  a_{2,lm} = -(a^E_lm + i a^B_lm)
  (Eqs. spin_y_def, EB_from_spin with sY_lm = sqrt((2l+1)/4pi) d^l_{m,-s} e^{imphi}),
  where d^l comes from the factorial sum (oracle.wigner.d_factorial) and all
  2l+1 values of m are summed explicitly.

The Fisher matrix, noise bias, quadratic estimates and likelihood then follow
from dense pixel-space traces with an explicit inverse of C (Eqs. fisher,
q_ell, noise_bias, pixel_likelihood).  Cost is O(n_a^2 n^3): tiny inputs only.
"""
from __future__ import annotations

import math

import numpy as np

from .wigner import d_factorial

SPEC_PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def legendre_sum_TT(theta, phi, transfer, l):
    """(2l+1)/(4pi) T_l^2 P_l(cos theta_pp') for one l (Eq. P_ell)."""
    st, ct = np.sin(theta), np.cos(theta)
    x = np.outer(ct, ct) + np.outer(st, st) * np.cos(phi[:, None] - phi[None, :])
    x = np.clip(x, -1.0, 1.0)
    p0, p1 = np.ones_like(x), x
    if l == 0:
        pl = p0
    else:
        for j in range(1, l):
            p0, p1 = p1, ((2 * j + 1) * x * p1 - j * p0) / (j + 1)
        pl = p1
    return (2 * l + 1) / (4.0 * math.pi) * transfer[l] ** 2 * pl


def _sY(l, m, s, theta, phi):
    nrm = math.sqrt((2 * l + 1) / (4.0 * math.pi))
    d = np.array([d_factorial(l, m, -s, t) for t in theta])
    return nrm * d * np.exp(1j * m * phi)


def responses(l, theta_T, phi_T, theta_P, phi_P, transfer_T, transfer_P, has_T, has_P):
    """Pixel responses to the real variables of multipole l.

    Returns dict comp -> array (n, 2l+1) of responses (T rows, Q rows, U rows)
    to the variables x_0, (x_m, y_m) for m = 1..l of that field, in the order
    x_0, x_1, y_1, x_2, y_2, ...  (comp: 0=T, 1=E, 2=B).
    """
    nT = len(theta_T) if has_T else 0
    nP = len(theta_P) if has_P else 0
    n = nT + 2 * nP
    out = {}
    if has_T:
        Yp = {m: _sY(l, m, 0, theta_T, phi_T) for m in range(-l, l + 1)}
        R = np.zeros((n, 2 * l + 1))
        for j, (m, a_m, a_mm) in enumerate(_unit_coeffs(l)):
            field = a_m * Yp[m] + (a_mm * Yp[-m] if m > 0 else 0.0)
            R[:nT, j] = field.real * transfer_T[l]
            assert np.max(np.abs(field.imag)) < 1e-12
        out[0] = R
    if has_P:
        A2 = {m: _sY(l, m, 2, theta_P, phi_P) for m in range(-l, l + 1)}
        Am2 = {m: _sY(l, m, -2, theta_P, phi_P) for m in range(-l, l + 1)}
        for comp in (1, 2):
            R = np.zeros((n, 2 * l + 1))
            for j, (m, a_m, a_mm) in enumerate(_unit_coeffs(l)):
                # a^E or a^B set, the other zero
                if comp == 1:
                    c_m, c_mm = -a_m, -a_mm
                    cc_m, cc_mm = -a_m, -a_mm          # a_{-2} = -(a^E - i a^B)
                else:
                    c_m, c_mm = -1j * a_m, -1j * a_mm
                    cc_m, cc_mm = 1j * a_m, 1j * a_mm
                P = c_m * A2[m] + (c_mm * A2[-m] if m > 0 else 0.0)
                Pm = cc_m * Am2[m] + (cc_mm * Am2[-m] if m > 0 else 0.0)
                # Q - iU synthesised independently must be the conjugate of Q + iU
                assert np.max(np.abs(Pm - np.conj(P))) < 1e-11
                R[nT:nT + nP, j] = P.real * transfer_P[l]
                R[nT + nP:, j] = P.imag * transfer_P[l]
            out[comp] = R
    return out


def _unit_coeffs(l):
    """(m, a_m, a_{-m}) for each real variable x_0, x_1, y_1, ..., x_l, y_l."""
    r2 = 1.0 / math.sqrt(2.0)
    res = [(0, 1.0 + 0j, 0j)]
    for m in range(1, l + 1):
        sgn = (-1) ** m
        res.append((m, r2 + 0j, sgn * r2 + 0j))          # x_m
        res.append((m, 1j * r2, -1j * sgn * r2))        # y_m
    return res


def pixel_derivatives(theta_T, phi_T, theta_P, phi_P, transfer_T, transfer_P,
                      has_T, has_P, lmin, lmax, spec):
    """P_a = dS/dC_a as dense (n x n) matrices, a = (spec, l) spectrum-major."""
    comps = ((0,) if has_T else ()) + ((1, 2) if has_P else ())
    R = {l: responses(l, theta_T, phi_T, theta_P, phi_P, transfer_T, transfer_P, has_T, has_P)
         for l in range(lmin, lmax + 1)}
    Ps = []
    for s in spec:
        x, y = SPEC_PAIRS[s]
        for l in range(lmin, lmax + 1):
            if x not in comps or y not in comps:
                raise ValueError("spectrum needs a field that is absent")
            Rx, Ry = R[l][x], R[l][y]
            P = Rx @ Ry.T
            if x != y:
                P = P + P.T
            Ps.append(P)
    return Ps


def signal_from_derivatives(Ps, cl, spec, lmin, lmax):
    """S = sum_a C_a P_a over the spectra listed (all six for a full S)."""
    S = np.zeros_like(Ps[0])
    nl = lmax - lmin + 1
    for A, s in enumerate(spec):
        for i, l in enumerate(range(lmin, lmax + 1)):
            S += cl[s, l] * Ps[A * nl + i]
    return S


def qml_dense(Ps, C, N, maps=None):
    """Dense pixel-space F, b, y and lnL (Eqs. fisher, q_ell, noise_bias, pixel_likelihood)."""
    Ci = np.linalg.inv(C)
    Ci = 0.5 * (Ci + Ci.T)
    CP = [Ci @ P for P in Ps]
    na = len(Ps)
    F = np.zeros((na, na))
    for a in range(na):
        for b in range(na):
            F[a, b] = 0.5 * np.sum(CP[a] * CP[b].T)   # 1/2 tr[C^-1 P_a C^-1 P_b]
    CN = Ci @ N
    b = np.array([0.5 * np.sum(CP[a] * CN.T) for a in range(na)])
    out = {"F": F, "b": b}
    if maps is not None:
        d = maps.reshape(maps.shape[0], -1)
        Cid = Ci @ d
        out["y"] = np.array([0.5 * np.sum(Cid * (Ps[a] @ Cid), axis=0) for a in range(na)])
        sign, logdet = np.linalg.slogdet(C)
        chi2 = np.sum(d * Cid, axis=0)
        out.update(chi2=chi2, logdet=logdet, lnL=-0.5 * (chi2 + logdet))
    return out
