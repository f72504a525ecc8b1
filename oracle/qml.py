"""QML estimator and pixel likelihood by their definitions (oracle).

Every function states the passage it follows.  Harmonic form: with the
transfer function folded into Y (see oracle.harmonic), S = Y Lambda Y^T and
the derivative of S with respect to one spectrum entry a = (XY, l) is
P_a = Y E_a Y^T (Sect. 2.3.3), where E_a is the 0/1 selector

    E_a = sum_{m-modes i of l} sum_{(u,v) in pairs(a)} e_{u,i} e_{v,i}^T,
    pairs(XX) = {(X,X)},  pairs(XY) = {(X,Y), (Y,X)} for X != Y

(the symmetric placement of a cross-spectrum entry in the 3x3 blocks of
Eq. Lambda_TEB).  With W = Y^T C^-1 Y and w = Y^T C^-1 d the trace identities
used below are the cyclic rewrites of Eqs. fisher, q_ell, noise_bias:

  F_ab = 1/2 tr[C^-1 P_a C^-1 P_b] = 1/2 sum W[v i, u' j] W[v' j, u i]  (Eq. sparse_trace)
  y_a  = 1/2 d^T C^-1 P_a C^-1 d  = 1/2 sum w[u i] w[v i]               (Eq. q_harmonic)
  b_a  = 1/2 tr[C^-1 P_a C^-1 N]  = 1/2 sum (Z^T N Z)[v i, u i], Z = C^-1 Y

The noise bias is evaluated with the explicit product Z^T N Z, not through any
identity the CUDA path may use.  Everything is float64 numpy/scipy.

Fisher index order: spectrum-major over the requested spectra, then l.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

SPEC_PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))  # TT EE BB TE TB EB


def pairs(spec: int):
    x, y = SPEC_PAIRS[spec]
    return [(x, x)] if x == y else [(x, y), (y, x)]


def lambda_blocks(cl: np.ndarray, comps, lmin: int, lmax: int) -> np.ndarray:
    """Lambda_l restricted to the fields present: shape (nl, nc, nc) (Eq. Lambda_TEB)."""
    nc = len(comps)
    lam = np.zeros((lmax - lmin + 1, nc, nc))
    for s, (x, y) in enumerate(SPEC_PAIRS):
        if x in comps and y in comps:
            i, j = comps.index(x), comps.index(y)
            lam[:, i, j] = cl[s, lmin:lmax + 1]
            lam[:, j, i] = cl[s, lmin:lmax + 1]
    return lam


def _l_of_mode(lmin: int, lmax: int) -> np.ndarray:
    return np.concatenate([np.full(2 * l + 1, l) for l in range(lmin, lmax + 1)])


def apply_lambda(Y: np.ndarray, cl, comps, lmin: int, lmax: int) -> np.ndarray:
    """Y Lambda (columns mixed within each (l, m) by the 3x3 spectrum block)."""
    k0 = (lmax + 1) ** 2 - lmin ** 2
    lam = lambda_blocks(cl, comps, lmin, lmax)
    lm = _l_of_mode(lmin, lmax) - lmin
    nc = len(comps)
    out = np.zeros_like(Y)
    for b in range(nc):
        for a in range(nc):
            out[:, b * k0:(b + 1) * k0] += Y[:, a * k0:(a + 1) * k0] * lam[lm, a, b][None, :]
    return out


def signal_cov(Y, cl, comps, lmin, lmax) -> np.ndarray:
    """S = Y Lambda Y^T (Eq. S_factored)."""
    return apply_lambda(Y, cl, comps, lmin, lmax) @ Y.T


def total_cov(Y, cl, comps, lmin, lmax, N) -> np.ndarray:
    """C = S + N (Eq. total_cov)."""
    return signal_cov(Y, cl, comps, lmin, lmax) + N


def mode_starts(lmin: int, lmax: int, edges=None) -> np.ndarray:
    """First harmonic mode of each multipole (edges None) or of each bin.

    The modes of multipoles l in [e, e') are the contiguous range
    [e^2 - lmin^2, e'^2 - lmin^2) of one field's k0 modes, so the selector of a
    bin, E_b = sum_{l in b} E_l (Sect. 2.4: P_b = sum_{l in b} P_l), sums over
    that range.  edges: lmin = e_0 < e_1 < ... < e_nb = lmax + 1.
    """
    if edges is None:
        edges = np.arange(lmin, lmax + 2)
    return np.array([e * e - lmin * lmin for e in edges[:-1]])


def _blocksum(H: np.ndarray, lmin: int, lmax: int, edges=None) -> np.ndarray:
    """Sum an (k0 x k0) array over (l, l') (or (bin, bin')) blocks of modes."""
    starts = mode_starts(lmin, lmax, edges)
    return np.add.reduceat(np.add.reduceat(H, starts, axis=0), starts, axis=1)


def fisher_from_W(W: np.ndarray, spec, comps, lmin: int, lmax: int, edges=None,
                  W2=None) -> np.ndarray:
    """F_ab = 1/2 tr[W E_a W E_b] (Eqs. fisher_harmonic, sparse_trace); with
    bin edges, a and b run over (spectrum, bin) and E_b is the bin selector
    (Sect. 2.4); with W2 the cross-QML mixing matrix 1/2 tr[W E_a W2 E_b]."""
    k0 = (lmax + 1) ** 2 - lmin ** 2
    nc = len(comps)
    nl = lmax - lmin + 1 if edges is None else len(edges) - 1
    W4 = W.reshape(nc, k0, nc, k0)
    V4 = W4 if W2 is None else W2.reshape(nc, k0, nc, k0)
    ci = {c: comps.index(c) for c in comps}
    ns = len(spec)
    F = np.zeros((ns * nl, ns * nl))
    cache = {}
    for A, sa in enumerate(spec):
        for B, sb in enumerate(spec):
            acc = np.zeros((nl, nl))
            for (u, v) in pairs(sa):
                for (up, vp) in pairs(sb):
                    key = (v, up, vp, u)
                    if key not in cache:
                        # H[i, j] = W[v i, u' j] * W[v' j, u i]
                        H = W4[ci[v], :, ci[up], :] * V4[ci[vp], :, ci[u], :].T
                        cache[key] = _blocksum(H, lmin, lmax, edges)
                    acc += cache[key]
            F[A * nl:(A + 1) * nl, B * nl:(B + 1) * nl] = 0.5 * acc
    return F


def trace_selector(M: np.ndarray, spec, comps, lmin: int, lmax: int, edges=None) -> np.ndarray:
    """t_a = sum_{(u,v) in pairs(a)} sum_{i in l} M[v i, u i]  (= tr[E_a M]);
    per bin with edges (Sect. 2.4)."""
    k0 = (lmax + 1) ** 2 - lmin ** 2
    nl = lmax - lmin + 1 if edges is None else len(edges) - 1
    starts = mode_starts(lmin, lmax, edges)
    out = np.zeros(len(spec) * nl)
    for A, sa in enumerate(spec):
        acc = np.zeros(nl)
        for (u, v) in pairs(sa):
            iu, iv = comps.index(u), comps.index(v)
            d = np.einsum("ii->i", M[iv * k0:(iv + 1) * k0, iu * k0:(iu + 1) * k0])
            acc += np.add.reduceat(d, starts)
        out[A * nl:(A + 1) * nl] = acc
    return out


def quad_selector(w: np.ndarray, spec, comps, lmin: int, lmax: int, edges=None,
                  w2=None) -> np.ndarray:
    """y_a = 1/2 w^T E_a w for each column of w (Eq. q_harmonic); shape (na, nsims);
    per bin with edges (Sect. 2.4); with w2 the cross form 1/2 w^T E_a w2."""
    w = np.atleast_2d(w.T).T if w.ndim == 1 else w
    w2 = w if w2 is None else (np.atleast_2d(w2.T).T if w2.ndim == 1 else w2)
    k0 = (lmax + 1) ** 2 - lmin ** 2
    nl = lmax - lmin + 1 if edges is None else len(edges) - 1
    starts = mode_starts(lmin, lmax, edges)
    out = np.zeros((len(spec) * nl, w.shape[1]))
    for A, sa in enumerate(spec):
        acc = np.zeros((nl, w.shape[1]))
        for (u, v) in pairs(sa):
            iu, iv = comps.index(u), comps.index(v)
            prod = w[iu * k0:(iu + 1) * k0] * w2[iv * k0:(iv + 1) * k0]
            acc += np.add.reduceat(prod, starts, axis=0)
        out[A * nl:(A + 1) * nl] = 0.5 * acc
    return out


def normalisations(F: np.ndarray, q: np.ndarray, cut: float = 1e-12):
    """The three output modes of Sect. 2.5.

    deconvolved  C = F^-1 q                          (Eq. deconvolved)
    decorrelated C = F^-1/2 q, F^-1/2 = U Xi^-1/2 U^T with eigenvalues below
                 cut * max set to zero               (Eq. decorrelated)
    convolved    q itself, window matrix F           (Eq. convolved)
    """
    cf = sla.cho_factor(F, lower=True)
    deconv = sla.cho_solve(cf, q)
    xi, U = np.linalg.eigh(F)
    keep = xi >= cut * xi.max()
    inv_sqrt = np.zeros_like(xi)
    inv_sqrt[keep] = 1.0 / np.sqrt(xi[keep])
    Fm12 = (U * inv_sqrt) @ U.T
    decorr = Fm12 @ q
    return deconv, decorr, q.copy(), Fm12


def loglike(C: np.ndarray, d: np.ndarray):
    """lnL = -1/2 [d^T C^-1 d + ln|C|] with const = 0 (Eq. pixel_likelihood).

    Returns (lnL, chi2, logdet); d may hold several maps as columns.
    """
    L = np.linalg.cholesky(C)
    logdet = 2.0 * np.sum(np.log(np.diag(L)))
    x = sla.solve_triangular(L, d, lower=True)
    chi2 = np.sum(x * x, axis=0)
    return -0.5 * (chi2 + logdet), chi2, logdet


def qml(Y, cl_fid, comps, lmin, lmax, N, spec, maps=None, want_bias=True, edges=None):
    """Fisher matrix, noise bias, quadratic estimates and Cl in three modes.

    Follows Sect. 2.2 (Eqs. fisher, q_ell, noise_bias, qml_estimate) in the
    harmonic factorisation of Sect. 2.3.3.  With bin edges (Sect. 2.4) the
    bin derivative P_b = sum_{l in b} P_l takes the place of P_l in F, q and
    the noise bias, and the normalisations act on the binned F.  Returns a
    dict.
    """
    C = total_cov(Y, cl_fid, comps, lmin, lmax, N)
    cf = sla.cho_factor(C, lower=True)
    Z = sla.cho_solve(cf, Y)          # C^-1 Y
    W = Y.T @ Z                       # Y^T C^-1 Y   (Eq. projected_inv)
    W = 0.5 * (W + W.T)
    F = fisher_from_W(W, spec, comps, lmin, lmax, edges)
    out = {"F": F, "W": W, "C": C}
    if want_bias:
        ZNZ = Z.T @ (N @ Z)
        out["b"] = 0.5 * trace_selector(ZNZ, spec, comps, lmin, lmax, edges)
    if maps is not None:
        maps = maps.reshape(maps.shape[0], -1)
        w = Y.T @ sla.cho_solve(cf, maps)   # Y^T C^-1 d  (Eq. weighted_data)
        y = quad_selector(w, spec, comps, lmin, lmax, edges)
        out["w"] = w
        out["y"] = y
        if want_bias:
            q = y - out["b"][:, None]
            out["q"] = q
            dec, decor, conv, Fm12 = normalisations(F, q)
            out.update(cl_deconv=dec, cl_decorr=decor, q_conv=conv, F_inv_sqrt=Fm12)
    return out


def qml_for(wl, Y, maps=None, want_bias=True, edges=None):
    """qml() for a synthetic workload description."""
    return qml(Y, wl.cl_fid, wl.comps, wl.lmin, wl.lmax, wl.N(), wl.spec, maps, want_bias, edges)


def lambda_dense(cl, comps, lmin: int, lmax: int) -> np.ndarray:
    """The (k x k) matrix Lambda of Eq. S_factored in the mode order of Y:
    entry (a k0 + i, b k0 + i) = Lambda_l[a, b] for the modes i of multipole l."""
    k0 = (lmax + 1) ** 2 - lmin ** 2
    nc = len(comps)
    lam = lambda_blocks(cl, comps, lmin, lmax)
    lm = _l_of_mode(lmin, lmax) - lmin
    L = np.zeros((nc * k0, nc * k0))
    idx = np.arange(k0)
    for a in range(nc):
        for b in range(nc):
            L[a * k0 + idx, b * k0 + idx] = lam[lm, a, b]
    return L


def qml_harmonic(Y, cl_fid, comps, lmin, lmax, N, spec, maps=None, want_bias=True, edges=None):
    """The same estimator in the harmonic basis (Sects. 2.3.2-2.3.3 with the
    stable evaluation of App. C.3), for the pixel-vs-harmonic cross-check.

    M = Y^T N^-1 Y (the noise-weighted Gramian), and with Lambda the fiducial
    spectrum matrix the projected inverse Y^T C^-1 Y = M - M K^-1 M,
    K = Lambda^-1 + M (Eqs. smw, K_kernel, projected_inv_smw), is evaluated
    without the subtraction as M (I + Lambda M)^-1 (Eq. smw_stable), one linear
    solve with (I + Lambda M)^T; the weighted data Y^T C^-1 d =
    (I + M Lambda)^-1 Y^T N^-1 d (Eq. smw_stable_data); the noise bias from
    Cov(w | noise) = A M A^T with A = (I + M Lambda)^-1 (Eq. smw_stable_A).
    With multipole switching N is N_eff (Sect. 2.3.4).
    """
    k = Y.shape[1]
    cN = sla.cho_factor(N, lower=True)
    NiY = sla.cho_solve(cN, Y)
    M = Y.T @ NiY
    M = 0.5 * (M + M.T)
    Lam = lambda_dense(cl_fid, comps, lmin, lmax)
    I = np.eye(k)
    W = np.linalg.solve((I + Lam @ M).T, M.T).T
    W = 0.5 * (W + W.T)
    F = fisher_from_W(W, spec, comps, lmin, lmax, edges)
    out = {"F": F, "W": W}
    A = np.linalg.inv(I + M @ Lam)
    if want_bias:
        out["b"] = 0.5 * trace_selector(A @ M @ A.T, spec, comps, lmin, lmax, edges)
    if maps is not None:
        maps = maps.reshape(maps.shape[0], -1)
        w = A @ (NiY.T @ maps)
        y = quad_selector(w, spec, comps, lmin, lmax, edges)
        out["w"] = w
        out["y"] = y
        if want_bias:
            q = y - out["b"][:, None]
            out["q"] = q
            dec, decor, conv, Fm12 = normalisations(F, q)
            out.update(cl_deconv=dec, cl_decorr=decor, q_conv=conv, F_inv_sqrt=Fm12)
    return out


def loglike_harmonic(Y, cl, comps, lmin, lmax, N, d):
    """lnL of Eq. pixel_likelihood through the determinant lemma and the SMW
    quadratic form (Eqs. logdet, quad_form_smw; App. C.2):
    ln|C| = ln|N| + ln|I + Lambda M|, d^T C^-1 d = d^T N^-1 d - v^T K^-1 v with
    v = Y^T N^-1 d and K^-1 = (Lambda^-1 + M)^-1 = Lambda (I + M Lambda)^-1.
    Returns (lnL, chi2, logdet) like loglike()."""
    d = d.reshape(d.shape[0], -1)
    cN = sla.cho_factor(N, lower=True)
    lnN = 2.0 * np.sum(np.log(np.abs(np.diag(cN[0]))))
    NiY = sla.cho_solve(cN, Y)
    M = Y.T @ NiY
    M = 0.5 * (M + M.T)
    Lam = lambda_dense(cl, comps, lmin, lmax)
    I = np.eye(Y.shape[1])
    sign, lnK = np.linalg.slogdet(I + Lam @ M)
    assert sign > 0
    v = NiY.T @ d
    dNd = np.sum(d * sla.cho_solve(cN, d), axis=0)
    chi2 = dNd - np.sum(v * (Lam @ np.linalg.solve(I + M @ Lam, v)), axis=0)
    logdet = lnN + lnK
    return -0.5 * (chi2 + logdet), chi2, logdet


def cross_qml(Y, cl_fid, comps, lmin, lmax, N1, N2, spec, d1=None, d2=None):
    """Cross-QML of two data sets on one pixel set, filtered independently
    (Eq. q_cross): q_x = 1/2 d1^T C1^-1 P_a C2^-1 d2 with C_i = S + N_i and
    the mode-mixing matrix W_x = 1/2 tr[C1^-1 P_a C2^-1 P_b]; in the harmonic
    factorisation (Sect. 2.3.3) with W_i = Y^T C_i^-1 Y, w_i = Y^T C_i^-1 d_i:
    W_x = 1/2 tr[W1 E_a W2 E_b], q_x = 1/2 w1^T E_a w2.  With independent noise
    there is no noise bias, and C_x = W_x^-1 q_x."""
    C1 = total_cov(Y, cl_fid, comps, lmin, lmax, N1)
    C2 = total_cov(Y, cl_fid, comps, lmin, lmax, N2)
    f1 = sla.cho_factor(C1, lower=True)
    f2 = sla.cho_factor(C2, lower=True)
    W1 = Y.T @ sla.cho_solve(f1, Y)
    W2 = Y.T @ sla.cho_solve(f2, Y)
    W1, W2 = 0.5 * (W1 + W1.T), 0.5 * (W2 + W2.T)
    out = {"Wx": fisher_from_W(W1, spec, comps, lmin, lmax, W2=W2), "C1": C1, "C2": C2}
    if d1 is not None:
        d1 = d1.reshape(d1.shape[0], -1)
        d2 = d2.reshape(d2.shape[0], -1)
        w1 = Y.T @ sla.cho_solve(f1, d1)
        w2 = Y.T @ sla.cho_solve(f2, d2)
        out["q"] = quad_selector(w1, spec, comps, lmin, lmax, w2=w2)
        out["cl_deconv"] = np.linalg.solve(out["Wx"], out["q"])
    return out


def window_columns(lsig0: int, lsig1: int, lmin: int, lmax: int, nc: int):
    """Columns of a Y built over [lsig0, lsig1] (nc blocks of modes, l-major)
    whose multipole lies in the window [lmin, lmax], below it and above it."""
    k0s = (lsig1 + 1) ** 2 - lsig0 ** 2

    def modes(l0, l1):  # multipoles l0 .. l1 - 1 of every block
        return np.concatenate([np.arange(c * k0s + l0 * l0 - lsig0 * lsig0,
                                         c * k0s + l1 * l1 - lsig0 * lsig0) for c in range(nc)])
    return modes(lmin, lmax + 1), modes(lsig0, lmin), modes(lmax + 1, lsig1 + 1)


def switched(Y_sig, cl_fid, comps, lsig, lmin, lmax, N, spec, maps=None, want_bias=True,
             edges=None):
    """Multipole switching (Sect. 2.3.4, Eqs. C_switched, N_eff).

    Y_sig spans the signal range lsig = (lmin_sig, lmax_sig); the spectrum is
    estimated on the inference window [lmin, lmax] only, the fiducial signal
    of the multipoles on either side is absorbed into
        N_eff = N + sum_{l in [lmin_sig, lmin) u (lmax, lmax_sig]} C_l^fid P_l
    (one transfer factor, already in P_l), and N_eff takes the place of N
    throughout: C = Y_inf Lambda_inf Y_inf^T + N_eff and the noise bias is
    1/2 tr[C^-1 P_l C^-1 N_eff].
    """
    lsig0, lsig1 = lsig
    win, low, high = window_columns(lsig0, lsig1, lmin, lmax, len(comps))
    Neff = N.copy()
    if lmin > lsig0:
        Neff = Neff + signal_cov(Y_sig[:, low], cl_fid, comps, lsig0, lmin - 1)
    if lsig1 > lmax:
        Neff = Neff + signal_cov(Y_sig[:, high], cl_fid, comps, lmax + 1, lsig1)
    out = qml(Y_sig[:, win], cl_fid, comps, lmin, lmax, Neff, spec, maps, want_bias, edges)
    out["N_eff"] = Neff
    return out


def bin_matrix(nspec: int, lmin: int, lmax: int, edges) -> np.ndarray:
    """P_Sigma: the 0/1 matrix summing each spectrum's multipoles into its bins
    (nspec nb x nspec nl, spectrum-major), for the identity of Sect. 3 (check
    of the binned path): F_bin = P_Sigma F P_Sigma^T, q_b = sum_{l in b} q_l."""
    nl, nb = lmax - lmin + 1, len(edges) - 1
    P = np.zeros((nspec * nb, nspec * nl))
    for s in range(nspec):
        for b in range(nb):
            P[s * nb + b, s * nl + edges[b] - lmin:s * nl + edges[b + 1] - lmin] = 1.0
    return P


def simulate(Y: np.ndarray, alm: np.ndarray, noise: np.ndarray) -> np.ndarray:
    """d = Y a + n (Eq. data_model with s = Y a)."""
    return Y @ alm + noise
