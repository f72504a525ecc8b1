"""Pins for the oracle's Fisher matrix, noise bias, estimates and likelihood.

P1 brute force, P2 exact closed form on a quadrature grid, P6 symmetry and
positive definiteness, P7 the expectation identity <q> = F C, P8 Monte Carlo
unbiasedness, P9 decorrelation.  Mutation tests plant a mistake in the oracle
(on the CPU) and check that a pin catches it.
"""
import math

import numpy as np
import pytest

from oracle import brute, harmonic, qml
from paper_2605_21149_gb300 import synth


def _tiny(has_T=True, has_P=True, nside=2, lmax=5, b0=20.0, cross=True, seed=1):
    th, ph, z = synth.healpix_ring_centres(nside)
    keep = synth.galactic_cut(z, b0)
    th, ph = th[keep], ph[keep]
    tl = synth.transfer(lmax, nside)
    cl = synth.spectra(lmax)
    if cross:
        cl[4, 2:] = 0.02
        cl[5, 2:] = 0.003
    comps = ((0,) if has_T else ()) + ((1, 2) if has_P else ())
    spec = tuple(s for s, (x, y) in enumerate(qml.SPEC_PAIRS) if x in comps and y in comps)
    Y = harmonic.build_Y(2, lmax, th, ph, th, ph, tl, tl, has_T, has_P)
    n = Y.shape[0]
    g = np.random.default_rng(seed)
    G = g.normal(size=(n, 5)) * 0.3
    N = G @ G.T + np.eye(n)
    d = g.normal(size=(n, 3))
    return dict(th=th, ph=ph, tl=tl, cl=cl, comps=comps, spec=spec, Y=Y, N=N, d=d,
                lmax=lmax, has_T=has_T, has_P=has_P)


@pytest.mark.parametrize("has_T,has_P", [(True, False), (False, True), (True, True)])
def test_P1_harmonic_vs_brute(has_T, has_P):
    t = _tiny(has_T, has_P)
    r = qml.qml(t["Y"], t["cl"], t["comps"], 2, t["lmax"], t["N"], t["spec"], maps=t["d"])
    Ps = brute.pixel_derivatives(t["th"], t["ph"], t["th"], t["ph"], t["tl"], t["tl"],
                                 has_T, has_P, 2, t["lmax"], t["spec"])
    rb = brute.qml_dense(Ps, r["C"], t["N"], maps=t["d"])
    for key in ("F", "b", "y"):
        assert np.abs(r[key] - rb[key]).max() <= 1e-12 * np.abs(rb[key]).max(), key
    lnl, chi2, logdet = qml.loglike(r["C"], t["d"])
    assert np.allclose(lnl, rb["lnL"], rtol=1e-12, atol=0)
    assert np.allclose(chi2, rb["chi2"], rtol=1e-12, atol=0)


def _closed_form(cl, tl, sigma2, spec, comps, lmin, lmax):
    """Per-l 3x3 closed forms on an exact quadrature grid (P2)."""
    nl = lmax - lmin + 1
    na = len(spec) * nl
    F = np.zeros((na, na))
    b = np.zeros(na)
    logdet_sig = 0.0
    for il, l in enumerate(range(lmin, lmax + 1)):
        lam = qml.lambda_blocks(cl, comps, lmin, lmax)[il]
        D = np.diag([tl[l]] * len(comps))
        Cl = D @ lam @ D + sigma2 * np.eye(len(comps))
        Ci = np.linalg.inv(Cl)
        dC = []
        for s in spec:
            x, y = qml.SPEC_PAIRS[s]
            E = np.zeros((len(comps), len(comps)))
            E[comps.index(x), comps.index(y)] = 1
            E[comps.index(y), comps.index(x)] = 1
            dC.append(D @ E @ D)
        for A in range(len(spec)):
            for B in range(len(spec)):
                F[A * nl + il, B * nl + il] = 0.5 * (2 * l + 1) * np.trace(Ci @ dC[A] @ Ci @ dC[B])
            b[A * nl + il] = 0.5 * (2 * l + 1) * sigma2 * np.trace(Ci @ Ci @ dC[A])
        logdet_sig += (2 * l + 1) * np.linalg.slogdet(np.eye(len(comps)) + D @ lam @ D / sigma2)[1]
    return F, b, logdet_sig


@pytest.mark.parametrize("has_T,has_P", [(True, False), (False, True), (True, True)])
def test_P2_quadrature_closed_form(has_T, has_P):
    """On a full-sky Gauss-Legendre grid with N = diag(sigma^2 / w_p) the harmonic
    Gram matrix is exactly I/sigma^2, so F, b and ln|C| take per-l closed forms:
      F^l_ab = (2l+1)/2 tr[Cl^-1 dCl_a Cl^-1 dCl_b],  b^l_a = (2l+1)/2 sigma^2 tr[Cl^-2 dCl_a],
      ln|C| = sum_p ln(sigma^2/w_p) + sum_l (2l+1) ln|I + T Cl T / sigma^2|,
    with Cl = T Chat_l T + sigma^2 I (3x3 over the fields present)."""
    lmin, lmax = 2, 7
    th, ph, w = synth.gauss_legendre_grid(lmax)
    tl = synth.gaussian_beam(lmax, 0.25)
    cl = synth.spectra(lmax)
    cl[4, 2:] = 0.03
    cl[5, 2:] = 0.002
    comps = ((0,) if has_T else ()) + ((1, 2) if has_P else ())
    spec = tuple(s for s, (x, y) in enumerate(qml.SPEC_PAIRS) if x in comps and y in comps)
    Y = harmonic.build_Y(lmin, lmax, th, ph, th, ph, tl, tl, has_T, has_P)
    sigma2 = 0.7
    wt = np.concatenate([w] * len(comps)) if has_T else np.concatenate([w, w])
    if has_T and has_P:
        wt = np.concatenate([w, w, w])
    N = np.diag(sigma2 / wt)
    r = qml.qml(Y, cl, comps, lmin, lmax, N, spec)
    Fc, bc, lds = _closed_form(cl, tl, sigma2, spec, comps, lmin, lmax)
    assert np.abs(r["F"] - Fc).max() <= 1e-12 * np.abs(Fc).max()
    assert np.abs(r["b"] - bc).max() <= 1e-12 * np.abs(bc).max()
    d = np.random.default_rng(3).normal(size=(Y.shape[0], 2))
    lnl, chi2, logdet = qml.loglike(r["C"], d)
    ref = np.sum(np.log(sigma2 / wt)) + lds
    assert abs(logdet - ref) <= 1e-12 * abs(ref)


def test_P6_P7_P9_invariants():
    """F symmetric positive definite (P6); 1/2 tr[C^-1 P_a] = (F C_fid)_a + b_a
    (P7, exact because C = sum_b C_b P_b + N); F^-1/2 F F^-1/2 = I (P9)."""
    t = _tiny(True, True, nside=4, lmax=9, cross=False)
    r = qml.qml(t["Y"], t["cl"], t["comps"], 2, t["lmax"], t["N"], t["spec"], maps=t["d"])
    F = r["F"]
    assert np.abs(F - F.T).max() <= 1e-14 * np.abs(F).max()
    assert np.linalg.eigvalsh(F).min() > 0
    nl = t["lmax"] - 1
    cfid = np.concatenate([t["cl"][s, 2:t["lmax"] + 1] for s in t["spec"]])
    lhs = 0.5 * qml.trace_selector(r["W"], t["spec"], t["comps"], 2, t["lmax"])
    rhs = F @ cfid + r["b"]
    assert np.abs(lhs - rhs).max() <= 1e-10 * np.abs(lhs).max()
    M = r["F_inv_sqrt"] @ F @ r["F_inv_sqrt"]
    assert np.abs(M - np.eye(len(F))).max() < 1e-10


@pytest.mark.slow
def test_P8_unbiased_monte_carlo():
    """Mean of deconvolved Cl over 1000 seeded sims is within 4 sigma/sqrt(N)
    of the fiducial for every (spectrum, l); the scatter matches F^-1 (P8)."""
    wl = synth.workload(0)
    Y = harmonic.build_Y_for(wl)
    nsims = 1000
    g = synth.rng(0, synth.P_SIMS)
    alm = synth.draw_alm(wl.cl_fid, wl.lmin, wl.lmax, wl.comps, nsims, g)
    noise = synth.noise_draws(wl.G, nsims, g)
    d = qml.simulate(Y, alm, noise)
    r = qml.qml_for(wl, Y, maps=d)
    chat = r["cl_deconv"]
    Finv = np.linalg.inv(r["F"])
    sig = np.sqrt(np.diag(Finv))
    cfid = np.concatenate([wl.cl_fid[s, wl.lmin:wl.lmax + 1] for s in wl.spec])
    z = (chat.mean(axis=1) - cfid) / (sig / math.sqrt(nsims))
    assert np.all(np.abs(z) < 4.0)
    ratio = chat.std(axis=1) / sig
    assert np.all((ratio > 0.85) & (ratio < 1.15))


# ---------------------------------------------------------------------------
# mutation tests: plant a mistake in the oracle and check a pin fails
# ---------------------------------------------------------------------------
def test_mutation_eb_sign_is_caught(monkeypatch):
    """Flipping the sign of the E combination (Eq. EB_from_spin) in the real
    basis flips TE/TB: the brute-force pin P1 must notice."""
    t = _tiny(True, True)
    orig = harmonic.theta_functions

    def flipped(l, theta):
        lam, F1, F2 = orig(l, theta)
        return lam, -F1, -F2

    monkeypatch.setattr(harmonic, "theta_functions", flipped)
    Y = harmonic.build_Y(2, t["lmax"], t["th"], t["ph"], t["th"], t["ph"], t["tl"], t["tl"], True, True)
    S = qml.signal_cov(Y, t["cl"], t["comps"], 2, t["lmax"])
    Ps = brute.pixel_derivatives(t["th"], t["ph"], t["th"], t["ph"], t["tl"], t["tl"],
                                 True, True, 2, t["lmax"], t["spec"])
    Sb = brute.signal_from_derivatives(Ps, t["cl"], t["spec"], 2, t["lmax"])
    assert np.abs(S - Sb).max() > 1e-3 * np.abs(S).max()


def test_mutation_dropped_cross_pair_is_caught(monkeypatch):
    """Dropping the (Y,X) half of a cross-spectrum selector breaks P2."""
    monkeypatch.setattr(qml, "pairs", lambda s: [qml.SPEC_PAIRS[s]])
    lmin, lmax = 2, 5
    th, ph, w = synth.gauss_legendre_grid(lmax)
    tl = np.ones(lmax + 1)
    cl = synth.spectra(lmax)
    comps = (0, 1, 2)
    spec = tuple(range(6))
    Y = harmonic.build_Y(lmin, lmax, th, ph, th, ph, tl, tl, True, True)
    N = np.diag(0.5 / np.concatenate([w, w, w]))
    r = qml.qml(Y, cl, comps, lmin, lmax, N, spec)
    Fc, _, _ = _closed_form(cl, tl, 0.5, spec, comps, lmin, lmax)
    assert np.abs(r["F"] - Fc).max() > 1e-3 * np.abs(Fc).max()


# ---- P10: native multipole binning (Sect. 2.4) ---------------------------
BIN_EDGES = {2: [2, 4, 6], 3: [2, 5, 6], 5: [2, 6], "ragged": [2, 3, 6]}  # lmax = 5


@pytest.mark.parametrize("dl", [2, 3, 5, "ragged"])
def test_P10_binning_identity(dl):
    """The check of the binned path (Sect. 3): F_bin = P_Sigma F P_Sigma^T and
    q_b = sum_{l in b} q_l (likewise the noise bias) to machine precision, the
    binned side computed with the bin selectors E_b = sum_{l in b} E_l."""
    t = _tiny()
    edges = np.array(BIN_EDGES[dl])
    r = qml.qml(t["Y"], t["cl"], t["comps"], 2, t["lmax"], t["N"], t["spec"], maps=t["d"])
    rb = qml.qml(t["Y"], t["cl"], t["comps"], 2, t["lmax"], t["N"], t["spec"], maps=t["d"],
                 edges=edges)
    P = qml.bin_matrix(len(t["spec"]), 2, t["lmax"], edges)
    assert np.abs(rb["F"] - P @ r["F"] @ P.T).max() <= 1e-13 * np.abs(rb["F"]).max()
    for key in ("y", "b", "q"):
        ref = P @ r[key]
        assert np.abs(rb[key] - ref).max() <= 1e-13 * np.abs(ref).max(), key
    # the normalisations act on the binned F: F_b C_b^deconv = q_b
    assert np.abs(rb["F"] @ rb["cl_deconv"] - rb["q"]).max() <= 1e-10 * np.abs(rb["q"]).max()


def test_P10_binning_vs_brute():
    """Binned F, noise bias and y against dense pixel traces with the bin
    derivative P_b = sum_{l in b} P_l built from the brute-force responses
    (independent of the harmonic selectors)."""
    t = _tiny()
    edges = np.array(BIN_EDGES[2])
    rb = qml.qml(t["Y"], t["cl"], t["comps"], 2, t["lmax"], t["N"], t["spec"], maps=t["d"],
                 edges=edges)
    Ps = brute.pixel_derivatives(t["th"], t["ph"], t["th"], t["ph"], t["tl"], t["tl"],
                                 True, True, 2, t["lmax"], t["spec"])
    nl = t["lmax"] - 1
    Pb = [sum(Ps[s * nl + l - 2] for l in range(edges[b], edges[b + 1]))
          for s in range(len(t["spec"])) for b in range(len(edges) - 1)]
    ref = brute.qml_dense(Pb, rb["C"], t["N"], maps=t["d"])
    for key in ("F", "b", "y"):
        assert np.abs(rb[key] - ref[key]).max() <= 1e-12 * np.abs(ref[key]).max(), key


def test_P10_unit_bins_are_per_l():
    """Bins of one multipole reproduce the per-l estimator (the single code
    path of Sect. 2.4 with Delta l = 1)."""
    t = _tiny(has_P=False)
    r = qml.qml(t["Y"], t["cl"], t["comps"], 2, t["lmax"], t["N"], t["spec"], maps=t["d"])
    rb = qml.qml(t["Y"], t["cl"], t["comps"], 2, t["lmax"], t["N"], t["spec"], maps=t["d"],
                 edges=np.arange(2, t["lmax"] + 2))
    for key in ("F", "b", "y", "cl_deconv", "cl_decorr"):
        assert np.array_equal(rb[key], r[key]), key


def test_mutation_bin_range_off_by_one_is_caught(monkeypatch):
    """Starting every bin's mode range one multipole late (a plausible index
    slip in E_b) breaks the brute-force binning pin."""
    orig = qml.mode_starts

    def late(lmin, lmax, edges=None):
        if edges is None:
            return orig(lmin, lmax)
        shifted = np.array([e + 1 if 0 < i < len(edges) - 1 else e for i, e in enumerate(edges)])
        return orig(lmin, lmax, shifted)

    monkeypatch.setattr(qml, "mode_starts", late)
    with pytest.raises(AssertionError):
        test_P10_binning_vs_brute()


# ---- P17: multipole switching (Sect. 2.3.4, Eqs. C_switched, N_eff) -------
def _switch_setup():
    """Signal over l = 2..7, inference window l = 3..5 (one multipole fixed
    below it, two above), TQU with all six spectra."""
    t = _tiny(nside=2, lmax=7)
    lsig, lmin, lmax = (2, 7), 3, 5
    rs = qml.switched(t["Y"], t["cl"], t["comps"], lsig, lmin, lmax, t["N"], t["spec"],
                      maps=t["d"])
    rf = qml.qml(t["Y"], t["cl"], t["comps"], 2, 7, t["N"], t["spec"], maps=t["d"])
    nlf = 6
    win = np.array([s * nlf + l - 2 for s in range(len(t["spec"])) for l in range(lmin, lmax + 1)])
    out = np.array([s * nlf + l - 2 for s in range(len(t["spec"]))
                    for l in list(range(2, lmin)) + list(range(lmax + 1, 8))])
    return t, rs, rf, win, out


def test_P17_switching_is_the_window_of_the_full_estimator():
    """C is the same matrix with or without switching, so F and y on the
    window equal the window blocks of the full-range estimator, and the noise
    bias (with N_eff) gains exactly the fixed signal's share:
    b_sw = b_full[win] + F_full[win, out] C_fid[out]."""
    t, rs, rf, win, out = _switch_setup()
    assert np.abs(rs["C"] - rf["C"]).max() <= 1e-13 * np.abs(rf["C"]).max()
    Ff = rf["F"][np.ix_(win, win)]
    assert np.abs(rs["F"] - Ff).max() <= 1e-11 * np.abs(Ff).max()
    assert np.abs(rs["y"] - rf["y"][win]).max() <= 1e-11 * np.abs(rf["y"][win]).max()
    cfid = np.concatenate([t["cl"][s, 2:8] for s in t["spec"]])
    bref = rf["b"][win] + rf["F"][np.ix_(win, out)] @ cfid[out]
    assert np.abs(rs["b"] - bref).max() <= 1e-11 * np.abs(bref).max()


def test_P17_switching_expectation_identity():
    """1/2 tr[C^-1 P_a] = (F C_fid)_a + b_a on the window (P7 with N_eff):
    exact, because C = sum_{a in window} C_a P_a + N_eff."""
    t, rs, rf, win, out = _switch_setup()
    cwin = np.concatenate([t["cl"][s, 3:6] for s in t["spec"]])
    lhs = 0.5 * qml.trace_selector(rs["W"], t["spec"], t["comps"], 3, 5)
    assert np.abs(lhs - (rs["F"] @ cwin + rs["b"])).max() <= 1e-10 * np.abs(lhs).max()


def test_P17_neff_vs_brute():
    """N_eff built from the dense pixel derivatives P_l of the brute-force
    responses (Eq. N_eff term by term), independent of Y."""
    t, rs, rf, win, out = _switch_setup()
    Ps = brute.pixel_derivatives(t["th"], t["ph"], t["th"], t["ph"], t["tl"], t["tl"],
                                 True, True, 2, 7, tuple(range(6)))
    Neff = t["N"].copy()
    for s in range(6):
        for l in (2, 6, 7):
            Neff = Neff + t["cl"][s, l] * Ps[s * 6 + l - 2]
    assert np.abs(rs["N_eff"] - Neff).max() <= 1e-12 * np.abs(Neff).max()


def test_P17_no_switching_is_plain_qml():
    """A signal range equal to the window leaves N_eff = N: plain QML (up to
    the rounding of products over a copied Y)."""
    t = _tiny(has_P=False)
    r = qml.qml(t["Y"], t["cl"], t["comps"], 2, t["lmax"], t["N"], t["spec"], maps=t["d"])
    rs = qml.switched(t["Y"], t["cl"], t["comps"], (2, t["lmax"]), 2, t["lmax"], t["N"],
                      t["spec"], maps=t["d"])
    assert np.array_equal(rs["N_eff"], t["N"])
    for key in ("F", "b", "y", "cl_deconv"):
        assert np.abs(rs[key] - r[key]).max() <= 1e-13 * np.abs(r[key]).max(), key


def test_mutation_switching_drops_high_side_is_caught(monkeypatch):
    """Absorbing only the multipoles below the window (a dropped term of
    Eq. N_eff) breaks the brute-force pin."""
    orig = qml.signal_cov

    def no_high(Y, cl, comps, lmin, lmax):
        S = orig(Y, cl, comps, lmin, lmax)
        return 0.0 * S if lmin == 6 else S  # the term above the window l = 3..5

    monkeypatch.setattr(qml, "signal_cov", no_high)
    with pytest.raises(AssertionError):
        test_P17_neff_vs_brute()


# ---- P16: cross-QML (Eq. q_cross) -----------------------------------------
def _cross_setup():
    t = _tiny()
    g = np.random.default_rng(21)
    n = t["Y"].shape[0]
    G2 = g.normal(size=(n, 4)) * 0.4
    N2 = G2 @ G2.T + 1.5 * np.eye(n)
    d2 = g.normal(size=(n, 3))
    return t, N2, d2


def test_P16_cross_reduces_to_auto():
    """Equal noise and equal maps: W_x is the Fisher matrix and q_x the
    bias-free auto estimate y."""
    t = _tiny()
    r = qml.qml(t["Y"], t["cl"], t["comps"], 2, t["lmax"], t["N"], t["spec"], maps=t["d"])
    x = qml.cross_qml(t["Y"], t["cl"], t["comps"], 2, t["lmax"], t["N"], t["N"], t["spec"],
                      t["d"], t["d"])
    assert np.abs(x["Wx"] - r["F"]).max() <= 1e-13 * np.abs(r["F"]).max()
    assert np.abs(x["q"] - r["y"]).max() <= 1e-13 * np.abs(r["y"]).max()


def test_P16_cross_vs_brute():
    """W_x and q_x against dense pixel traces with the brute-force P_a."""
    t, N2, d2 = _cross_setup()
    x = qml.cross_qml(t["Y"], t["cl"], t["comps"], 2, t["lmax"], t["N"], N2, t["spec"],
                      t["d"], d2)
    Ps = brute.pixel_derivatives(t["th"], t["ph"], t["th"], t["ph"], t["tl"], t["tl"],
                                 True, True, 2, t["lmax"], t["spec"])
    S = brute.signal_from_derivatives(Ps, t["cl"], t["spec"], 2, t["lmax"])
    C1i, C2i = np.linalg.inv(S + t["N"]), np.linalg.inv(S + N2)  # built here, not by the oracle
    na = len(Ps)
    Wx = np.array([[0.5 * np.trace(C1i @ Ps[a] @ C2i @ Ps[b]) for b in range(na)]
                   for a in range(na)])
    q = np.array([0.5 * np.sum((C1i @ t["d"]) * (Ps[a] @ (C2i @ d2)), axis=0) for a in range(na)])
    assert np.abs(x["Wx"] - Wx).max() <= 1e-12 * np.abs(Wx).max()
    assert np.abs(x["q"] - q).max() <= 1e-12 * np.abs(q).max()


def test_P16_cross_is_unbiased_exactly():
    """With independent noise the cross-covariance of the two maps is S, so
    <q_x> = 1/2 tr[C1^-1 P_a C2^-1 S] = W_x C_fid exactly (no noise bias)."""
    t, N2, d2 = _cross_setup()
    x = qml.cross_qml(t["Y"], t["cl"], t["comps"], 2, t["lmax"], t["N"], N2, t["spec"])
    Ps = brute.pixel_derivatives(t["th"], t["ph"], t["th"], t["ph"], t["tl"], t["tl"],
                                 True, True, 2, t["lmax"], tuple(range(6)))
    S = brute.signal_from_derivatives(Ps, t["cl"], tuple(range(6)), 2, t["lmax"])
    C1i, C2i = np.linalg.inv(x["C1"]), np.linalg.inv(x["C2"])
    nl = t["lmax"] - 1
    mean = np.array([0.5 * np.trace(C1i @ Ps[s * nl + l] @ C2i @ S)
                     for s in t["spec"] for l in range(nl)])
    cfid = np.concatenate([t["cl"][s, 2:t["lmax"] + 1] for s in t["spec"]])
    assert np.abs(mean - x["Wx"] @ cfid).max() <= 1e-11 * np.abs(mean).max()


def test_mutation_cross_filters_both_with_C1_is_caught(monkeypatch):
    """Filtering the second map with C1 (the two-filter structure lost) breaks
    the brute-force cross pin."""
    orig = qml.total_cov
    first = {}

    def same(Y, cl, comps, lmin, lmax, N):
        first.setdefault("N", N)
        return orig(Y, cl, comps, lmin, lmax, first["N"])

    monkeypatch.setattr(qml, "total_cov", same)
    with pytest.raises(AssertionError):
        test_P16_cross_vs_brute()


# ---- P11: harmonic basis (SMW) against the pixel basis (Sects. 2.3.2-2.3.3,
# App. C.2-C.3); the paper's own cross-check agrees to ~1e-13 on F ---------
@pytest.mark.parametrize("has_T,has_P", [(True, False), (False, True), (True, True)])
def test_P11_harmonic_basis_equals_pixel_basis(has_T, has_P):
    """F, b, y and the three normalisations from the SMW stable form equal the
    pixel-basis definition (C factored directly), all six spectra with non-zero
    TB and EB; and lnL through the determinant lemma equals the Cholesky
    log-likelihood."""
    t = _tiny(has_T, has_P, nside=4, lmax=7)
    rp = qml.qml(t["Y"], t["cl"], t["comps"], 2, t["lmax"], t["N"], t["spec"], maps=t["d"])
    rh = qml.qml_harmonic(t["Y"], t["cl"], t["comps"], 2, t["lmax"], t["N"], t["spec"],
                          maps=t["d"])
    for key in ("F", "b", "y", "cl_deconv", "q_conv"):
        assert np.abs(rh[key] - rp[key]).max() <= 1e-11 * np.abs(rp[key]).max(), key
    lp = qml.loglike(rp["C"], t["d"])
    lh = qml.loglike_harmonic(t["Y"], t["cl"], t["comps"], 2, t["lmax"], t["N"], t["d"])
    for a, b in zip(lh, lp):
        assert np.abs(np.asarray(a) - np.asarray(b)).max() <= 1e-11 * np.abs(np.asarray(b)).max()


def test_P11_harmonic_basis_high_signal_to_noise():
    """Noise scaled down by 1e9 (the cosmic-variance-limited regime of
    App. C.3): the stable form keeps F within 1e-11 of the pixel basis, while
    the subtractive form M - M K^-1 M loses digits to cancellation."""
    t = _tiny(True, True, nside=4, lmax=7)
    N = t["N"] * 1e-9
    rp = qml.qml(t["Y"], t["cl"], t["comps"], 2, t["lmax"], N, t["spec"])
    rh = qml.qml_harmonic(t["Y"], t["cl"], t["comps"], 2, t["lmax"], N, t["spec"])
    assert np.abs(rh["F"] - rp["F"]).max() <= 1e-11 * np.abs(rp["F"]).max()
    # the subtractive form on the same inputs
    M = t["Y"].T @ np.linalg.solve(N, t["Y"])
    Lam = qml.lambda_dense(t["cl"], t["comps"], 2, t["lmax"])
    K = np.linalg.inv(Lam) + M
    Wsub = M - M @ np.linalg.solve(K, M)
    Fsub = qml.fisher_from_W(0.5 * (Wsub + Wsub.T), t["spec"], t["comps"], 2, t["lmax"])
    assert np.abs(Fsub - rp["F"]).max() > 100 * np.abs(rh["F"] - rp["F"]).max()


def test_P11_harmonic_with_switching_equals_switched_pixel():
    """With N_eff in place of N (Sect. 2.3.4) the harmonic basis on the window
    modes reproduces the switched pixel-basis estimator."""
    t, rs, rf, win, out = _switch_setup()
    wcols, lo, hi = qml.window_columns(2, 7, 3, 5, len(t["comps"]))
    rh = qml.qml_harmonic(t["Y"][:, wcols], t["cl"], t["comps"], 3, 5, rs["N_eff"], t["spec"],
                          maps=t["d"])
    for key in ("F", "b", "y", "cl_deconv"):
        assert np.abs(rh[key] - rs[key]).max() <= 1e-11 * np.abs(rs[key]).max(), key


def test_mutation_harmonic_lambda_transposed_is_caught(monkeypatch):
    """Using (I + M Lambda) where the stable form needs (I + Lambda M) for the
    projected inverse changes F once Lambda has off-diagonal (TE, TB, EB)
    entries; the pixel-basis pin catches it."""
    orig = qml.lambda_dense

    def skewed(cl, comps, lmin, lmax):
        L = orig(cl, comps, lmin, lmax)
        return np.triu(L) + 0.5 * np.tril(L, -1)   # not the symmetric Lambda

    monkeypatch.setattr(qml, "lambda_dense", skewed)
    with pytest.raises(AssertionError):
        test_P11_harmonic_basis_equals_pixel_basis(True, True)
