"""Pins for the oracle's real harmonic matrix Y (Sect. 2.3.1, App. A)."""
import math

import numpy as np
import pytest

from oracle import brute, harmonic, qml
from paper_2605_21149_gb300 import synth


def _gl(lmax):
    return synth.gauss_legendre_grid(lmax)


@pytest.mark.parametrize("lmax", [4, 12])
def test_orthonormal_under_exact_quadrature(lmax):
    """P13: Y^T diag(w) Y = I on a Gauss-Legendre grid that integrates every
    product of band-limited (spin-0 and spin-2) harmonics exactly."""
    th, ph, w = _gl(lmax + 1)
    one = np.ones(lmax + 1)
    Y = harmonic.build_Y(2, lmax, th, ph, th, ph, one, one, True, True)
    wt = np.concatenate([w, w, w])
    G = Y.T @ (wt[:, None] * Y)
    assert np.abs(G - np.eye(G.shape[0])).max() < 1e-13


def test_spin0_addition_theorem():
    """P4: Y Lambda Y^T of the T block equals the Legendre sum of Eq. signal_cov."""
    th, ph, z = synth.healpix_ring_centres(4)
    keep = synth.galactic_cut(z, 30.0)
    th, ph = th[keep], ph[keep]
    lmin, lmax = 2, 11
    tl = synth.transfer(lmax, 4)
    cl = synth.spectra(lmax)
    Y = harmonic.build_Y(lmin, lmax, th, ph, th, ph, tl, tl, True, False)
    S = qml.signal_cov(Y, cl, (0,), lmin, lmax)
    ref = sum(cl[0, l] * brute.legendre_sum_TT(th, ph, tl, l) for l in range(lmin, lmax + 1))
    assert np.abs(S - ref).max() < 1e-13 * np.abs(ref).max() * 10


def test_spin2_pointwise_invariants():
    """P5: at p = p', S_QQ + S_UU = sum (2l+1)/4pi T^2 (EE+BB); S_QU = 0 when
    EB = 0; S_TQ = S_TU = 0 (spin addition theorem: sum_m s1Y* s2Y = delta)."""
    th, ph, z = synth.healpix_ring_centres(8)
    keep = synth.galactic_cut(z, 20.0)[::7]
    th, ph = th[keep], ph[keep]
    lmin, lmax = 2, 20
    tl = synth.transfer(lmax, 8)
    cl = synth.spectra(lmax)
    Y = harmonic.build_Y(lmin, lmax, th, ph, th, ph, tl, tl, True, True)
    S = qml.signal_cov(Y, cl, (0, 1, 2), lmin, lmax)
    n = len(th)
    dq = np.diag(S[n:2 * n, n:2 * n]) + np.diag(S[2 * n:, 2 * n:])
    ell = np.arange(lmin, lmax + 1)
    ref = np.sum((2 * ell + 1) / (4 * math.pi) * tl[lmin:] ** 2 * (cl[1, lmin:] + cl[2, lmin:]))
    assert np.allclose(dq, ref, rtol=1e-13, atol=0)
    assert np.abs(np.diag(S[n:2 * n, 2 * n:])).max() < 1e-14 * ref
    assert np.abs(np.diag(S[:n, n:2 * n])).max() < 1e-14 * ref
    assert np.abs(np.diag(S[:n, 2 * n:])).max() < 1e-14 * ref
    # T variance
    reft = np.sum((2 * ell + 1) / (4 * math.pi) * tl[lmin:] ** 2 * cl[0, lmin:])
    assert np.allclose(np.diag(S[:n, :n]), reft, rtol=1e-13, atol=0)


def test_spin2_matches_complex_pair_sums():
    """P1 (signal part): Y Lambda Y^T equals the complex spin-weighted synthesis
    of oracle.brute (factorial-sum d, explicit m < 0 terms) for all six spectra,
    including non-zero TB and EB, whose sign the E/B convention of
    Eq. EB_from_spin fixes."""
    th, ph, z = synth.healpix_ring_centres(2)
    lmin, lmax = 2, 6
    tl = synth.transfer(lmax, 2)
    cl = synth.spectra(lmax)
    cl[4, 2:] = 0.07
    cl[5, 2:] = -0.01
    Y = harmonic.build_Y(lmin, lmax, th, ph, th, ph, tl, tl, True, True)
    S = qml.signal_cov(Y, cl, (0, 1, 2), lmin, lmax)
    Ps = brute.pixel_derivatives(th, ph, th, ph, tl, tl, True, True, lmin, lmax, tuple(range(6)))
    Sb = brute.signal_from_derivatives(Ps, cl, tuple(range(6)), lmin, lmax)
    assert np.abs(S - Sb).max() < 1e-13 * np.abs(S).max()


def test_layout_component_blocks():
    """T columns vanish on Q/U rows and E/B columns vanish on T rows (Eq. V_multifield)."""
    th, ph, _ = synth.healpix_ring_centres(2)
    Y = harmonic.build_Y(2, 5, th, ph, th, ph, np.ones(6), np.ones(6), True, True)
    n, k0 = len(th), 32
    assert Y.shape == (3 * n, 3 * k0)
    assert np.all(Y[n:, :k0] == 0) and np.all(Y[:n, k0:] == 0)
