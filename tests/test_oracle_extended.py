"""Pins of oracle/extended.py (the decorrelated normalisation, Eq. decorrelated,
evaluated in long double): an exact closed form, an arbitrary-precision
reference where mpmath is installed, and the oracle's float64 result."""
import numpy as np
import pytest

from oracle import extended, qml
from paper_2605_21149_gb300 import synth

EPS_LD = float(np.finfo(np.longdouble).eps)


def _shear_block(k):
    """F = M^T M with M = [[1, k], [0, 1]]: integer entries, det F = 1,
    kappa ~ k^4, and F^-1/2 = [[k^2 + 2, -k], [-k, 2]] / sqrt(k^2 + 4) exactly
    (F + I = [[2, k], [k, k^2 + 2]], det(F + I) = k^2 + 4, and for 2 x 2 SPD
    matrices F^1/2 = (F + sqrt(det F) I) / sqrt(tr F + 2 sqrt(det F)))."""
    F = np.array([[1.0, k], [k, k * k + 1.0]])
    kl = np.longdouble(k)
    Z = np.array([[kl * kl + 2, -kl], [-kl, np.longdouble(2)]], dtype=np.longdouble)
    return F, Z / np.sqrt(kl * kl + 4)


def test_closed_form_shear_blocks():
    """Block-diagonal F of shear blocks (kappa up to 1.6e9), rows and columns
    permuted: the long-double result matches the exact F^-1/2 q far below the
    float64 error eps kappa / 2."""
    ks = [200.0, 57.0, 3.0, 120.0]
    n = 2 * len(ks)
    F = np.zeros((n, n))
    Zx = np.zeros((n, n), dtype=np.longdouble)
    for i, k in enumerate(ks):
        Fb, Zb = _shear_block(k)
        F[2 * i:2 * i + 2, 2 * i:2 * i + 2] = Fb
        Zx[2 * i:2 * i + 2, 2 * i:2 * i + 2] = Zb
    perm = np.random.default_rng(1).permutation(n)
    F = F[np.ix_(perm, perm)]
    Zx = Zx[np.ix_(perm, perm)]
    q = np.random.default_rng(2).normal(size=(n, 3))
    exact = Zx @ q.astype(np.longdouble)
    got = extended.decorrelated_extended(F, q)
    kappa = np.linalg.cond(F)
    err = float(np.abs(got - exact).max() / np.abs(exact).max())
    assert err <= 50 * EPS_LD * kappa, (err, kappa)
    # the float64 evaluation misses by far more: the pin is sharp
    _, dec64, _, _ = qml.normalisations(F, q)
    err64 = float(np.abs(dec64 - exact).max() / np.abs(exact).max())
    assert err64 > 10 * err


def test_matches_mpmath_reference():
    """A random SPD matrix with kappa ~ 1e8 against a 60-digit mpmath
    eigendecomposition (skipped where mpmath is not installed)."""
    mp = pytest.importorskip("mpmath")
    rng = np.random.default_rng(3)
    n = 10
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    F = (Q * np.logspace(0, 8, n)) @ Q.T
    F = 0.5 * (F + F.T)
    q = rng.normal(size=n)
    mp.mp.dps = 60
    E, V = mp.eigsy(mp.matrix(F.tolist()))
    Zm = V * mp.diag([1 / mp.sqrt(E[i]) for i in range(n)]) * V.T
    ref = np.array([float(x) for x in (Zm * mp.matrix(q.tolist()))], dtype=np.float64)
    got = extended.decorrelated_extended(F, q).astype(np.float64)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= 50 * EPS_LD * 1e8 + 1e-15, err


@pytest.mark.parametrize("cfg,scale", [(0, "full"), (1, "small")])
def test_workload_fisher(cfg, scale):
    """On the oracle's Fisher matrices: Z F Z = I to the long-double floor, and
    the float64 decorrelated estimate agrees within its own error eps kappa."""
    from oracle import harmonic
    wl = synth.workload(cfg, scale=scale)
    Y = harmonic.build_Y_for(wl)
    g = synth.rng(0, synth.P_MAPS)
    alm = synth.draw_alm(wl.cl_fid, wl.lmin, wl.lmax, wl.comps, 2, g)
    maps = qml.simulate(Y, alm, synth.noise_draws(wl.G, 2, g))
    ref = qml.qml_for(wl, Y, maps=maps)
    F, q = ref["F"], ref["q"]
    kappa = np.linalg.cond(F)
    Z, res = extended.inv_sqrt_extended(F)
    assert res <= 100 * EPS_LD * kappa, (res, kappa)
    ext = extended.decorrelated_extended(F, q).astype(np.float64)
    err64 = np.abs(ref["cl_decorr"] - ext).max() / max(np.abs(ext).max(), 1.0)
    assert err64 <= 20 * np.finfo(np.float64).eps * kappa, (err64, kappa)
