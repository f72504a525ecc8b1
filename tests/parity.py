"""Shared helpers of the GPU parity tests: oracle runs and the tolerance
metrics (float64 path: 1e-10, measured with the metrics below).

F      max |dF| / max |F|, and elementwise relative error on the entries with
       |F_ab| >= 1e-6 max |F|.
b, y   max |d| / max |ref| per quantity.
Cl     deconvolved: |dC_a| / max(|C_a|, sqrt((F^-1)_aa)) (error-bar scale);
       decorrelated: |dC_a| / max(|C_a|, 1) (unit covariance), bounded by
       max(1e-10, 20 eps kappa(F)) because F -> F^-1/2 has relative condition
       number kappa(F)/2 (two float64 evaluations of the oracle itself differ
       by ~eps kappa(F)).
lnL    |d lnL| / |lnL|, same for chi2 and ln|C|.
"""
import numpy as np

from oracle import harmonic, qml

EPS = np.finfo(np.float64).eps
TOL = 1e-10


def to_np(x):
    if hasattr(x, "detach"):
        return x.detach().cpu().numpy()
    return np.asarray(x)


def rel_max(a, ref):
    a, ref = to_np(a), to_np(ref)
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-300))


def fisher_errors(F, Fref):
    F, Fref = to_np(F), to_np(Fref)
    mx = np.abs(Fref).max()
    glob = np.abs(F - Fref).max() / mx
    sig = np.abs(Fref) >= 1e-6 * mx
    elem = (np.abs(F - Fref)[sig] / np.abs(Fref)[sig]).max()
    return float(glob), float(elem)


def cl_deconv_error(C, Cref, Fref):
    C, Cref = to_np(C), to_np(Cref)
    sig = np.sqrt(np.diag(np.linalg.inv(to_np(Fref))))[:, None]
    return float((np.abs(C - Cref) / np.maximum(np.abs(Cref), sig)).max())


def decorr_tol(Fref):
    return max(TOL, 20 * EPS * np.linalg.cond(to_np(Fref)))


def cl_decorr_error(C, Cref):
    C, Cref = to_np(C), to_np(Cref)
    return float((np.abs(C - Cref) / np.maximum(np.abs(Cref), 1.0)).max())


def oracle_maps(wl, nsims, seed_purpose=2):
    """Seeded maps d = Y a + n built by the oracle (also returns alm, noise)."""
    from paper_2605_21149_gb300 import synth
    g = synth.rng(0, seed_purpose)
    alm = synth.draw_alm(wl.cl_fid, wl.lmin, wl.lmax, wl.comps, nsims, g)
    noise = synth.noise_draws(wl.G, nsims, g)
    Y = harmonic.build_Y_for(wl)
    return Y, alm, noise, qml.simulate(Y, alm, noise)
