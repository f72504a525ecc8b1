"""Monte Carlo right-hand sides at the counts the benchmark times (100 maps
per step, 1000 maps per qml_estimate call) on the TQU Nside 16 workload
(n = 5952, k = 6900), float64 and split precision, against the oracle
element by element with the S20 metrics; and the decorrelated estimate
against an extended-precision evaluation of F^-1/2 q (Eq. decorrelated).

At 100 and 1000 maps the float64 product w = X^T (L^-1 D) takes other tiles
than at a few maps, and the split products slice 1 and 8 column tiles of
128; every column must still match the oracle."""
import numpy as np
import pytest

import parity as P
from oracle import extended, harmonic, qml
from paper_2605_21149_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
NMAPS = 1000


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_21149_gb300 import api as A
    from paper_2605_21149_gb300 import build
    build.build()
    return A


def td(x):
    return torch.as_tensor(np.asarray(x), device="cuda").t().contiguous().t()


@pytest.fixture(scope="module")
def tqu16():
    """Oracle reference for 1000 seeded maps of the TQU Nside 16 workload."""
    wl = synth.workload(1)
    g = synth.rng(1, synth.P_SIMS)
    alm = synth.draw_alm(wl.cl_fid, wl.lmin, wl.lmax, wl.comps, NMAPS, g)
    noise = synth.noise_draws(wl.G, NMAPS, g)
    Y = harmonic.build_Y_for(wl)
    maps = qml.simulate(Y, alm, noise)
    ref = qml.qml_for(wl, Y, maps=maps)
    del Y, alm, noise
    return wl, maps, ref


_PLANS = {}


def _plan(api, wl, precision):
    if precision not in _PLANS:
        _PLANS[precision] = api.fisher(api.Problem.from_workload(wl, precision=precision))
    return _PLANS[precision]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nsims", [100, NMAPS])
def test_estimate_bench_rhs_counts(api, tqu16, precision, nsims):
    wl, maps, ref = tqu16
    tol = P.TOL if precision == 0 else 1e-8
    F, plan = _plan(api, wl, precision)
    ge, ee = P.fisher_errors(F, ref["F"])
    assert ge <= tol and ee <= tol, (ge, ee)
    est = plan.estimate(td(maps[:, :nsims]))
    assert P.rel_max(est["y"], ref["y"][:, :nsims]) <= tol
    assert P.rel_max(est["q_conv"], ref["q"][:, :nsims]) <= tol
    assert P.rel_max(est["b"], ref["b"]) <= tol
    assert P.cl_deconv_error(est["cl_deconv"], ref["cl_deconv"][:, :nsims], ref["F"]) <= tol
    assert (P.cl_decorr_error(est["cl_decorr"], ref["cl_decorr"][:, :nsims])
            <= max(tol, P.decorr_tol(ref["F"])))
    # every column, not just the worst one: per-map relative error of y
    y, yr = P.to_np(est["y"]), ref["y"][:, :nsims]
    col = np.abs(y - yr).max(axis=0) / np.abs(yr).max(axis=0)
    assert col.max() <= tol, int(np.argmax(col))


def _decorr_errors(api, wl, maps, ref):
    """(GPU error, oracle float64 error, kappa) of the decorrelated estimate
    against F^-1/2 q in long double from the oracle's (F, q), in the units of
    the parity metric (|dC| / max(|C|, 1))."""
    F, plan = api.fisher(api.Problem.from_workload(wl))
    est = plan.estimate(td(maps))
    plan.free()
    ext = extended.decorrelated_extended(ref["F"], ref["q"]).astype(np.float64)
    scale = np.maximum(np.abs(ext), 1.0)
    e_gpu = float((np.abs(P.to_np(est["cl_decorr"]) - ext) / scale).max())
    e_ora = float((np.abs(ref["cl_decorr"] - ext) / scale).max())
    return e_gpu, e_ora, float(np.linalg.cond(ref["F"]))


@pytest.mark.parametrize("cfg,scale", [(0, "full"), (1, "small")])
def test_decorrelated_vs_extended_small(api, cfg, scale):
    """Where float64 allows it (20 eps kappa(F) below 1e-10) the GPU's
    decorrelated estimate is within 1e-10 of the extended-precision value."""
    wl = synth.workload(cfg, scale=scale)
    Y, alm, noise, maps = P.oracle_maps(wl, 3)
    ref = qml.qml_for(wl, Y, maps=maps)
    e_gpu, e_ora, kappa = _decorr_errors(api, wl, maps, ref)
    print(f"decorrelated vs long double: {wl.name}: kappa {kappa:.3g}, GPU {e_gpu:.3g}, "
          f"oracle float64 {e_ora:.3g}")
    assert e_gpu <= max(P.TOL, 20 * P.EPS * kappa), (e_gpu, kappa)


@pytest.mark.parametrize("mode", ["mixed16", "mixed8", "float64", "onesided"])
def test_decorrelated_vs_extended_tqu16(api, tqu16, mode):
    """TQU Nside 16 (kappa(F) ~ 7e8): the GPU's float64 F^-1/2 q against the
    extended-precision value; the measured error stays within the bound
    20 eps kappa(F) that the float64 parity tests use.  Every eigensolver
    form: the two-sided Jacobi on F after the float32 pre-rotation on a
    cluster of 16 or of 8 CTAs (default: eig_mixed = 1), the two-sided
    Jacobi alone (eig_mixed = 0), and the one-sided Jacobi on the Cholesky
    factor (eig_onesided = 1); with each, the deconvolved estimate stays
    within the parity tolerance too."""
    wl, maps, ref = tqu16
    sub = {"F": ref["F"], "q": ref["q"][:, :100], "cl_decorr": ref["cl_decorr"][:, :100]}
    keys = {"mixed16": {"eig_mixed": 1, "eig_cluster": 16},
            "mixed8": {"eig_mixed": 1, "eig_cluster": 8},
            "float64": {"eig_mixed": 0},
            "onesided": {"eig_onesided": 1}}[mode]
    for k, v in keys.items():
        api.tune_set(k, v)
    try:
        e_gpu, e_ora, kappa = _decorr_errors(api, wl, maps[:, :100], sub)
        F, plan = api.fisher(api.Problem.from_workload(wl))
        est = plan.estimate(td(maps[:, :100]))
        plan.free()
    finally:
        api.tune_set("eig_onesided", 0)
        api.tune_set("eig_mixed", 1)
        api.tune_set("eig_cluster", 16)
    print(f"decorrelated vs long double: {wl.name}: {mode}, kappa {kappa:.3g}, "
          f"GPU {e_gpu:.3g}, oracle float64 {e_ora:.3g}, bound {20 * P.EPS * kappa:.3g}")
    assert e_gpu <= 20 * P.EPS * kappa, (e_gpu, kappa)
    assert P.cl_deconv_error(est["cl_deconv"], ref["cl_deconv"][:, :100], ref["F"]) <= P.TOL


@pytest.mark.parametrize("mode", ["mixed16", "mixed8", "float64"])
def test_eigensolver_odd_order(api, mode):
    """QU Nside 8, l = 2..22: F of odd order 63, padded to 64 with a
    decoupled index, the smallest order the float32 pre-rotation takes (32
    pairs, two per CTA at 16 CTAs).  Deconvolved and decorrelated estimates
    against the oracle with every eigensolver form."""
    wl = synth.make_workload("QU nside8 lmax22", 8, 22, False, True, 20.0, ("EE", "BB", "EB"), 20, 15)
    Y, alm, noise, maps = P.oracle_maps(wl, 3)
    ref = qml.qml_for(wl, Y, maps=maps)
    assert ref["F"].shape[0] == 63
    keys = {"mixed16": {"eig_mixed": 1, "eig_cluster": 16},
            "mixed8": {"eig_mixed": 1, "eig_cluster": 8},
            "float64": {"eig_mixed": 0}}[mode]
    for k, v in keys.items():
        api.tune_set(k, v)
    try:
        F, plan = api.fisher(api.Problem.from_workload(wl))
        est = plan.estimate(td(maps))
        plan.free()
    finally:
        api.tune_set("eig_mixed", 1)
        api.tune_set("eig_cluster", 16)
    ge, ee = P.fisher_errors(F, ref["F"])
    assert ge <= P.TOL and ee <= P.TOL, (ge, ee)
    assert P.cl_deconv_error(est["cl_deconv"], ref["cl_deconv"], ref["F"]) <= P.TOL
    assert P.cl_decorr_error(est["cl_decorr"], ref["cl_decorr"]) <= P.decorr_tol(ref["F"])


def test_free_plans():
    for F, plan in _PLANS.values():
        plan.free()
    _PLANS.clear()
