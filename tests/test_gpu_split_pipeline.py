"""Split-precision form of the whole path (precision = QML_SPLIT_BF16) against
the float64 oracle: F, b, y, Cl and lnL within 1e-8 (the split-form tolerance;
same metrics as the float64 parity tests, decorrelated Cl bounded by
max(1e-8, 20 eps kappa(F)))."""
import numpy as np
import pytest

import parity as P
from oracle import harmonic, qml
from paper_2605_21149_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-8
SPLIT = 1


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


def _check(api, wl, nsims=3, bias=True):
    Y, alm, noise, maps = P.oracle_maps(wl, nsims)
    ref = qml.qml_for(wl, Y, maps=maps, want_bias=bias)
    prob = api.Problem.from_workload(wl, precision=SPLIT)
    F, plan = api.fisher(prob)
    ge, ee = P.fisher_errors(F, ref["F"])
    assert ge <= TOL and ee <= TOL, (ge, ee)
    est = plan.estimate(td(maps))
    assert P.rel_max(est["y"], ref["y"]) <= TOL
    if bias:
        assert P.rel_max(est["b"], ref["b"]) <= TOL
        assert P.cl_deconv_error(est["cl_deconv"], ref["cl_deconv"], ref["F"]) <= TOL
        assert P.cl_decorr_error(est["cl_decorr"], ref["cl_decorr"]) <= max(TOL, P.decorr_tol(ref["F"]))
    plan.free()
    lnl, chi2, ld = qml.loglike(ref["C"], maps)
    g_lnl, g_chi2, g_ld = api.loglike(prob, torch.as_tensor(wl.cl_fid.reshape(-1), device="cuda"),
                                      td(maps))
    assert P.rel_max(g_lnl, lnl) <= TOL
    assert abs(float(P.to_np(g_ld)) - ld) <= TOL * abs(ld)
    return ge, ee


@pytest.mark.parametrize("cfg,scale", [(0, "full"), (1, "small"), (2, "small")])
def test_split_small(api, cfg, scale):
    _check(api, synth.workload(cfg, scale=scale))


def test_split_tqu_nside16_full(api):
    """n = 5952 > 512: panels, split panel solves and trailing updates."""
    _check(api, synth.workload(1), nsims=4)


def test_split_qu_nside32_full(api):
    """The split-precision workload: QU, Nside 32, f_sky 0.7, l = 2..95
    (n = 17152, k = 18424), against the full float64 oracle."""
    _check(api, synth.workload(2), nsims=2)


def test_split_tqu_nside16_float_float_diagonal(api):
    """The opt-in float-float 64-blocks of the split Cholesky (tuning key
    split_diag_df) keep the whole path within the split tolerance."""
    api.tune_set("split_diag_df", 1)
    try:
        _check(api, synth.workload(1), nsims=4)
    finally:
        api.tune_set("split_diag_df", 0)


@pytest.mark.parametrize("basis", [0, 1])
def test_split_lookahead_bit_identical(api, basis):
    """Lookahead in the split Cholesky (the next panel's float64 chain on a
    second stream beside the trailing update and the forward substitution,
    tuning key split_lookahead = 1, the default) changes when kernels run, not
    what they compute: F, b, y, every normalisation and lnL equal the
    single-stream order bit for bit (TQU Nside 16, twelve 512 panels; the
    harmonic basis factors N the same way)."""
    wl = synth.workload(1)
    Y, alm, noise, maps = P.oracle_maps(wl, 3)
    prob = api.Problem.from_workload(wl, precision=SPLIT, basis=basis)
    cl = torch.as_tensor(wl.cl_fid.reshape(-1), device="cuda")
    outs = []
    try:
        for look in (1, 0):
            api.tune_set("split_lookahead", look)
            F, plan = api.fisher(prob)
            est = plan.estimate(td(maps))
            plan.free()
            lnl, chi2, ld = api.loglike(prob, cl, td(maps))
            outs.append([P.to_np(F)] + [P.to_np(est[k]) for k in sorted(est)] +
                        [P.to_np(lnl), P.to_np(chi2), np.atleast_1d(P.to_np(ld))])
    finally:
        api.tune_set("split_lookahead", 1)
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_split_potrf_lookahead_bit_identical(api):
    """qml_potrf in split precision (n = 1700: four panels, the last one
    ragged) with and without lookahead: the same factor and log det."""
    rng = np.random.default_rng(5)
    n = 1700
    G = rng.normal(size=(n, n + 50))
    A = G @ G.T / n + np.eye(n)
    outs = []
    try:
        for look in (1, 0):
            api.tune_set("split_lookahead", look)
            Ad = td(A)
            ld = api.potrf(Ad, precision=SPLIT)
            outs.append((np.tril(P.to_np(Ad)), float(P.to_np(ld))))
    finally:
        api.tune_set("split_lookahead", 1)
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]
