"""Cross-QML (qml_cross, Sect. 2.2 Eq. q_cross) against the oracle's
cross_qml: two data sets with the same signal and independent noise on the
same pixels, each filtered by its own C_i = S + N_i.  The mode-mixing matrix
Wx = 1/2 tr[C1^-1 P_a C2^-1 P_b], the cross estimates q = 1/2 d1^T C1^-1 P_a
C2^-1 d2 and Wx^-1 q, element by element (float64 1e-10, split 1e-8), with
plans in either basis; equal inputs reduce to the auto estimator's F and y."""
import numpy as np
import pytest

import parity as P
from oracle import harmonic, qml
from paper_2605_21149_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def _pair(nside, lmax, has_T, has_P, cut, spec, rank, config, nsims=3):
    """Two workloads on the same pixels (same cut) whose noise differs, one
    signal draw seen through both noises; the oracle's cross estimator."""
    wl1 = synth.make_workload("cross 1", nside, lmax, has_T, has_P, cut, spec, rank, config)
    wl2 = synth.make_workload("cross 2", nside, lmax, has_T, has_P, cut, spec, rank, config + 50)
    g = synth.rng(config, synth.P_MAPS)
    alm = synth.draw_alm(wl1.cl_fid, wl1.lmin, wl1.lmax, wl1.comps, nsims, g)
    Y = harmonic.build_Y_for(wl1)
    d1 = qml.simulate(Y, alm, synth.noise_draws(wl1.G, nsims, g))
    d2 = qml.simulate(Y, alm, synth.noise_draws(wl2.G, nsims, g))
    ref = qml.cross_qml(Y, wl1.cl_fid, wl1.comps, wl1.lmin, wl1.lmax, wl1.N(), wl2.N(), wl1.spec,
                        d1=d1, d2=d2)
    return wl1, wl2, d1, d2, ref


def _check(api, wl1, wl2, d1, d2, ref, bases=(0, 0), precision=0):
    tol = P.TOL if precision == 0 else 1e-8
    plans = []
    for wl, basis in zip((wl1, wl2), bases):
        _, plan = api.fisher(api.Problem.from_workload(wl, precision=precision, basis=basis))
        plans.append(plan)
    out = api.cross(plans[0], plans[1], td(d1), td(d2))
    for p in plans:
        p.free()
    Wx = P.to_np(out["Wx"])
    assert P.rel_max(Wx, ref["Wx"]) <= tol
    assert P.rel_max(out["q"], ref["q"]) <= tol
    sig = np.sqrt(np.abs(np.diag(np.linalg.inv(ref["Wx"]))))[:, None]
    cl, clr = P.to_np(out["cl"]), ref["cl_deconv"]
    assert (np.abs(cl - clr) / np.maximum(np.abs(clr), sig)).max() <= tol
    return Wx


@pytest.mark.parametrize("bases", [(0, 0), (1, 1), (0, 1)])
def test_cross_tqu_matches_oracle(api, bases):
    """TQU Nside 8 up to l = 13, six spectra; pixel, harmonic and mixed plans."""
    args = _pair(8, 13, True, True, 20.0, synth.SPEC_NAMES, 15, 61)
    _check(api, *args, bases=bases)


def test_cross_qu_and_t(api):
    _check(api, *_pair(8, 12, False, True, 30.0, ("EE", "BB", "EB"), 10, 62))
    _check(api, *_pair(8, 16, True, False, 20.0, ("TT",), 10, 63))


def test_cross_split_precision(api):
    _check(api, *_pair(8, 13, True, True, 20.0, synth.SPEC_NAMES, 15, 64), precision=1)


def test_cross_tqu_nside16_full(api):
    """TQU Nside 16, l = 2..47 (n = 5952, k = 6900): Wx is 276 x 276."""
    _check(api, *_pair(16, 47, True, True, 20.0, synth.SPEC_NAMES, 200, 65, nsims=2))


def test_cross_with_itself_is_auto(api):
    """The same plan twice: Wx is the Fisher matrix and q the auto y."""
    wl = synth.workload(0)
    Y, alm, noise, maps = P.oracle_maps(wl, 2)
    F, plan = api.fisher(api.Problem.from_workload(wl))
    est = plan.estimate(td(maps))
    out = api.cross(plan, plan, td(maps), td(maps))
    plan.free()
    assert P.rel_max(out["Wx"], F) <= 1e-12
    assert P.rel_max(out["q"], est["y"]) <= 1e-12


def test_cross_rejects_mismatched_plans(api):
    _, p1 = api.fisher(api.Problem.from_workload(synth.workload(0)))
    wl = synth.make_workload("other", 8, 12, True, False, 20.0, ("TT",), 10, 66)
    _, p2 = api.fisher(api.Problem.from_workload(wl))
    with pytest.raises(api.QMLError) as ei:
        api.cross(p1, p2)
    assert ei.value.status == 1
    p1.free()
    p2.free()
