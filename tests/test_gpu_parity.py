"""GPU parity: every entry point of the C ABI against the CPU oracle,
element by element, on seeded inputs shaped like the paper's workloads.
All calls go through the C ABI (ctypes binding)."""
import math

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


def _small_workloads():
    """Small TQU / QU / T problems: several 64-wide tiles and a ragged tail."""
    out = []
    th, ph, z = synth.healpix_ring_centres(4)
    keep = synth.galactic_cut(z, 20.0)
    out.append(synth.make_workload("TQU nside4 lmax9", 4, 9, True, True, 20.0,
                                   synth.SPEC_NAMES, 12, 11))
    out.append(synth.make_workload("QU nside8 lmax13", 8, 13, False, True, 30.0,
                                   ("EE", "BB", "EB"), 20, 12))
    out.append(synth.workload(0))
    out.append(synth.workload(1, scale="small"))
    return out


def _gl_workload(lmax=10):
    th, ph, w = synth.gauss_legendre_grid(lmax)
    return synth.make_workload("GL TQU", 0, lmax, True, True, 0.0, synth.SPEC_NAMES, 8, 13,
                               geometry=(th, ph))


# ----------------------------------------------------------------- Y ------
@pytest.mark.parametrize("idx", [0, 1, 2, 3])
def test_ybuild_matches_oracle(api, idx):
    wl = _small_workloads()[idx]
    prob = api.Problem.from_workload(wl)
    Y = P.to_np(api.ybuild(prob))
    Yref = harmonic.build_Y_for(wl)
    assert Y.shape == Yref.shape
    assert np.abs(Y - Yref).max() <= 1e-12 * np.abs(Yref).max()


def test_ybuild_arbitrary_geometry(api):
    wl = _gl_workload(12)
    prob = api.Problem.from_workload(wl)
    Y = P.to_np(api.ybuild(prob))
    assert np.abs(Y - harmonic.build_Y_for(wl)).max() <= 1e-12


def test_ybuild_full_sizes_sampled(api):
    """TQU Nside 16 l<=47 in full, QU Nside 32 l<=95 on sampled columns."""
    wl = synth.workload(1)
    Y = P.to_np(api.ybuild(api.Problem.from_workload(wl)))
    Yref = harmonic.build_Y_for(wl)
    assert np.abs(Y - Yref).max() <= 1e-12 * np.abs(Yref).max()
    wl = synth.workload(2)
    Yd = api.ybuild(api.Problem.from_workload(wl))
    rng = np.random.default_rng(5)
    cols = np.sort(rng.choice(wl.k, 400, replace=False))
    Ysub = Yd[:, torch.as_tensor(cols, device="cuda")].cpu().numpy()
    # the oracle evaluates the sampled columns' multipoles only
    from oracle.harmonic import build_Y
    Yref = build_Y(wl.lmin, wl.lmax, wl.theta_T, wl.phi_T, wl.theta_P, wl.phi_P,
                   wl.transfer_T, wl.transfer_P, wl.has_T, wl.has_P)[:, cols]
    assert np.abs(Ysub - Yref).max() <= 1e-12 * np.abs(Yref).max()


# ----------------------------------------------------- dense kernels ------
@pytest.mark.parametrize("n", [1, 7, 33, 64, 65, 130, 257])
def test_potrf_trsm_ragged(api, n):
    rng = np.random.default_rng(n)
    G = rng.normal(size=(n, n))
    A = G @ G.T + n * np.eye(n)
    Ad = torch.as_tensor(np.asfortranarray(A), device="cuda").t().contiguous().t()
    ld = api.potrf(Ad)
    L = np.tril(P.to_np(Ad))
    Lref = np.linalg.cholesky(A)
    assert np.abs(L - Lref).max() <= 1e-12 * np.abs(Lref).max()
    assert abs(float(P.to_np(ld)) - 2 * np.log(np.diag(Lref)).sum()) <= 1e-12 * n
    B = rng.normal(size=(n, 5))
    Bd = torch.as_tensor(B, device="cuda").t().contiguous().t()
    api.trsm(Ad, Bd)
    import scipy.linalg as sla
    Xref = sla.solve_triangular(Lref, B, lower=True)
    assert np.abs(P.to_np(Bd) - Xref).max() <= 1e-11 * max(1.0, np.abs(Xref).max())


@pytest.mark.parametrize("ta,tb,m,nn,kk", [(0, 0, 1, 1, 1), (0, 1, 65, 33, 7), (1, 0, 130, 64, 257),
                                           (1, 1, 17, 200, 65), (0, 0, 300, 129, 100)])
def test_gemm_ragged(api, ta, tb, m, nn, kk):
    rng = np.random.default_rng(m + nn + kk)
    A = rng.normal(size=(kk, m) if ta else (m, kk))
    B = rng.normal(size=(nn, kk) if tb else (kk, nn))
    C0 = rng.normal(size=(m, nn))
    td = lambda x: torch.as_tensor(x, device="cuda").t().contiguous().t()
    Cd = td(C0)
    api.gemm(td(A), td(B), Cd, transA=bool(ta), transB=bool(tb), alpha=0.7, beta=-1.3)
    ref = 0.7 * ((A.T if ta else A) @ (B.T if tb else B)) - 1.3 * C0
    assert np.abs(P.to_np(Cd) - ref).max() <= 1e-13 * kk * np.abs(ref).max()


def test_gemm_lower_only_leaves_upper(api):
    rng = np.random.default_rng(3)
    n, kk = 150, 70
    A = rng.normal(size=(n, kk))
    C0 = rng.normal(size=(n, n))
    td = lambda x: torch.as_tensor(x, device="cuda").t().contiguous().t()
    Cd = td(C0)
    api.gemm(td(A), td(A), Cd, transB=True, beta=1.0, lower=True)
    out = P.to_np(Cd)
    ref = A @ A.T + C0
    il = np.tril_indices(n)
    iu = np.triu_indices(n, 1)
    assert np.abs(out[il] - ref[il]).max() <= 1e-12 * np.abs(ref).max()
    assert np.array_equal(out[iu], C0[iu])


def test_not_positive_definite_is_reported(api):
    """A host-made indefinite matrix: the pivot check returns QML_ENOTSPD with
    the failing column; no fault, the context stays usable."""
    n = 100
    A = np.eye(n)
    A[70, 70] = -1.0
    Ad = torch.as_tensor(A, device="cuda").t().contiguous().t()
    with pytest.raises(api.QMLError) as ei:
        api.potrf(Ad)
    assert ei.value.status == 2 and "column 70" in str(ei.value)
    # context still usable
    B = torch.eye(4, dtype=torch.float64, device="cuda")
    api.potrf(B)


# ------------------------------------------------------- QML pipeline ------
def _qml_check(api, wl, nsims=3):
    Y, alm, noise, maps = P.oracle_maps(wl, nsims)
    ref = qml.qml_for(wl, Y, maps=maps)
    prob = api.Problem.from_workload(wl)
    F, plan = api.fisher(prob)
    ge, ee = P.fisher_errors(F, ref["F"])
    assert ge <= P.TOL and ee <= P.TOL, (ge, ee)
    md = torch.as_tensor(maps, device="cuda").t().contiguous().t()
    est = plan.estimate(md)
    assert P.rel_max(est["b"], ref["b"]) <= P.TOL
    assert P.rel_max(est["y"], ref["y"]) <= P.TOL
    assert P.rel_max(est["q_conv"], ref["q"]) <= P.TOL
    assert P.cl_deconv_error(est["cl_deconv"], ref["cl_deconv"], ref["F"]) <= P.TOL
    assert P.cl_decorr_error(est["cl_decorr"], ref["cl_decorr"]) <= P.decorr_tol(ref["F"])
    plan.free()
    return F, est, ref


@pytest.mark.parametrize("idx", [0, 1, 2, 3])
def test_qml_small_matches_oracle(api, idx):
    _qml_check(api, _small_workloads()[idx])


def test_qml_gauss_legendre_closed_form(api):
    """GPU F on the exact quadrature grid also equals the per-l closed form."""
    lmin, lmax = 2, 7
    th, ph, w = synth.gauss_legendre_grid(lmax)
    wl = synth.make_workload("GL", 0, lmax, True, True, 0.0, synth.SPEC_NAMES, 1, 14,
                             geometry=(th, ph))
    wl.transfer_T = wl.transfer_P = synth.gaussian_beam(lmax, 0.25)
    sigma2 = 0.7
    wt = np.concatenate([w, w, w])
    # N = diag(sigma^2 / w_p): G G^T + sigma2 I replaced by an explicit diagonal
    wl.G = np.zeros((len(wt), 1))
    prob = api.Problem(lmin, lmax, theta_T=torch.as_tensor(th, device="cuda"),
                       phi_T=torch.as_tensor(ph, device="cuda"),
                       theta_P=torch.as_tensor(th, device="cuda"),
                       phi_P=torch.as_tensor(ph, device="cuda"),
                       transfer_T=torch.as_tensor(wl.transfer_T, device="cuda"),
                       transfer_P=torch.as_tensor(wl.transfer_P, device="cuda"),
                       spec=synth.SPEC_NAMES,
                       cl_fid=torch.as_tensor(wl.cl_fid.reshape(-1), device="cuda"),
                       N=torch.as_tensor(np.diag(sigma2 / wt), device="cuda"))
    F, _ = api.fisher(prob, keep_plan=False)
    import test_oracle_qml as T
    Fc, bc, _ = T._closed_form(wl.cl_fid, wl.transfer_T, sigma2, tuple(range(6)), (0, 1, 2),
                               lmin, lmax)
    assert np.abs(P.to_np(F) - Fc).max() <= 1e-11 * np.abs(Fc).max()


def test_qml_tqu_nside16_full(api):
    """The TQU Nside 16, l = 2..47 workload (n = 5952, k = 6900) in full."""
    _qml_check(api, synth.workload(1), nsims=4)


def test_estimate_host_buffers_match_device(api):
    """The same entry points with host (numpy) buffers give identical results."""
    wl = synth.workload(0)
    Y, alm, noise, maps = P.oracle_maps(wl, 2)
    pd = api.Problem.from_workload(wl, device=True)
    ph = api.Problem.from_workload(wl, device=False)
    Fd, pld = api.fisher(pd)
    Fh, plh = api.fisher(ph)
    assert np.array_equal(P.to_np(Fd), Fh)
    ed = pld.estimate(torch.as_tensor(maps, device="cuda").t().contiguous().t())
    eh = plh.estimate(maps)
    for k in ("y", "b", "cl_deconv", "cl_decorr", "q_conv"):
        assert np.array_equal(P.to_np(ed[k]), eh[k]), k


def test_deterministic_bitwise(api):
    wl = _small_workloads()[0]
    prob = api.Problem.from_workload(wl)
    F1, _ = api.fisher(prob, keep_plan=False)
    F2, _ = api.fisher(prob, keep_plan=False)
    assert torch.equal(F1, F2)


# ---------------------------------------------------------- likelihood ------
@pytest.mark.parametrize("idx", [0, 1, 2, 3])
def test_loglike_matches_oracle(api, idx):
    wl = _small_workloads()[idx]
    Y, alm, noise, maps = P.oracle_maps(wl, 3)
    cl = synth.spectra(wl.lmax, tau=0.07, r=0.05)
    C = qml.total_cov(Y, cl, wl.comps, wl.lmin, wl.lmax, wl.N())
    lnl, chi2, ld = qml.loglike(C, maps)
    prob = api.Problem.from_workload(wl)
    g_lnl, g_chi2, g_ld = api.loglike(prob, torch.as_tensor(cl.reshape(-1), device="cuda"),
                                      torch.as_tensor(maps, device="cuda").t().contiguous().t())
    assert P.rel_max(g_lnl, lnl) <= P.TOL
    assert P.rel_max(g_chi2, chi2) <= P.TOL
    assert abs(float(P.to_np(g_ld)) - ld) <= P.TOL * abs(ld)


def test_synthesize_matches_oracle(api):
    wl = _small_workloads()[0]
    Y, alm, noise, maps = P.oracle_maps(wl, 4)
    prob = api.Problem.from_workload(wl)
    td = lambda x: torch.as_tensor(x, device="cuda").t().contiguous().t()
    out = api.synthesize(prob, td(alm), td(noise))
    assert np.abs(P.to_np(out) - maps).max() <= 1e-12 * np.abs(maps).max()


# --------------------------------------------------- native binning -------
BINNED_CASES = [
    (0, "full", [2, 5, 8, 11, 14, 17], 0),            # T, l 2..16, Delta l = 3
    (0, "full", [2, 7, 12, 17], 0),                    # Delta l = 5
    (1, "small", list(range(2, 17, 2)), 0),            # TQU, l 2..15, Delta l = 2
    (1, "small", [2, 3, 7, 16], 0),                    # ragged bins
    (1, "small", list(range(2, 17, 2)), 1),            # split precision
]


@pytest.mark.parametrize("cfg,scale,edges,precision", BINNED_CASES)
def test_qml_binned_matches_oracle(api, cfg, scale, edges, precision):
    """Sect. 2.4: with bin edges, F, the noise bias, y and the three
    normalisations are the binned ones (the oracle forms them from the bin
    selectors E_b = sum_{l in b} E_l); tolerance 1e-10, split 1e-8."""
    wl = synth.workload(cfg, scale=scale)
    tol = P.TOL if precision == 0 else 1e-8
    Y, alm, noise, maps = P.oracle_maps(wl, 3)
    ref = qml.qml_for(wl, Y, maps=maps, edges=np.asarray(edges))
    prob = api.Problem.from_workload(wl, precision=precision, bin_edges=edges)
    F, plan = api.fisher(prob)
    nab = len(wl.spec) * (len(edges) - 1)
    assert tuple(F.shape) == (nab, nab)
    ge, ee = P.fisher_errors(F, ref["F"])
    assert ge <= tol and ee <= tol, (ge, ee)
    md = torch.as_tensor(maps, device="cuda").t().contiguous().t()
    est = plan.estimate(md)
    assert P.rel_max(est["b"], ref["b"]) <= tol
    assert P.rel_max(est["y"], ref["y"]) <= tol
    assert P.rel_max(est["q_conv"], ref["q"]) <= tol
    assert P.cl_deconv_error(est["cl_deconv"], ref["cl_deconv"], ref["F"]) <= tol
    assert P.cl_decorr_error(est["cl_decorr"], ref["cl_decorr"]) <= max(tol, P.decorr_tol(ref["F"]))
    plan.free()


def test_qml_unit_bins_equal_per_l(api):
    """One multipole per bin is the per-l estimator (the single code path of
    Sect. 2.4): identical outputs."""
    wl = synth.workload(0)
    Y, alm, noise, maps = P.oracle_maps(wl, 2)
    md = torch.as_tensor(maps, device="cuda").t().contiguous().t()
    out = []
    for edges in (None, list(range(wl.lmin, wl.lmax + 2))):
        F, plan = api.fisher(api.Problem.from_workload(wl, bin_edges=edges))
        est = plan.estimate(md)
        out.append((P.to_np(F), {k: P.to_np(v) for k, v in est.items()}))
        plan.free()
    assert np.array_equal(out[0][0], out[1][0])
    for k in out[0][1]:
        assert np.array_equal(out[0][1][k], out[1][1][k]), k
