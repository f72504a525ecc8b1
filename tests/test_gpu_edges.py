"""Edge cases of the GPU path: sizes across the 512-wide split panels, empty
inputs (no maps, no scan items, empty products), the emulator without a
held-out set, and arguments the host rejects."""
import numpy as np
import pytest
import scipy.linalg as sla

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


def colmajor(x):
    return torch.as_tensor(np.asarray(x), device="cuda").t().contiguous().t()


def spd(n, seed):
    g = np.random.default_rng(seed)
    B = g.normal(size=(n, n))
    return B @ B.T / n + np.eye(n)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n", [1, 100, 511, 512, 513, 1100, 1537])
def test_potrf_trsm_across_panels(api, precision, n):
    """Split Cholesky panels are 512 wide, float64 blocks 64: sizes just
    below, at and above the panel edge, and several panels with a ragged one.
    Reference: LAPACK Cholesky and triangular solve (scipy), float64."""
    _potrf_trsm_check(api, precision, n)


@pytest.mark.parametrize("n", [1, 100, 513, 1537])
def test_potrf_float_float_diagonal(api, n):
    """The opt-in float-float 64-blocks of the split Cholesky (tuning key
    split_diag_df) against the same LAPACK reference and tolerances."""
    api.tune_set("split_diag_df", 1)
    try:
        _potrf_trsm_check(api, 1, n)
    finally:
        api.tune_set("split_diag_df", 0)


def _potrf_trsm_check(api, precision, n):
    A = spd(n, n)
    Lref = np.linalg.cholesky(A)
    At = colmajor(A)
    ld = api.potrf(At, precision=precision)
    ld = float(ld.item() if hasattr(ld, "item") else ld)
    L = np.tril(At.cpu().numpy())
    tol = 1e-12 if precision == 0 else 1e-10
    assert np.abs(L - Lref).max() <= tol * np.abs(Lref).max()
    assert abs(ld - 2 * np.log(np.diag(Lref)).sum()) <= 1e-12 * max(1.0, abs(ld))
    # the strict upper triangle is left untouched
    assert np.array_equal(np.triu(At.cpu().numpy(), 1), np.triu(A, 1))
    g = np.random.default_rng(n + 1)
    B = g.normal(size=(n, 37))
    X = api.trsm(colmajor(Lref), colmajor(B), precision=precision).cpu().numpy()
    Xref = sla.solve_triangular(Lref, B, lower=True)
    assert np.abs(X - Xref).max() <= tol * 10 * np.abs(Xref).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_gemm_empty_and_k0(api, precision):
    g = np.random.default_rng(3)
    A = colmajor(np.zeros((0, 5)))
    B = colmajor(g.normal(size=(5, 4)))
    C = api.gemm(A, B, precision=precision)  # m = 0: nothing to do
    assert tuple(C.shape) == (0, 4)
    # K = 0: C <- beta C
    C0 = g.normal(size=(6, 4))
    Ct = colmajor(C0)
    api.gemm(colmajor(np.zeros((6, 0))), colmajor(np.zeros((0, 4))), Ct, beta=0.5, precision=precision)
    assert np.allclose(Ct.cpu().numpy(), 0.5 * C0, rtol=0, atol=0)


def test_estimate_without_maps_gives_bias(api):
    wl = synth.workload(0)
    prob = api.Problem.from_workload(wl)
    F, plan = api.fisher(prob)
    n = wl.n
    g = np.random.default_rng(4)
    one = plan.estimate(colmajor(g.normal(size=(n, 1))))
    none = plan.estimate(torch.zeros((0, n), dtype=torch.float64, device="cuda").t())
    assert tuple(none["y"].shape) == (plan.prob.na, 0)
    assert np.array_equal(none["b"].cpu().numpy(), one["b"].cpu().numpy())
    plan.free()


def test_batch_without_items(api):
    masks, taus, rs = synth.batch_workload(nside=8, lmax=15, rank=10, ngrid=2)
    prob = api.Problem.from_workload(masks[0])
    maps = colmajor(np.random.default_rng(5).normal(size=(masks[0].n, 1)))
    lnl, chi2, ld = api.loglike_batch([(prob, maps)], np.zeros(0, dtype=np.int32),
                                      torch.zeros((0, 6, 16), dtype=torch.float64, device="cuda"))
    assert lnl.shape[0] == 0 and chi2.shape[0] == 0 and ld.shape[0] == 0


def test_batch_rejects_mask_index(api):
    masks, taus, rs = synth.batch_workload(nside=8, lmax=15, rank=10, ngrid=2)
    prob = api.Problem.from_workload(masks[0])
    maps = colmajor(np.random.default_rng(6).normal(size=(masks[0].n, 1)))
    cl = torch.as_tensor(synth.batch_item_spectra(15, taus[:2], rs[:2]), device="cuda")
    with pytest.raises(RuntimeError):
        api.loglike_batch([(prob, maps)], np.array([0, 1], dtype=np.int32), cl)


def test_emulator_small_training_set(api):
    """Below 512 labels nothing is held out: the threshold is tol / 2."""
    g = np.random.default_rng(8)
    th = g.uniform(-1, 1, size=(256, 3))
    y = (th ** 2).sum(axis=1)
    emu = api.Emulator(-np.ones(3), np.ones(3), width=64, depth=2, seed=2)
    emu.train(th, y, epochs=5, batch=64)
    thr, nheld = emu.threshold(0.05)
    assert nheld == 0 and thr == pytest.approx(0.025)
    pred, flags = emu.predict(th[:1])
    assert pred.shape[0] == 1 and flags.shape[0] == 1
    emu.free()
