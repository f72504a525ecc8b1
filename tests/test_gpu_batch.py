"""Batched likelihood scan (pix_loglike_batch, harmonic SMW form) against
the oracle's pixel-definition lnL, item by item, mixed masks."""
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


_ORACLE = {}


def _oracle(nside, lmax, items, nmaps, ngrid):
    key = (nside, lmax, items, nmaps, ngrid)
    if key not in _ORACLE:
        masks, taus, rs = synth.batch_workload(nside=nside, lmax=lmax, rank=30, ngrid=ngrid)
        sel = np.linspace(0, len(taus) - 1, items).astype(int)
        item_mask = sel % len(masks)
        item_cl = synth.batch_item_spectra(lmax, taus[sel], rs[sel])
        ys, mapss = [], []
        for j, wl in enumerate(masks):
            Y, alm, noise, maps = P.oracle_maps(wl, nmaps, seed_purpose=20 + j)
            ys.append(Y)
            mapss.append(maps)
        refs = []
        for i in range(items):
            m = item_mask[i]
            C = qml.total_cov(ys[m], item_cl[i], masks[m].comps, masks[m].lmin, masks[m].lmax,
                              masks[m].N())
            refs.append(qml.loglike(C, mapss[m]))
        _ORACLE[key] = (masks, item_mask, item_cl, mapss, refs)
    return _ORACLE[key]


def _run(api, nside, lmax, items, precision, tol, nmaps=2, ngrid=8):
    masks, item_mask, item_cl, mapss, refs = _oracle(nside, lmax, items, nmaps, ngrid)
    probs = [(api.Problem.from_workload(wl, precision=precision), td(mp)) for wl, mp in zip(masks, mapss)]
    lnl, chi2, ld = api.loglike_batch(probs, item_mask, torch.as_tensor(item_cl, device="cuda"))
    lnl, chi2, ld = P.to_np(lnl), P.to_np(chi2), P.to_np(ld)
    for i in range(items):
        rl, rc, rd = refs[i]
        assert np.abs(lnl[i, :nmaps] - rl).max() <= tol * np.abs(rl).max(), i
        assert np.abs(chi2[i, :nmaps] - rc).max() <= tol * np.abs(rc).max(), i
        assert abs(ld[i] - rd) <= tol * abs(rd), i


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-8)])
def test_batch_small(api, precision, tol):
    _run(api, 8, 15, 9, precision, tol)


def _with_split_kt(api, fn):
    api.tune_set("batch_split_kt", 1)
    try:
        fn()
    finally:
        api.tune_set("batch_split_kt", 0)


def test_batch_split_kt_64_items_nside8(api):
    """The opt-in split-precision inner factor (batch_split_kt = 1: Kt's
    trailing updates and panel products as split products, k = 756 > 512 so
    two panels) on 64 items over the three masks, against the oracle's pixel
    lnL at the split tolerance."""
    _with_split_kt(api, lambda: _run(api, 8, 15, 64, 1, 1e-8))


def test_batch_split_kt_grid_corners_nside16(api):
    """Split Kt at TQU Nside 16 (k = 6900) on the f_sky 0.5 mask, 64 items of
    the 64 x 64 (tau, r) grid including its four corners (tau = 0.03, 0.09 and
    r = 0, 0.1), every item against the oracle's pixel lnL within 1e-8."""
    masks, taus, rs = synth.batch_workload(nside=16, lmax=47, rank=30, ngrid=64)
    wl = masks[0]
    corners = [0, 63, 64 * 63, 64 * 64 - 1]
    rest = np.linspace(1, 64 * 64 - 2, 60).astype(int)
    sel = np.array(corners + list(rest))
    item_cl = synth.batch_item_spectra(47, taus[sel], rs[sel])
    Y, alm, noise, maps = P.oracle_maps(wl, 1, seed_purpose=20)
    refs = [qml.loglike(qml.total_cov(Y, item_cl[i], wl.comps, wl.lmin, wl.lmax, wl.N()), maps)
            for i in range(len(sel))]
    del Y

    def run():
        prob = api.Problem.from_workload(wl, precision=1)
        lnl, chi2, ld = api.loglike_batch([(prob, td(maps))], np.zeros(len(sel), dtype=np.int32),
                                          torch.as_tensor(item_cl, device="cuda"))
        lnl, chi2, ld = P.to_np(lnl), P.to_np(chi2), P.to_np(ld)
        for i, (rl, rc, rd) in enumerate(refs):
            assert abs(lnl[i, 0] - rl[0]) <= 1e-8 * abs(rl[0]), (i, taus[sel[i]], rs[sel[i]])
            assert abs(chi2[i, 0] - rc[0]) <= 1e-8 * abs(rc[0]), i
            assert abs(ld[i] - rd) <= 1e-8 * abs(rd), i
    _with_split_kt(api, run)


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-8)])
def test_batch_tqu_nside16(api, precision, tol):
    """Nside 16 TQU, l <= 47 (k = 6900), masks f_sky 0.5 / 0.7 / 0.9
    (n = 4800 / 6336 / 8256), six items across the (tau, r) grid."""
    _run(api, 16, 47, 6, precision, tol, nmaps=1)


def test_batch_rejects_mixed_bands(api):
    masks, taus, rs = synth.batch_workload(nside=8, lmax=15, rank=10, ngrid=2)
    m2 = synth.make_workload("other band", 8, 11, True, True, 20.0, synth.SPEC_NAMES, 10, 99)
    p1 = api.Problem.from_workload(masks[0])
    p2 = api.Problem.from_workload(m2)
    d1 = torch.zeros(p1.n, 1, dtype=torch.float64, device="cuda")
    d2 = torch.zeros(p2.n, 1, dtype=torch.float64, device="cuda")
    with pytest.raises(api.QMLError) as ei:
        api.loglike_batch([(p1, d1), (p2, d2)], [0, 1], torch.zeros(2, 6, 16, dtype=torch.float64, device="cuda"))
    assert ei.value.status == 1


def test_batch_schedules_agree_bitwise(api):
    """Worker count, CUDA-graph replay and the GEMM tile autotuner change the
    schedule only: every item's results are bit-identical across them."""
    masks, item_mask, item_cl, mapss, refs = _oracle(8, 15, 9, 2, 8)
    cl = torch.as_tensor(item_cl, device="cuda")
    outs = []
    saved = {k: api.tune_get(k) for k in ("batch_streams", "batch_graphs", "dgemm_autotune")}
    try:
        for precision in (0, 1):
            probs = [(api.Problem.from_workload(wl, precision=precision), td(mp))
                     for wl, mp in zip(masks, mapss)]
            res = []
            for streams, graphs, tune in ((1, 0, 0), (4, 1, 1), (3, 1, 1), (2, 0, 1)):
                api.tune_set("batch_streams", streams)
                api.tune_set("batch_graphs", graphs)
                api.tune_set("dgemm_autotune", tune)
                res.append([P.to_np(x) for x in api.loglike_batch(probs, item_mask, cl)])
            for r in res[1:]:
                for a, b in zip(res[0], r):
                    assert np.array_equal(a, b)
            outs.append(res[0])
    finally:
        for k, v in saved.items():
            api.tune_set(k, {"batch_streams": 4, "batch_graphs": 1, "dgemm_autotune": 1}[k]
                         if v is None else v)
    # and the graph-replayed results still match the oracle
    for i in range(len(refs)):
        assert np.abs(outs[0][0][i, :2] - refs[i][0]).max() <= 1e-10 * np.abs(refs[i][0]).max()
    assert "dgemm:" in api.tune_table()
