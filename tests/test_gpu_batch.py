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
