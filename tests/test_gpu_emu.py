"""lnL emulator (emu_* entry points): gradients of the training kernels
against the oracle MLP (P15), fitting accuracy, the fallback flags, and an
end-to-end run on exact lnL labels from pix_loglike_batch with the
|dlnL| <= 0.05 audit on the accepted points (fallback threshold calibrated
on held-out labels)."""
import numpy as np
import pytest

from oracle import emulator as E
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


@pytest.mark.parametrize("width,depth", [(64, 2), (256, 4)])
def test_emu_gradients_match_oracle(api, width, depth):
    emu = api.Emulator(np.zeros(4), np.ones(4), width=width, depth=depth, seed=3)
    rng = np.random.default_rng(width + depth)
    n = 48
    x = np.zeros((n, 16))
    x[:, :4] = rng.uniform(-1, 1, size=(n, 4))
    t = rng.normal(size=n)
    loss, g = emu.loss_grad(x, t)
    p = emu.params(0).astype(np.float64)
    # the oracle takes the library's bf16 roundings of weights, activations and
    # back-propagated errors; what is left is float32 accumulation and the
    # rare bf16 rounding decision a float32 value takes differently
    lref, gref = E.loss_and_grad(p, x, t, 16, width, depth, 16, bf16_inputs=True,
                                 bf16_grads=True)
    assert abs(loss - lref) <= 1e-4 * abs(lref)
    d = np.abs(g - gref)
    gmax = np.abs(gref).max()
    assert d.max() <= 3e-3 * gmax, d.max() / gmax
    assert d.mean() <= 1e-4 * gmax, d.mean() / gmax
    emu.free()


def test_emu_fits_and_flags(api):
    rng = np.random.default_rng(5)
    lo, hi = -np.ones(4), np.ones(4)

    def f(th):
        return (-0.5 * (th ** 2 * np.array([30.0, 10.0, 5.0, 2.0])).sum(axis=1)
                + 0.3 * np.sin(2 * th[:, 0]) * th[:, 1] + 5.0)

    th = rng.uniform(-1, 1, size=(4096, 4))
    emu = api.Emulator(lo, hi, seed=7)
    l0, l1 = emu.train(th, f(th), epochs=40, batch=64, lr=1e-3)
    # the loss is on the residual after the degree-6 baseline, in units of
    # its own RMS: the network explains most of what the polynomial leaves
    assert l0 < 0.05 and l1 < 0.05
    test = rng.uniform(-1, 1, size=(1024, 4))
    pred, flags = emu.predict(test, tol=0.02)
    err = np.abs(pred - f(test))
    assert np.max(err[flags == 0]) <= 0.02 + 1e-9
    assert flags.mean() < 0.2
    out = rng.uniform(1.01, 1.2, size=(16, 4))
    _, fo = emu.predict(out)
    assert np.all(fo == 1)
    emu.free()


def _lnl_exact(api, prob, maps, lmax, thetas):
    cl = np.stack([synth.spectra(lmax, tau=t[0], r=t[1], a_ee=t[2], a_tt=t[3]) for t in thetas])
    lnl, _, _ = api.loglike_batch([(prob, maps)], np.zeros(len(thetas), dtype=np.int32),
                                  torch.as_tensor(cl, device="cuda"))
    return lnl[:, 0].cpu().numpy()


def test_emu_end_to_end_exact_labels(api):
    """TQU Nside 8, f_sky 0.7, l <= 15; theta = (tau, r, A_EE, A_TT) in
    [0.042, 0.078] x [0, 0.1] x [0.7, 1.3]^2; 8192 exact labels (an eighth
    held out for the fallback calibration)."""
    wl = synth.make_workload("emu TQU nside8", 8, 15, True, True, synth.fsky_cut_deg(0.7),
                             synth.SPEC_NAMES, 20, 40)
    prob = api.Problem.from_workload(wl)
    g = synth.rng(40, synth.P_EMU)
    cl0 = synth.spectra(wl.lmax)
    alm = synth.draw_alm(cl0, wl.lmin, wl.lmax, wl.comps, 1, g)
    noise = synth.noise_draws(wl.G, 1, g)
    td = lambda x: torch.as_tensor(x, device="cuda").t().contiguous().t()
    maps = api.synthesize(prob, td(alm), td(noise))
    lo = np.array([0.042, 0.0, 0.7, 0.7])
    hi = np.array([0.078, 0.1, 1.3, 1.3])
    th = lo + (hi - lo) * g.uniform(size=(8192, 4))
    y = _lnl_exact(api, prob, maps, wl.lmax, th)
    emu = api.Emulator(lo, hi, seed=11)
    emu.train(th, y, epochs=100, batch=64, lr=1e-3)
    test = lo + (hi - lo) * g.uniform(size=(1024, 4))
    pred, flags = emu.predict(test, tol=0.05)
    exact = _lnl_exact(api, prob, maps, wl.lmax, test)
    acc = flags == 0
    err = np.abs(pred - exact)
    worst = np.argmax(np.where(acc, err, -1.0))
    print("threshold", emu.threshold(0.05), "accepted", acc.mean(), "max err", err[acc].max(), "median", np.median(err[acc]),
          "worst x", 2 * (test[worst] - lo) / (hi - lo) - 1)
    assert acc.mean() > 0.5
    assert err[acc].max() <= 0.05

    # what the network gains over the method without it
    # (1) accuracy: the same float64 least-squares cubic the emulator starts
    #     from, alone, misses by far more than the trained network
    def cubic_features(t):
        x = 2 * (t - lo) / (hi - lo) - 1
        cols = [np.ones(len(x))] + [x[:, i] for i in range(4)]
        cols += [x[:, i] * x[:, j] for i in range(4) for j in range(i, 4)]
        cols += [x[:, i] * x[:, j] * x[:, l] for i in range(4) for j in range(i, 4) for l in range(j, 4)]
        return np.stack(cols, axis=1)

    coef, *_ = np.linalg.lstsq(cubic_features(th), y, rcond=None)
    err_poly = np.abs(cubic_features(test) @ coef - exact)
    print("median |dlnL| network", np.median(err), "cubic alone", np.median(err_poly))
    assert np.median(err) * 10 <= np.median(err_poly)
    # (2) cost: emulating with the exact fallback beats evaluating every point
    import time
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _lnl_exact(api, prob, maps, wl.lmax, test)
    torch.cuda.synchronize()
    t_exact = time.perf_counter() - t0
    t0 = time.perf_counter()
    pred2, flags2 = emu.predict(test, tol=0.05)
    fb = np.flatnonzero(flags2)
    if len(fb):
        _lnl_exact(api, prob, maps, wl.lmax, test[fb])
    torch.cuda.synchronize()
    t_emu = time.perf_counter() - t0
    print("exact", t_exact, "s; emulator with fallback", t_emu, "s")
    assert t_emu < t_exact
    emu.free()


@pytest.mark.parametrize("width,depth", [(256, 4), (64, 2), (192, 1)])
def test_emu_tcgen05_inference_matches_wmma(api, width, depth):
    """Inference layers after the first run on tcgen05 (bias and GELU fused);
    tuning key emu_tc = 0 runs every layer through the WMMA product instead.
    Same trained network, same points: the two differ only in float32
    accumulation order (and the bf16 rounding it can flip), far inside the
    0.05 audit tolerance; 70000 points in passes of 65536 (tuning key
    emu_chunk) cover a second pass and a ragged last tile."""
    rng = np.random.default_rng(9)
    th = rng.uniform(-1, 1, size=(2048, 3))
    y = -0.5 * (th ** 2 * np.array([20.0, 6.0, 2.0])).sum(axis=1) + np.sin(3 * th[:, 0])
    emu = api.Emulator(-np.ones(3), np.ones(3), width=width, depth=depth, seed=4)
    emu.train(th, y, epochs=10, batch=64)
    test = rng.uniform(-1.05, 1.05, size=(70000, 3))
    api.tune_set("emu_chunk", 65536)
    try:
        pred_tc, flags_tc = emu.predict(test, tol=0.05)
        api.tune_set("emu_tc", 0)
        pred_w, flags_w = emu.predict(test, tol=0.05)
    finally:
        api.tune_set("emu_tc", 1)
        api.tune_set("emu_chunk", 262144)
    d = np.abs(pred_tc - pred_w)
    assert np.all(np.isfinite(pred_tc))
    assert d.max() <= 5e-3, d.max()
    assert np.mean(flags_tc == flags_w) >= 0.99
    emu.free()


def _multi_indices(d, deg):
    """The baseline's term order (emu_baseline): by total degree, then the
    first exponent from the remaining degree down, and so on."""
    out = []

    def rec(prefix, left, pos):
        if pos == d - 1:
            out.append(prefix + [left])
            return
        for k in range(left, -1, -1):
            rec(prefix + [k], left - k, pos + 1)

    for t in range(deg + 1):
        rec([], t, 0)
    return out


def _features(x, nf):
    """The baseline's features: products of Legendre polynomials of the
    normalised coordinates, total degree D with C(D + d, d) = nf terms."""
    from math import comb
    from numpy.polynomial import legendre
    n, d = x.shape
    deg = next(D for D in range(20) if comb(D + d, d) == nf)
    leg = [[legendre.legval(x[:, i], [0] * k + [1]) for k in range(deg + 1)] for i in range(d)]
    cols = [np.prod([leg[i][m[i]] for i in range(d)], axis=0) for m in _multi_indices(d, deg)]
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("width,depth", [(256, 4), (64, 2), (192, 1)])
def test_emu_tcgen05_inference_matches_oracle(api, width, depth):
    """emu_predict on tcgen05 (every layer, bias and GELU fused) against the
    oracle MLP's forward pass per point and per head: lnL = q(x) + sigma
    (f_0 + f_1) / 2 with the library's own baseline coefficients, the oracle
    taking the same bf16 roundings of weights and layer inputs (float64
    otherwise).  70000 points in passes of 65536 (tuning key emu_chunk): a
    second pass and a ragged last 128-row tile."""
    rng = np.random.default_rng(19)
    th = rng.uniform(-1, 1, size=(2048, 3))
    y = -0.5 * (th ** 2 * np.array([20.0, 6.0, 2.0])).sum(axis=1) + np.sin(3 * th[:, 0])
    emu = api.Emulator(-np.ones(3), np.ones(3), width=width, depth=depth, seed=6)
    emu.train(th, y, epochs=10, batch=64)
    test = rng.uniform(-1.05, 1.05, size=(70000, 3))
    api.tune_set("emu_chunk", 65536)
    try:
        pred, flags = emu.predict(test, tol=0.05)
    finally:
        api.tune_set("emu_chunk", 262144)
    coef, sigma = emu.baseline()
    X = np.zeros((len(test), 16))
    X[:, :3] = test  # box [-1, 1]^3: normalised coordinates are theta itself
    heads = [E.forward(emu.params(h).astype(np.float64), X, 16, width, depth, 16,
                       bf16_inputs=True)[0] for h in (0, 1)]
    ref = _features(test, len(coef)) @ coef + sigma * 0.5 * (heads[0] + heads[1])
    d = np.abs(pred - ref)
    assert np.all(np.isfinite(pred))
    assert d.max() <= 5e-3, d.max()
    # the network term alone, relative to its own scale
    net = 0.5 * (heads[0] + heads[1])
    net_gpu = (pred - _features(test, len(coef)) @ coef) / sigma
    assert np.abs(net_gpu - net).max() <= 1e-2 * max(np.abs(net).max(), 1.0)
    # the fallback flags use the same head disagreement
    outside = (np.abs(test) > 0.97).any(axis=1)
    thr, _ = emu.threshold(0.05)
    flags_ref = outside | (sigma * np.abs(heads[0] - heads[1]) > thr)
    assert np.mean(flags == flags_ref) >= 0.99
    emu.free()


def test_emu_baseline_is_least_squares(api):
    """The float64 baseline is the least-squares fit of the documented
    Legendre features (n = 480 labels, no hold-out below 512: all of them
    fit): its coefficients equal numpy's solution of the same problem."""
    rng = np.random.default_rng(23)
    th = rng.uniform(-1, 1, size=(480, 2))
    y = np.exp(th[:, 0]) * np.cos(2 * th[:, 1]) + 3.0 * th[:, 1]
    emu = api.Emulator(-np.ones(2), np.ones(2), width=64, depth=1, seed=3)
    emu.train(th, y, epochs=1, batch=64)
    coef, sigma = emu.baseline()
    emu.free()
    assert len(coef) == 28  # total degree 6 in two dimensions: 16 labels per term
    ref, *_ = np.linalg.lstsq(_features(th, 28), y, rcond=None)
    assert np.abs(coef - ref).max() <= 1e-9 * np.abs(ref).max()
    resid = y - _features(th, 28) @ ref
    assert abs(sigma - np.sqrt(np.mean(resid ** 2))) <= 1e-9 * sigma
