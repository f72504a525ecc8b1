"""The Sect. 4 validation experiments through the library (paper_2605_21149_gb300.
validate): the mean-chi^2 likelihood scan of r (Eq. mean_chi2_likelihood)
peaks at the input r within its Monte Carlo error, and its per-map -2 lnL
equals the oracle's pixel likelihood; the scatter of the deconvolved BB
estimates over simulations matches the Fisher error bars sqrt((F^-1)_ll) at
every multipole for sky fractions from the full sky to a +-40 deg cut, and
their mean matches the input spectrum."""
import numpy as np
import pytest

from oracle import harmonic, qml
from paper_2605_21149_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def val():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_21149_gb300 import build, validate
    build.build()
    return validate


def _rscan_workload():
    return synth.make_workload("QU nside8 rscan", 8, 15, False, True, synth.fsky_cut_deg(0.7),
                               ("EE", "BB", "EB"), 10, 80)


def test_mean_chi2_rscan_peaks_at_r_true(val):
    """1000 maps drawn at r = 0.05, 31 grid points on [0, 0.1]: the peak of
    Lbar(r) lies within 4 sigma_1 / sqrt(N) (or one grid step) of r_true."""
    wl = _rscan_workload()
    grid = np.linspace(0.0, 0.1, 31)
    out = val.mean_chi2_rscan(wl, grid, r_true=0.05, nsims=1000)
    tol = max(4.0 * out["sigma1"] / np.sqrt(out["nsims"]), grid[1] - grid[0])
    print("r_peak", out["r_peak"], "sigma_1", out["sigma1"], "tol", tol)
    assert np.isfinite(out["sigma1"])
    assert abs(out["r_peak"] - 0.05) <= tol
    # the normalised likelihood integrates to one on the grid and is monotone
    # away from the peak
    assert abs(np.sum(0.5 * (out["like"][1:] + out["like"][:-1]) * np.diff(grid)) - 1) < 1e-12


def test_mean_chi2_rscan_zero_input_gives_upper_limits(val):
    """r_true = 0 (the paper's case): the peak sits at the lower edge r = 0 and
    the 68 % limit lies below the 95 % one."""
    out = val.mean_chi2_rscan(_rscan_workload(), np.linspace(0.0, 0.02, 31), r_true=0.0,
                              nsims=1000)
    print("r_peak", out["r_peak"], "68%", out["upper68"], "95%", out["upper95"])
    assert out["r_peak"] <= 2 * out["sigma1"] / np.sqrt(out["nsims"]) + 1e-12
    assert 0 < out["upper68"] < out["upper95"] <= 0.02


def test_rscan_per_map_matches_oracle(val):
    """-2 lnL of the first maps at three grid points against the oracle's pixel
    likelihood on the same seeded maps (1e-10 relative)."""
    wl = _rscan_workload()
    grid = np.array([0.0, 0.03, 0.1])
    out = val.mean_chi2_rscan(wl, grid, r_true=0.05, nsims=4, seed=7)
    g = synth.rng(7, synth.P_SIMS)
    cl_true = synth.spectra(wl.lmax, tau=0.06, r=0.05)
    alm = synth.draw_alm(cl_true, wl.lmin, wl.lmax, wl.comps, 4, g)
    Y = harmonic.build_Y_for(wl)
    maps = qml.simulate(Y, alm, synth.noise_draws(wl.G, 4, g))
    for i, r in enumerate(grid):
        C = qml.total_cov(Y, synth.spectra(wl.lmax, tau=0.06, r=r), wl.comps, wl.lmin, wl.lmax,
                          wl.N())
        lnl, _, _ = qml.loglike(C, maps)
        ref = -2.0 * lnl
        assert np.abs(out["m2_per_sim"][i] - ref).max() <= 1e-10 * np.abs(ref).max(), r


def test_fsky_sweep_scatter_matches_fisher(val):
    """QU Nside 8, l = 2..14, cuts 0 (full sky), 10, 18, 30, 40 deg, 2000 maps
    each: per multipole, the BB scatter over maps agrees with the Fisher error
    bar within 5 standard errors of a standard deviation, 5 / sqrt(2 N), and
    the mean agrees with the input BB within 5 sigma / sqrt(N)."""
    nsims = 2000
    rows = val.fsky_sweep(8, 14, (0.0, 10.0, 18.0, 30.0, 40.0), nsims=nsims)
    fsk = [r["fsky"] for r in rows]
    assert fsk[0] == 1.0 and all(a > b for a, b in zip(fsk, fsk[1:]))
    for r in rows:
        print(f"cut {r['cut_deg']:4.0f} f_sky {r['fsky']:.2f} ratio "
              f"{r['ratio'].min():.3f}..{r['ratio'].max():.3f}")
        assert np.all(np.abs(r["ratio"] - 1.0) <= 5.0 / np.sqrt(2 * nsims)), r["ratio"]
        pull = (r["mean"] - r["cl_fid"]) / (r["sigma_fisher"] / np.sqrt(nsims))
        assert np.all(np.abs(pull) <= 5.0), pull
    # error bars grow as the sky shrinks
    assert np.all(rows[-1]["sigma_fisher"] > rows[0]["sigma_fisher"])
