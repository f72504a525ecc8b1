"""Validation experiments of Sect. 4 run through the library (NEXT-3 of the
build): the mean-chi^2 likelihood scan of r (Eq. mean_chi2_likelihood) and
the Fisher-vs-scatter comparison over sky fractions (the multi-f_sky test).

Every likelihood and estimate comes from the C ABI (pix_loglike_batch,
qml_fisher, qml_estimate, qml_synthesize); what this module adds is the
small host-side reduction the experiments define: means and standard
deviations over simulations, and the normalisation and quantiles of a 1-D
likelihood on a grid.
"""
from __future__ import annotations

import numpy as np

from . import api, synth


def _td(x):
    import torch
    return torch.as_tensor(np.asarray(x), device="cuda").t().contiguous().t()


def mean_chi2_rscan(wl, r_grid, r_true=0.0, nsims=1000, tau=0.06, seed=7, precision=0):
    """Mean-chi^2 likelihood of r (Eq. mean_chi2_likelihood) on one mask.

    nsims maps are drawn at r_true (d = Y a + n, a ~ N(0, Lambda(r_true)),
    n ~ N(0, N)) and evaluated together at every grid point by one
    pix_loglike_batch call (the maps share each point's factor).  With
    m(r) = <-2 lnL(r)>_sims = <chi^2(r)> + ln|C(r)|, the likelihood is
    Lbar(r) ~ exp(-(m(r) - min m) / 2); its peak is the unbiasedness test
    (E[m(r)] is minimised exactly at r_true).  Returns a dict: the grid, m,
    Lbar normalised on the grid (trapezoid rule), the peak, the 68 % and 95 %
    upper limits with the prior r >= 0, the per-sim -2 lnL array, and sigma_1,
    the single-map error from the curvature of m at its minimum.
    """
    r_grid = np.asarray(r_grid, dtype=np.float64)
    prob = api.Problem.from_workload(wl, device=True, precision=precision)
    g = synth.rng(seed, synth.P_SIMS)
    cl_true = synth.spectra(wl.lmax, tau=tau, r=r_true)
    alm = synth.draw_alm(cl_true, wl.lmin, wl.lmax, wl.comps, nsims, g)
    maps = api.synthesize(prob, _td(alm), _td(synth.noise_draws(wl.G, nsims, g)))
    item_cl = np.stack([synth.spectra(wl.lmax, tau=tau, r=r) for r in r_grid])
    import torch
    lnl, chi2, logdet = api.loglike_batch([(prob, maps)], np.zeros(len(r_grid), dtype=np.int32),
                                          torch.as_tensor(item_cl, device="cuda"))
    m2 = -2.0 * lnl.cpu().numpy()[:, :nsims]     # (grid, sims)
    m = m2.mean(axis=1)
    like = np.exp(-0.5 * (m - m.min()))
    like /= float(np.sum(0.5 * (like[1:] + like[:-1]) * np.diff(r_grid)))
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (like[1:] + like[:-1]) * np.diff(r_grid))])
    upper = {q: float(np.interp(q, cdf, r_grid)) for q in (0.68, 0.95)}
    i0 = int(np.argmin(m))
    # curvature of m around its minimum (parabola through three grid points):
    # m = a (r - r0)^2 + c, so one map's error is sigma_1 = 1 / sqrt(a)
    j = min(max(i0, 1), len(r_grid) - 2)
    a = np.polyfit(r_grid[j - 1:j + 2], m[j - 1:j + 2], 2)[0]
    return {"r": r_grid, "m": m, "like": like, "r_peak": float(r_grid[i0]),
            "upper68": upper[0.68], "upper95": upper[0.95], "m2_per_sim": m2,
            "sigma1": float(1.0 / np.sqrt(a)) if a > 0 else float("nan"), "nsims": nsims}


def fsky_sweep(nside, lmax, cuts_deg, nsims=1000, rank=10, seed=9, spectrum="BB", precision=0):
    """Fisher error bars against the scatter of the deconvolved estimates over
    simulations, for several Galactic cuts |b| < b0 (QU; the multi-f_sky test).

    For each cut: qml_fisher gives F, nsims maps drawn from the fiducial model
    go through qml_estimate, and the standard deviation of C_hat over the maps
    is compared with sqrt((F^-1)_ll) for the chosen spectrum.  Returns a list
    of dicts (cut, f_sky, n, ells, sigma_fisher, sigma_empirical, ratio)."""
    out = []
    spec = ("EE", "BB", "EB")
    si = spec.index(spectrum)
    for j, b0 in enumerate(cuts_deg):
        wl = synth.make_workload(f"QU nside{nside} cut{b0}", nside, lmax, False, True, b0, spec,
                                 rank, 90 + j)
        prob = api.Problem.from_workload(wl, device=True, precision=precision)
        F, plan = api.fisher(prob)
        g = synth.rng(seed + j, synth.P_SIMS)
        alm = synth.draw_alm(wl.cl_fid, wl.lmin, wl.lmax, wl.comps, nsims, g)
        maps = api.synthesize(prob, _td(alm), _td(synth.noise_draws(wl.G, nsims, g)))
        est = plan.estimate(maps)
        plan.free()
        Fn = F.cpu().numpy()
        nl = wl.lmax - wl.lmin + 1
        rows = slice(si * nl, (si + 1) * nl)
        sig_f = np.sqrt(np.diag(np.linalg.inv(Fn)))[rows]
        c = est["cl_deconv"].cpu().numpy()[rows]
        sig_e = c.std(axis=1, ddof=1)
        npix = len(synth.healpix_ring_centres(nside)[0])
        out.append({"cut_deg": b0, "fsky": wl.npix_P / npix, "n": wl.n,
                    "ells": np.arange(wl.lmin, wl.lmax + 1), "sigma_fisher": sig_f,
                    "sigma_empirical": sig_e, "ratio": sig_e / sig_f,
                    "mean": c.mean(axis=1), "cl_fid": wl.cl_fid[[1, 2, 5][si], wl.lmin:]})
    return out
