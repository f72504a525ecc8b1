"""Seeded synthetic inputs shaped like the low-ell CMB workloads of the paper.

This module draws and lays out INPUTS only: HEALPix RING pixel centres, galactic
cut masks, beam and pixel-window transfer functions, power-spectrum templates,
dense noise covariances and Gaussian random numbers.  It contains none of the
estimator's arithmetic (no harmonics, no covariances of the signal, no solves),
so that the CUDA library and the CPU oracle can both be fed from it without
sharing any part of the method.

Recipe (stated once here, repeated in the design notes):

* Geometry: HEALPix RING pixel centres from the closed-form ring formulae of
  Gorski et al. (2005); a galactic cut keeps pixel p iff |z_p| >= sin(b0) - 1e-12
  with the map equator standing in for the galactic plane.
* Beam: Gaussian, FWHM = 2 x pixel size, pixel size = sqrt(4 pi / Npix);
  B_l = exp(-l(l+1) sigma_b^2 / 2), sigma_b = FWHM / sqrt(8 ln 2).
* Pixel window: healpy's tables are not available; the stand-in is the window
  of a spherical cap of the pixel's solid angle,
  p_l = [P_{l-1}(x0) - P_{l+1}(x0)] / [(2l+1)(1-x0)], x0 = 1 - Omega_pix/(2 pi).
* Spectra (muK^2): TT = 1000/(l(l+1)); EE = 0.05 TT + 0.02 exp(-(l-4)^2/8)
  (the bump scaled by (tau/0.06)^2 in the parameter scan); BB = 0.01 EE
  (+ 0.1 r TT in the scan); TE = 0.3 sqrt(TT EE); TB = EB = 0.
* Noise: N = sigma^2 I + G G^T, G_ij ~ N(0, sigma^2 / rank), sigma^2 = 1 muK^2,
  one matrix over all rows (T, Q and U rows fully coupled).
* Maps: harmonic coefficients a ~ N(0, Lambda) per (l, m) and a noise draw
  n = sigma eta_1 + G eta_2 (exactly N-distributed); the map itself is
  d = Y a + n, which each side forms with its own Y.

Seeds: numpy Generator(PCG64(2605_21149 + 100 * config + purpose)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2605_21149

# spectrum order used everywhere: index into cl[6][lmax+1]
SPEC_NAMES = ("TT", "EE", "BB", "TE", "TB", "EB")
SPEC_INDEX = {name: i for i, name in enumerate(SPEC_NAMES)}
# component pair (X, Y) of each spectrum, X, Y in {T=0, E=1, B=2}
SPEC_PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))

# purposes (seed offsets)
P_NOISE, P_MAPS, P_SIMS, P_GRID, P_EMU, P_MISC = 1, 2, 3, 4, 5, 6


def rng(config: int, purpose: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + 100 * config + purpose))


# ---------------------------------------------------------------------------
# HEALPix RING geometry (Gorski et al. 2005, Sect. 4)
# ---------------------------------------------------------------------------
def healpix_ring_centres(nside: int):
    """(theta, phi, z) of all 12 nside^2 pixel centres in RING order."""
    th, ph, zz = [], [], []
    ns = nside
    for i in range(1, 4 * ns):
        if i < ns:  # north polar cap
            z = 1.0 - i * i / (3.0 * ns * ns)
            npr = 4 * i
            phis = (np.pi / (2.0 * i)) * (np.arange(1, npr + 1) - 0.5)
        elif i <= 3 * ns:  # equatorial belt
            z = 4.0 / 3.0 - 2.0 * i / (3.0 * ns)
            npr = 4 * ns
            s = (i - ns + 1) % 2
            phis = (np.pi / (2.0 * ns)) * (np.arange(1, npr + 1) - 0.5 * s)
        else:  # south polar cap
            ip = 4 * ns - i
            z = -(1.0 - ip * ip / (3.0 * ns * ns))
            npr = 4 * ip
            phis = (np.pi / (2.0 * ip)) * (np.arange(1, npr + 1) - 0.5)
        zz.append(np.full(npr, z))
        ph.append(phis)
    z = np.concatenate(zz)
    phi = np.concatenate(ph)
    theta = np.arccos(np.clip(z, -1.0, 1.0))
    return theta, phi, z


def galactic_cut(z: np.ndarray, b0_deg: float) -> np.ndarray:
    """Indices of kept pixels: |z| >= sin(b0) (with a 1e-12 tie-break)."""
    return np.nonzero(np.abs(z) >= math.sin(math.radians(b0_deg)) - 1e-12)[0]


def fsky_cut_deg(fsky: float) -> float:
    """Galactic half-width b0 such that 1 - sin(b0) = fsky."""
    return math.degrees(math.asin(1.0 - fsky))


# ---------------------------------------------------------------------------
# transfer functions
# ---------------------------------------------------------------------------
def pixel_size(nside: int) -> float:
    return math.sqrt(4.0 * math.pi / (12 * nside * nside))


def gaussian_beam(lmax: int, fwhm: float) -> np.ndarray:
    sig = fwhm / math.sqrt(8.0 * math.log(2.0))
    ell = np.arange(lmax + 1, dtype=np.float64)
    return np.exp(-0.5 * ell * (ell + 1.0) * sig * sig)


def _legendre_table(lmax: int, x: float) -> np.ndarray:
    """P_0..P_lmax at one point by Bonnet's recurrence (input helper only)."""
    p = np.zeros(lmax + 1)
    p[0] = 1.0
    if lmax >= 1:
        p[1] = x
    for l in range(1, lmax):
        p[l + 1] = ((2 * l + 1) * x * p[l] - l * p[l - 1]) / (l + 1)
    return p


def cap_pixel_window(lmax: int, nside: int) -> np.ndarray:
    """Spherical-cap stand-in for the HEALPix pixel window (see module doc)."""
    omega = 4.0 * math.pi / (12 * nside * nside)
    x0 = 1.0 - omega / (2.0 * math.pi)
    p = _legendre_table(lmax + 1, x0)
    w = np.ones(lmax + 1)
    for l in range(1, lmax + 1):
        w[l] = (p[l - 1] - p[l + 1]) / ((2 * l + 1) * (1.0 - x0))
    return w


def transfer(lmax: int, nside: int) -> np.ndarray:
    """T_l = B_l p_l with FWHM = 2 x pixel size."""
    return gaussian_beam(lmax, 2.0 * pixel_size(nside)) * cap_pixel_window(lmax, nside)


# ---------------------------------------------------------------------------
# spectra templates
# ---------------------------------------------------------------------------
def spectra(lmax: int, tau: float = 0.06, r: float = 0.0,
            a_ee: float = 1.0, a_tt: float = 1.0) -> np.ndarray:
    """cl[6][lmax+1] in SPEC_NAMES order; entries below l = 2 are zero."""
    ell = np.arange(lmax + 1, dtype=np.float64)
    cl = np.zeros((6, lmax + 1))
    l2 = ell[2:]
    tt = a_tt * 1000.0 / (l2 * (l2 + 1.0))
    tt0 = 1000.0 / (l2 * (l2 + 1.0))
    ee = a_ee * (0.05 * tt0 + 0.02 * (tau / 0.06) ** 2 * np.exp(-((l2 - 4.0) ** 2) / 8.0))
    bb = 0.01 * ee + 0.1 * r * tt0
    cl[0, 2:] = tt
    cl[1, 2:] = ee
    cl[2, 2:] = bb
    cl[3, 2:] = 0.3 * np.sqrt(tt * ee)
    return cl


# ---------------------------------------------------------------------------
# noise
# ---------------------------------------------------------------------------
def noise_factor(n: int, rank: int, g: np.random.Generator, sigma2: float = 1.0):
    """G (n x rank) with N = sigma2 I + G G^T."""
    return g.normal(0.0, math.sqrt(sigma2 / rank), size=(n, rank))


def noise_matrix(G: np.ndarray, sigma2: float = 1.0) -> np.ndarray:
    """Dense N = sigma2 I + G G^T, column-major friendly (symmetric)."""
    n = G.shape[0]
    N = G @ G.T
    N[np.diag_indices(n)] += sigma2
    return N


def noise_draws(G: np.ndarray, nsims: int, g: np.random.Generator, sigma2: float = 1.0):
    """n = sigma eta_1 + G eta_2, shape (n, nsims); exactly N(0, N)."""
    n, r = G.shape
    return math.sqrt(sigma2) * g.normal(size=(n, nsims)) + G @ g.normal(size=(r, nsims))


# ---------------------------------------------------------------------------
# harmonic coefficient draws
# ---------------------------------------------------------------------------
def mode_count(lmin: int, lmax: int) -> int:
    return (lmax + 1) ** 2 - lmin ** 2


def draw_alm(cl: np.ndarray, lmin: int, lmax: int, comps: tuple, nsims: int,
             g: np.random.Generator, transfer_by_comp=None) -> np.ndarray:
    """Real harmonic coefficients a ~ N(0, Lambda), shape (k, nsims).

    Rows follow the library's column layout: component-major over `comps`
    (subset of (0=T, 1=E, 2=B)), then l ascending, then within l the 2l+1 real
    modes.  Lambda at each (l, m) is the 3x3 (T,E,B) block of cl restricted to
    `comps`; every real mode at l shares it.  The transfer function is NOT
    applied here (the library folds it into its own matrix).
    """
    k0 = mode_count(lmin, lmax)
    nc = len(comps)
    out = np.zeros((nc * k0, nsims))
    full = np.zeros((3, 3, lmax + 1))
    for s, (x, y) in enumerate(SPEC_PAIRS):
        full[x, y] = cl[s]
        full[y, x] = cl[s]
    for l in range(lmin, lmax + 1):
        lam = full[np.ix_(comps, comps, [l])][:, :, 0]
        w, v = np.linalg.eigh(lam)
        root = v * np.sqrt(np.clip(w, 0.0, None))
        z = g.normal(size=(nc, 2 * l + 1, nsims))
        a = np.einsum("ij,jmn->imn", root, z)
        off = l * l - lmin * lmin
        for c in range(nc):
            out[c * k0 + off: c * k0 + off + 2 * l + 1] = a[c]
    return out


# ---------------------------------------------------------------------------
# problem descriptions of the workloads
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    nside: int
    lmin: int
    lmax: int
    has_T: bool
    has_P: bool
    theta_T: np.ndarray
    phi_T: np.ndarray
    theta_P: np.ndarray
    phi_P: np.ndarray
    transfer_T: np.ndarray
    transfer_P: np.ndarray
    spec: tuple            # tuple of SPEC_INDEX values estimated
    cl_fid: np.ndarray     # (6, lmax+1)
    G: np.ndarray          # noise factor, n x rank
    sigma2: float = 1.0
    extra: dict = field(default_factory=dict)

    @property
    def npix_T(self):
        return len(self.theta_T) if self.has_T else 0

    @property
    def npix_P(self):
        return len(self.theta_P) if self.has_P else 0

    @property
    def n(self):
        return self.npix_T + 2 * self.npix_P

    @property
    def comps(self):
        return ((0,) if self.has_T else ()) + ((1, 2) if self.has_P else ())

    @property
    def k0(self):
        return mode_count(self.lmin, self.lmax)

    @property
    def k(self):
        return len(self.comps) * self.k0

    @property
    def nl(self):
        return self.lmax - self.lmin + 1

    def N(self):
        return noise_matrix(self.G, self.sigma2)


def make_workload(name: str, nside: int, lmax: int, has_T: bool, has_P: bool,
                  b0_deg: float, spec, rank: int, config: int, lmin: int = 2,
                  geometry=None, cl=None) -> Workload:
    if geometry is None:
        theta, phi, z = healpix_ring_centres(nside)
        keep = galactic_cut(z, b0_deg)
        theta, phi = theta[keep], phi[keep]
    else:
        theta, phi = geometry
    tl = transfer(lmax, nside) if nside > 0 else np.ones(lmax + 1)
    npix = len(theta)
    n = (npix if has_T else 0) + (2 * npix if has_P else 0)
    G = noise_factor(n, rank, rng(config, P_NOISE))
    if cl is None:
        cl = spectra(lmax)
    e = np.empty(0)
    return Workload(name=name, nside=nside, lmin=lmin, lmax=lmax, has_T=has_T, has_P=has_P,
                    theta_T=theta if has_T else e, phi_T=phi if has_T else e,
                    theta_P=theta if has_P else e, phi_P=phi if has_P else e,
                    transfer_T=tl.copy(), transfer_P=tl.copy(),
                    spec=tuple(SPEC_INDEX[s] if isinstance(s, str) else s for s in spec),
                    cl_fid=cl, G=G)


def workload(config: int, scale: str = "full") -> Workload:
    """The paper-shaped workloads.

    config 0: T only, Nside 8, |b| < 20 deg cut (480 px), l = 2..16, rank-10 N.
    config 1: TQU, Nside 16, |b| < 20 deg cut (3 x 1984 rows), l = 2..47, rank-200 N.
    config 2: QU, Nside 32, f_sky 0.7 cut (2 x 8576 rows), l = 2..95, rank-200 N.
    config 3: TQU, Nside 16, batched scan setup (masks f_sky 0.5/0.7/0.9).
    scale="small" shrinks configs 1-2 (Nside 8, lmax 2 Nside-1) for fast tests.
    """
    if config == 0:
        return make_workload("T nside8 lmax16", 8, 16, True, False, 20.0, ("TT",), 10, 0)
    if config == 1:
        if scale == "small":
            return make_workload("TQU nside8 lmax15", 8, 15, True, True, 20.0,
                                 SPEC_NAMES, 40, 1)
        return make_workload("TQU nside16 lmax47", 16, 47, True, True, 20.0, SPEC_NAMES, 200, 1)
    if config == 2:
        if scale == "small":
            return make_workload("QU nside8 lmax23", 8, 23, False, True, fsky_cut_deg(0.7),
                                 ("EE", "BB", "EB"), 40, 2)
        return make_workload("QU nside32 lmax95", 32, 95, False, True, fsky_cut_deg(0.7),
                             ("EE", "BB", "EB"), 200, 2)
    raise ValueError(f"unknown config {config}")


def gauss_legendre_grid(lmax: int):
    """Full-sky Gauss-Legendre grid: lmax+1 rings in cos(theta) x 2 lmax + 2
    uniform longitudes; returns (theta, phi, w) with sum(w) = 4 pi."""
    x, wx = np.polynomial.legendre.leggauss(lmax + 1)
    nphi = 2 * lmax + 2
    ph = 2.0 * np.pi * np.arange(nphi) / nphi
    theta = np.repeat(np.arccos(x), nphi)
    phi = np.tile(ph, lmax + 1)
    w = np.repeat(wx * (2.0 * np.pi / nphi), nphi)
    return theta, phi, w


def batch_workload(nside: int = 16, lmax: int = 47, fskies=(0.5, 0.7, 0.9), rank: int = 200,
                   ngrid: int = 64, config: int = 3):
    """The parameter-scan workload: TQU masks at the given sky fractions (each
    its own seeded rank-`rank` noise), and the (tau, r) grid of the scan,
    tau in [0.03, 0.09] (the EE reionisation bump scales as tau^2), r in
    [0, 0.1] (BB gains 0.1 r TT).  Item i = (grid point i, mask i mod nmask).
    Returns (masks, taus, rs)."""
    masks = []
    for j, fs in enumerate(fskies):
        masks.append(make_workload(f"TQU nside{nside} fsky{fs}", nside, lmax, True, True,
                                   fsky_cut_deg(fs), SPEC_NAMES, rank, 10 * config + j))
    tau = np.linspace(0.03, 0.09, ngrid)
    r = np.linspace(0.0, 0.1, ngrid)
    T, R = np.meshgrid(tau, r, indexing="ij")
    return masks, T.reshape(-1), R.reshape(-1)


def batch_item_spectra(lmax: int, taus, rs) -> np.ndarray:
    """item_cl array (nitems, 6, lmax+1) for the scan grid."""
    return np.stack([spectra(lmax, tau=t, r=r) for t, r in zip(taus, rs)])

