"""Seeded synthetic inputs shaped like the paper's workloads.

The paper simulates with MIST v1.2 isochrones, Tiny Tim PSFs and PySynphot zero-points
(Section 2.2, Section 3.1).  None of those data sets is available here, so this module makes
seeded stand-ins with the same shapes: isochrone grids of ages x [Fe/H] x masses with
per-band absolute magnitudes, Moffat PSFs, per-band exposure times and zero-points, and the
model-parameter vectors of Table 1.  Both the CUDA path and the CPU oracle receive these
arrays as inputs; the module computes no step of the forward model itself (no weights, no
Poisson draws, no fluxes, no histograms).

Workloads (sizes as stated in the build's configuration list):

* ``tiny``    64x64, 2 bands, one isochrone of 200 masses (0.1-2 Msun, top 15% on a giant
              branch), Npix = 100, no dust / PSF / noise.
* ``full``    256x256, 2 bands, 7 age bins (log age 6.5-10.1) x 7 [Fe/H] (-0.8..-0.2) x 300
              masses, Gaussian MDF (mean -0.5, sigma 0.2), log-normal dust screen
              (mu -0.5, sigma 0.1, F_dust 0.5), 25x25 Moffat PSF, sky + photon noise,
              log10 Npix in {2, 3, 4, 5} with the distance that keeps surface brightness fixed.
* ``batch``   512 parameter sets drawn uniformly over the paper's priors (Section 3.1) on the
              ``tiny`` isochrone, image sizes 128..512 (step 16), log10 Npix 1..6.
* ``large``   1024x1024, 3 bands, 10 ages x 9 [Fe/H] x 400 masses, log10 Npix 5..6.5.
* ``surrogate`` the ``full`` physics at 64x64 with the 12 free parameters drawn over a box.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# Per-band instrument constants.  Band 0 is the red (F814W-like) band and gives the
# magnitude axis; band 1 is the blue (F475W-like) band.  Exposure times of bands 0/1 are the
# PHAT values quoted in Section 3.1; zero-points and extinction ratios A_b / E(B-V) are
# synthetic stand-ins for the PySynphot and Schlafly & Finkbeiner values.
EXPTIME = (3235.0, 3620.0, 3000.0, 3000.0)
ZEROPOINT = (25.94, 26.05, 25.50, 25.50)
R_EXT = (1.526, 3.268, 0.850, 0.850)

FLAG_DUST = 1
FLAG_NOISE = 2
FLAG_KAHAN = 4
FLAG_SIGMA_SQRTSUM = 8
FLAG_POOL = 16                      # total-count sampler for the points below lambda 640

LL_PAPER = 0
LL_POISSON = 1

MAX_BANDS = 4
MAX_SFH = 16


@dataclasses.dataclass
class Isochrones:
    log_age: np.ndarray   # [n_ages]            log10 years
    feh: np.ndarray       # [n_feh]             [Fe/H] grid
    mass: np.ndarray      # [n_ages, n_feh, n_mass]  ascending initial masses (Msun)
    abs_mag: np.ndarray   # [n_ages, n_feh, n_mass, n_bands]  absolute magnitudes

    @property
    def n_points(self) -> int:
        return int(self.mass.size)


@dataclasses.dataclass
class Params:
    """One point of the model-parameter space (Table 1): non-parametric SFH (S5) bins in
    log10 stars per pixel, Gaussian MDF mean/width (M2/M3; width 0 selects one grid
    metallicity), dust median log10 E(B-V) and log-normal width (E1-E3), distance modulus."""
    log_sfh: np.ndarray
    feh_mean: float = -0.5
    feh_sigma: float = 0.2
    log_ebv: float = -0.5
    dust_sigma: float = 0.0
    dmod: float = 25.0

    def vector(self) -> np.ndarray:
        return np.concatenate([np.asarray(self.log_sfh, np.float64),
                               [self.feh_mean, self.feh_sigma, self.log_ebv,
                                self.dust_sigma, self.dmod]])


@dataclasses.dataclass
class Workload:
    name: str
    iso: Isochrones
    n_bands: int
    n_im: int
    params: List[Params]
    n_ims: List[int]
    imf_slope: float = 2.35
    imf: int = 0                              # 0 power law (imf_slope), 1 Kroupa (2001)
    exptime: Sequence[float] = EXPTIME
    zeropoint: Sequence[float] = ZEROPOINT
    sky: Sequence[float] = (0.0, 0.0, 0.0, 0.0)
    r_ext: Sequence[float] = R_EXT
    f_dust: float = 0.5
    mdf_cut: float = 0.01
    psf: Optional[np.ndarray] = None          # [n_bands, S, S] or [16, n_bands, S, S] float32, or None
    hess_nx: int = 100
    hess_ny: int = 100
    hess_c_lo: float = 0.0
    hess_m_lo: float = 0.0
    hess_width: float = 0.05
    seed: int = 1
    flags: int = 0
    ll_mode: int = LL_PAPER

    @property
    def n_sets(self) -> int:
        return len(self.params)


# ----------------------------------------------------------------------------------------
# isochrones
# ----------------------------------------------------------------------------------------

def _smooth_jitter(rng: np.random.Generator, x: np.ndarray, amp: float) -> np.ndarray:
    """Smooth seeded wiggle of peak amplitude <= amp along x in [0, 1]."""
    out = np.zeros_like(x)
    for _ in range(3):
        f = rng.uniform(0.5, 3.0)
        ph = rng.uniform(0.0, 2 * math.pi)
        out += np.sin(2 * math.pi * f * x + ph)
    return amp * out / 3.0


def make_isochrones(seed: int, log_ages: Sequence[float], fehs: Sequence[float], n_mass: int,
                    n_bands: int = 2, m_min: float = 0.1, m_max: Optional[float] = None,
                    giant_frac: Optional[float] = None) -> Isochrones:
    """Seeded stand-in for a MIST isochrone grid.

    Main sequence: L ~ m^4 below 1 Msun, m^3 above (red-band magnitude 4.1 at 1 Msun), colour
    bluer with mass and redder with [Fe/H]; a smooth seeded +-0.02 mag jitter per band.  Masses
    above the age's turnoff (or the top ``giant_frac`` of the mass grid) sit on a giant branch
    3-6 mag brighter than the turnoff and 0.5-1.5 mag redder.
    """
    rng = np.random.default_rng(seed)
    log_ages = np.asarray(log_ages, np.float64)
    fehs = np.asarray(fehs, np.float64)
    n_a, n_f = len(log_ages), len(fehs)
    mass = np.zeros((n_a, n_f, n_mass))
    mags = np.zeros((n_a, n_f, n_mass, n_bands))
    for j, la in enumerate(log_ages):
        m_to = float(np.clip(10.0 ** (-0.4 * (la - 10.0)), 0.9, 40.0))
        hi = m_max if m_max is not None else 1.15 * m_to
        m = np.geomspace(m_min, hi, n_mass)
        if giant_frac is not None:
            first_giant = int(round(n_mass * (1.0 - giant_frac)))
            m_to = float(m[first_giant - 1])
        else:
            first_giant = int(np.searchsorted(m, m_to, side="right"))
        lm = np.log10(m)
        for k, fe in enumerate(fehs):
            mred = np.where(lm <= 0.0, 4.1 - 10.0 * lm, 4.1 - 7.5 * lm) + 0.1 * fe
            col = 0.9 - 1.5 * lm + 0.3 * fe
            lto = math.log10(m_to)
            mred_to = (4.1 - 10.0 * lto if lto <= 0 else 4.1 - 7.5 * lto) + 0.1 * fe
            col_to = 0.9 - 1.5 * lto + 0.3 * fe
            ng = n_mass - first_giant
            if ng > 0:
                s = np.linspace(0.0, 1.0, ng) if ng > 1 else np.zeros(1)
                mred[first_giant:] = mred_to - (3.0 + 3.0 * s)
                col[first_giant:] = col_to + 0.5 + 1.0 * s + 0.3 * fe
            x = (lm - lm[0]) / max(lm[-1] - lm[0], 1e-12)
            mags[j, k, :, 0] = mred + _smooth_jitter(rng, x, 0.02)
            mags[j, k, :, 1] = mred + col + _smooth_jitter(rng, x, 0.02)
            for b in range(2, n_bands):
                mags[j, k, :, b] = mred - (0.35 + 0.1 * b) * col + _smooth_jitter(rng, x, 0.02)
            mass[j, k] = m
    return Isochrones(log_ages, fehs, mass, mags)


def moffat_psf(size: int, fwhm: Sequence[float], beta: float = 2.5,
               n_bands: int = 2, shift: Sequence[float] = (0.0, 0.0)) -> np.ndarray:
    """Moffat PSF per band on a size x size grid, centred (plus an optional sub-pixel shift),
    normalised to unit sum in float64 and returned as float32 [n_bands, size, size]."""
    r = size // 2
    yy, xx = np.mgrid[-r:r + 1, -r:r + 1].astype(np.float64)
    out = np.zeros((n_bands, size, size), np.float32)
    for b in range(n_bands):
        alpha = fwhm[b] / (2.0 * math.sqrt(2.0 ** (1.0 / beta) - 1.0))
        rr = ((xx - shift[0]) ** 2 + (yy - shift[1]) ** 2) / alpha ** 2
        k = (1.0 + rr) ** (-beta)
        out[b] = (k / k.sum()).astype(np.float32)
    return out


def subpixel_psf_grid(size: int, fwhm: Sequence[float], beta: float = 2.5,
                      n_bands: int = 2) -> np.ndarray:
    """The 4x4 grid of sub-pixel PSFs (Section 2.2): region (ry, rx) of the image gets the Moffat
    PSF shifted by ((rx + 1/2)/4 - 1/2, (ry + 1/2)/4 - 1/2) pixels; [16, n_bands, S, S]."""
    out = np.zeros((16, n_bands, size, size), np.float32)
    for ry in range(4):
        for rx in range(4):
            out[4 * ry + rx] = moffat_psf(size, fwhm, beta, n_bands,
                                          shift=((rx + 0.5) / 4 - 0.5, (ry + 0.5) / 4 - 0.5))
    return out


def constant_sfr_log_sfh(log_age_edges: Sequence[float], npix: float) -> np.ndarray:
    """log10 stars/pixel per bin for a constant star-formation rate summing to npix."""
    e = 10.0 ** np.asarray(log_age_edges, np.float64)
    w = np.diff(e)
    return np.log10(npix * w / w.sum())


# ----------------------------------------------------------------------------------------
# the named workloads
# ----------------------------------------------------------------------------------------

TINY_LOG_AGE = 10.0


def tiny(seed: int = 1, n_im: int = 64, npix: float = 100.0) -> Workload:
    iso = make_isochrones(seed=11, log_ages=[TINY_LOG_AGE], fehs=[-0.5], n_mass=200,
                          n_bands=2, m_min=0.1, m_max=2.0, giant_frac=0.15)
    p = Params(log_sfh=np.array([math.log10(npix)]), feh_mean=-0.5, feh_sigma=0.0,
               log_ebv=-1.0, dust_sigma=0.0, dmod=25.0)
    return Workload("tiny", iso, 2, n_im, [p], [n_im], psf=None,
                    hess_c_lo=-1.0, hess_m_lo=21.0, seed=seed, flags=0)


FULL_LOG_AGES = (6.5, 7.1, 7.7, 8.3, 8.9, 9.5, 10.1)
FULL_FEH = (-0.8, -0.7, -0.6, -0.5, -0.4, -0.3, -0.2)


def _edges(mid: Sequence[float], top: float = 10.15) -> List[float]:
    m = list(mid)
    e = [m[0] - 0.5 * (m[1] - m[0])]
    e += [0.5 * (a + b) for a, b in zip(m[:-1], m[1:])]
    e.append(min(m[-1] + 0.5 * (m[-1] - m[-2]), top))
    return e


def full(seed: int = 2, n_im: int = 256, log_npix: float = 2.0, sky: float = 0.0,
         noise: bool = True, psf: bool = True, dust: bool = True, psf_grid: bool = False) -> Workload:
    iso = make_isochrones(seed=12, log_ages=FULL_LOG_AGES, fehs=FULL_FEH, n_mass=300, n_bands=2)
    npix = 10.0 ** log_npix
    dmod = 25.0 + 2.5 * (log_npix - 2.0)   # Npix ~ d^2 (Eq. 1): fixed surface brightness
    p = Params(log_sfh=constant_sfr_log_sfh(_edges(FULL_LOG_AGES), npix), feh_mean=-0.5,
               feh_sigma=0.2, log_ebv=-0.5, dust_sigma=0.1 if dust else 0.0, dmod=dmod)
    flags = (FLAG_DUST if dust else 0) | (FLAG_NOISE if noise else 0)
    return Workload("full", iso, 2, n_im, [p], [n_im],
                    psf=(subpixel_psf_grid(25, (2.0, 1.8)) if psf_grid else moffat_psf(25, (2.0, 1.8)))
                    if psf else None,
                    sky=(sky, sky, 0.0, 0.0), hess_c_lo=-1.0, hess_m_lo=21.5, seed=seed,
                    flags=flags)


def batch(seed: int = 3, n_sets: int = 512, n_min: int = 128, n_max: int = 512,
          step: int = 16) -> Workload:
    """Sampler live points: uniform over log Npix [1, 6], dmod [22, 26], log E(B-V) [-1, 0]
    (fixed dust screen E1, F_dust 0.5) on the tiny isochrone, uneven image sizes."""
    rng = np.random.default_rng(seed)
    base = tiny()
    sizes = rng.integers(0, (n_max - n_min) // step + 1, size=n_sets) * step + n_min
    params = []
    for _ in range(n_sets):
        params.append(Params(log_sfh=np.array([rng.uniform(1.0, 6.0)]), feh_mean=-0.5,
                             feh_sigma=0.0, log_ebv=rng.uniform(-1.0, 0.0), dust_sigma=0.0,
                             dmod=rng.uniform(22.0, 26.0)))
    return Workload("batch", base.iso, 2, int(sizes.max()), params, [int(s) for s in sizes],
                    psf=None, hess_c_lo=-0.8, hess_m_lo=16.1, seed=seed, flags=FLAG_DUST,
                    ll_mode=LL_POISSON)


def batch_mock_params() -> Params:
    """Prior centre of the batch workload; its 256x256 simulation is the mock."""
    return Params(log_sfh=np.array([3.5]), feh_mean=-0.5, feh_sigma=0.0, log_ebv=-0.5,
                  dust_sigma=0.0, dmod=24.0)


LARGE_LOG_AGES = (6.6, 7.0, 7.4, 7.8, 8.2, 8.6, 9.0, 9.4, 9.8, 10.1)
LARGE_FEH = (-0.9, -0.8, -0.7, -0.6, -0.5, -0.4, -0.3, -0.2, -0.1)


def large(seed: int = 4, n_im: int = 1024, log_npix: float = 5.0) -> Workload:
    iso = make_isochrones(seed=14, log_ages=LARGE_LOG_AGES, fehs=LARGE_FEH, n_mass=400,
                          n_bands=3)
    npix = 10.0 ** log_npix
    dmod = 25.0 + 2.5 * (log_npix - 2.0)
    p = Params(log_sfh=constant_sfr_log_sfh(_edges(LARGE_LOG_AGES), npix), feh_mean=-0.5,
               feh_sigma=0.3, log_ebv=-0.5, dust_sigma=0.1, dmod=dmod)
    return Workload("large", iso, 3, n_im, [p], [n_im], psf=moffat_psf(25, (2.0, 1.8, 2.2), n_bands=3),
                    hess_c_lo=-1.0, hess_m_lo=21.5, seed=seed,
                    flags=FLAG_DUST | FLAG_NOISE | FLAG_KAHAN)


SURROGATE_BOX = np.array(
    # 7 log SFH (+-0.5 dex around constant SFR at Npix=100), feh mean, feh sigma,
    # log E(B-V), dust sigma, dmod
    [[-0.5, 0.5]] * 7 + [[-0.7, -0.3], [0.1, 0.3], [-1.0, 0.0], [0.05, 0.3], [24.5, 25.5]])


def surrogate(seed: int = 5, n_sets: int = 512, n_im: int = 64, draw_seed: int = 0) -> Workload:
    """The full physics at 64x64; parameters uniform over SURROGATE_BOX (the SFH rows are
    offsets from a constant-SFR history with Npix = 100)."""
    base = full(log_npix=2.0)
    rng = np.random.default_rng(1000 + draw_seed)
    u = rng.uniform(size=(n_sets, 12))
    theta = SURROGATE_BOX[:, 0] + u * (SURROGATE_BOX[:, 1] - SURROGATE_BOX[:, 0])
    return surrogate_from_theta(theta, seed=seed, n_im=n_im, base=base)


def surrogate_from_theta(theta: np.ndarray, seed: int = 5, n_im: int = 64,
                         base: Optional[Workload] = None) -> Workload:
    base = base or full(log_npix=2.0)
    sfh0 = base.params[0].log_sfh
    params = [Params(log_sfh=sfh0 + t[:7], feh_mean=float(t[7]), feh_sigma=float(t[8]),
                     log_ebv=float(t[9]), dust_sigma=float(t[10]), dmod=float(t[11]))
              for t in np.atleast_2d(theta)]
    return dataclasses.replace(base, name="surrogate", params=params,
                               n_ims=[n_im] * len(params), n_im=n_im, seed=seed)


def with_params(w: Workload, params: List[Params], n_ims: Optional[List[int]] = None) -> Workload:
    n_ims = n_ims if n_ims is not None else [w.n_im] * len(params)
    return dataclasses.replace(w, params=params, n_ims=n_ims, n_im=max(n_ims))
