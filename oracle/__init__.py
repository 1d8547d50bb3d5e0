"""CPU oracle of the pCMD forward model -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  It shares no code with the CUDA path: the sampler, weights, fluxes, dust, PSF,
noise, magnitudes and Hess binning are in ``oracle.c`` (plain C, FP64 fluxes, the sampler's
decisions per its written specification); the likelihood (Eq. 2-4 and the Poisson mode) is
written out below in numpy FP64.  Inputs come from ``paper_1904_00011_gb300.workloads``, a
module of seeded input generators that holds no step of the method.

Parity status: every function here is pinned by ``tests/test_oracle_*.py`` against
published known-answer vectors (Philox), libm / scipy (log, Poisson pmf), exact Poisson
probabilities, brute-force enumeration, closed-form moments, FFT convolution and hand-computed
likelihoods.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

LL_PAPER = 0
LL_POISSON = 1
FLAG_DUST = 1
FLAG_NOISE = 2
FLAG_SIGMA_SQRTSUM = 8
FLAG_POOL = 16


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no FMA contraction, no fast-math; OpenMP when available)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-fno-strict-aliasing", _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            f32p = ctypes.POINTER(ctypes.c_float)
            f64p = ctypes.POINTER(ctypes.c_double)
            L.or_philox.argtypes = [u32p, u32p, u32p]
            L.or_philox.restype = None
            L.or_lnf.argtypes = [ctypes.c_float]
            L.or_lnf.restype = ctypes.c_float
            L.or_uniform.argtypes = [ctypes.c_uint32]
            L.or_uniform.restype = ctypes.c_float
            L.or_draw_word.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_uint32]
            L.or_draw_word.restype = ctypes.c_uint32
            L.or_poisson_inversion.argtypes = [ctypes.c_float, ctypes.c_uint32]
            L.or_poisson_inversion.restype = ctypes.c_uint32
            L.or_ptrs_setup.argtypes = [ctypes.c_float, f32p]
            L.or_ptrs_setup.restype = None
            L.or_poisson_ptrs.argtypes = [f32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_uint32, ctypes.c_uint32, u32p]
            L.or_poisson_ptrs.restype = ctypes.c_uint32
            L.or_log_pmf.argtypes = [ctypes.c_float, ctypes.c_float]
            L.or_log_pmf.restype = ctypes.c_float
            L.or_draw.argtypes = [ctypes.c_float, ctypes.c_uint64, ctypes.c_uint32,
                                  ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                  ctypes.POINTER(ctypes.c_int)]
            L.or_draw.restype = ctypes.c_uint32
            L.or_weights.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, f64p, ctypes.c_double, ctypes.c_int,
                                     f64p, f64p, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, f64p]
            L.or_weights.restype = None
            L.or_fluxes.argtypes = [ctypes.c_int, ctypes.c_int, f64p, ctypes.c_double, f64p, f64p,
                                    f64p]
            L.or_fluxes.restype = None
            L.or_halves.argtypes = [ctypes.c_int, f64p, ctypes.c_int, ctypes.c_double, f32p]
            L.or_halves.restype = ctypes.c_int
            L.or_simulate.argtypes = [ctypes.c_int, ctypes.c_int, f32p, f64p, ctypes.c_int,
                                      ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint64, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, f64p, f64p, u32p, ctypes.c_int,
                                      ctypes.c_int]
            L.or_simulate.restype = ctypes.c_int
            L.or_pool_tables.argtypes = [f32p, ctypes.c_int, u32p, u32p, f32p]
            L.or_pool_tables.restype = ctypes.c_int
            L.or_psf.argtypes = [ctypes.c_int, ctypes.c_int, f32p, f64p, f64p]
            L.or_psf.restype = None
            L.or_psf_grid.argtypes = L.or_psf.argtypes
            L.or_psf_grid.restype = None
            L.or_noise_mags.argtypes = [ctypes.c_int, ctypes.c_int, f64p, ctypes.c_int, f64p, f64p,
                                        f64p, ctypes.c_uint32, ctypes.c_uint64, f32p, f32p,
                                        ctypes.POINTER(ctypes.c_uint8), f64p]
            L.or_noise_mags.restype = None
            L.or_hess.argtypes = [ctypes.c_size_t, f32p, f32p, ctypes.POINTER(ctypes.c_uint8),
                                  ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, u32p, u32p, f64p]
            L.or_hess.restype = None
            _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


# ----------------------------------------------------------------------------------------
# RNG and sampler primitives
# ----------------------------------------------------------------------------------------

def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return out


def lnf(x: float) -> float:
    return float(lib().or_lnf(ctypes.c_float(x)))


def uniform(w: int) -> float:
    return float(lib().or_uniform(ctypes.c_uint32(w)))


def draw_word(seed: int, pix: int, i: int, set_id: int, half: int) -> int:
    return int(lib().or_draw_word(seed, pix, i, set_id, half))


def poisson_inversion(lam: float, x: int) -> int:
    return int(lib().or_poisson_inversion(ctypes.c_float(lam), ctypes.c_uint32(x)))


def ptrs_setup(lam: float) -> np.ndarray:
    out = np.zeros(6, np.float32)
    lib().or_ptrs_setup(ctypes.c_float(lam), _p(out, ctypes.c_float))
    return out


def poisson_ptrs(lam: float, seed: int, pix: int, i: int, set_id: int, half: int
                 ) -> Tuple[int, int]:
    c6 = ptrs_setup(lam)
    att = ctypes.c_uint32(0)
    n = lib().or_poisson_ptrs(_p(c6, ctypes.c_float), seed, pix, i, set_id, half,
                              ctypes.byref(att))
    return int(n), int(att.value)


def log_pmf(k: float, lam: float) -> float:
    return float(lib().or_log_pmf(ctypes.c_float(k), ctypes.c_float(lam)))


def draw(lam: float, seed: int, pix: int, i: int, set_id: int, half: int) -> int:
    err = ctypes.c_int(0)
    n = lib().or_draw(ctypes.c_float(lam), seed, pix, i, set_id, half, ctypes.byref(err))
    if err.value:
        raise RuntimeError("oracle sampler attempt cap reached")
    return int(n)


# ----------------------------------------------------------------------------------------
# model tables
# ----------------------------------------------------------------------------------------

def m1_bracket(feh: np.ndarray, mu: float) -> Tuple[int, float]:
    """M1, one [Fe/H] (Section 2.2: isochrones interpolated between grid metallicities): the
    grid isochrone k with feh[k] <= mu < feh[k + 1] and the fraction t of the way to k + 1;
    outside the grid, the end isochrone with t = 0."""
    feh = np.asarray(feh, np.float64)
    nf = feh.size
    if nf == 1 or mu <= feh[0]:
        return 0, 0.0
    if mu >= feh[-1]:
        return nf - 1, 0.0
    k = int(np.nonzero(feh[:-1] <= mu)[0][-1])
    return k, float((mu - feh[k]) / (feh[k + 1] - feh[k]))


def model_isochrones(w, params) -> Tuple[np.ndarray, np.ndarray, float]:
    """(mass, abs_mag, [Fe/H] selector) that the weights and fluxes of one parameter set use.
    M2/M3 (feh_sigma > 0): the grid as it is.  M1 (feh_sigma <= 0): grid slot k holds the
    isochrone at [Fe/H] = feh_mean, every mass point's initial mass and absolute magnitudes
    linearly interpolated in [Fe/H] between the same point of grid isochrones k and k + 1,
    and the selector is feh[k] (all weight on that slot)."""
    iso = w.iso
    mass = np.array(iso.mass, np.float64)
    mags = np.array(iso.abs_mag, np.float64)
    if params.feh_sigma > 0.0:
        return mass, mags, params.feh_mean
    k, t = m1_bracket(iso.feh, params.feh_mean)
    if t > 0.0:
        u = 1.0 - t
        mass[:, k] = u * iso.mass[:, k] + t * iso.mass[:, k + 1]
        mags[:, k] = u * iso.abs_mag[:, k] + t * iso.abs_mag[:, k + 1]
    return mass, mags, float(iso.feh[k])


def weights(w, params) -> np.ndarray:
    """FP64 lambda[n_ages, n_feh, n_mass] of one parameter set (sums to Npix)."""
    iso = w.iso
    na, nf, nm = iso.mass.shape
    mass, _, feh_sel = model_isochrones(w, params)
    mass = np.ascontiguousarray(mass)
    feh = np.ascontiguousarray(iso.feh, np.float64)
    sfh = np.ascontiguousarray(params.log_sfh, np.float64)
    if sfh.size != na:
        raise ValueError("one SFH value per age bin required")
    out = np.zeros((na, nf, nm))
    lib().or_weights(na, nf, nm, _p(mass, ctypes.c_double), w.imf_slope, int(getattr(w, "imf", 0)),
                     _p(feh, ctypes.c_double),
                     _p(sfh, ctypes.c_double), feh_sel, params.feh_sigma, w.mdf_cut,
                     _p(out, ctypes.c_double))
    return out


def fluxes(w, params) -> np.ndarray:
    """FP64 electrons per star [n_points, n_bands]."""
    nb = w.n_bands
    _, mags, _ = model_isochrones(w, params)
    mags = np.ascontiguousarray(mags.reshape(-1, nb), np.float64)
    zp = np.ascontiguousarray(w.zeropoint[:nb], np.float64)
    et = np.ascontiguousarray(w.exptime[:nb], np.float64)
    out = np.zeros((mags.shape[0], nb))
    lib().or_fluxes(mags.shape[0], nb, _p(mags, ctypes.c_double), params.dmod,
                    _p(zp, ctypes.c_double), _p(et, ctypes.c_double), _p(out, ctypes.c_double))
    return out


def halves(w, lam: np.ndarray) -> np.ndarray:
    lam = np.ascontiguousarray(lam.reshape(-1), np.float64)
    out = np.zeros((2, lam.size), np.float32)
    lib().or_halves(lam.size, _p(lam, ctypes.c_double), int(bool(w.flags & FLAG_DUST)), w.f_dust,
                    _p(out, ctypes.c_float))
    return out


def tables(w, set_index: int = 0):
    p = w.params[set_index]
    lam = weights(w, p)
    return halves(w, lam), fluxes(w, p), lam


# ----------------------------------------------------------------------------------------
# simulation
# ----------------------------------------------------------------------------------------

def simulate(w, set_index: int = 0, set_id: Optional[int] = None, pix_begin: int = 0,
             pix_end: Optional[int] = None, counts: bool = False, n_threads: int = 1,
             n_im: Optional[int] = None, pool: Optional[bool] = None):
    """Raw (pre-PSF) image [n_bands, N*N] FP64 for pixels [pix_begin, pix_end) and, when asked,
    the counts [pixels, 2, n_points] (uint32).  pool: the total-count sampler for the points
    below lambda 10 (default: the workload's FLAG_POOL)."""
    if pool is None:
        pool = bool(w.flags & FLAG_POOL)
    p = w.params[set_index]
    n_im = n_im if n_im is not None else w.n_ims[set_index]
    set_id = set_index if set_id is None else set_id
    lam_h, flux, _ = tables(w, set_index)
    npts = lam_h.shape[1]
    nb = w.n_bands
    npix = n_im * n_im
    pix_end = npix if pix_end is None else pix_end
    image = np.zeros((nb, npix))
    cnt = np.zeros((pix_end - pix_begin, 2, npts), np.uint32) if counts else None
    r_ext = np.ascontiguousarray(w.r_ext[:nb], np.float64)
    flux = np.ascontiguousarray(flux, np.float64)
    lam_h = np.ascontiguousarray(lam_h)
    err = lib().or_simulate(npts, nb, _p(lam_h, ctypes.c_float), _p(flux, ctypes.c_double), n_im,
                            pix_begin, pix_end, set_id, w.seed, int(bool(w.flags & FLAG_DUST)),
                            p.log_ebv, p.dust_sigma, _p(r_ext, ctypes.c_double),
                            _p(image, ctypes.c_double),
                            _p(cnt, ctypes.c_uint32) if counts else None, n_threads, int(bool(pool)))
    if err:
        raise RuntimeError("oracle sampler attempt cap reached")
    return (image, cnt) if counts else image


def pool_tables(lam: np.ndarray) -> Tuple[np.ndarray, np.ndarray, float]:
    """Total-count sampler pool of one half (FP32 lambdas): point indices, star-assignment
    thresholds T_j and the total's mean Lambda."""
    lam = np.ascontiguousarray(lam, np.float32)
    idx = np.zeros(max(lam.size, 1), np.uint32)
    thr = np.zeros(max(lam.size, 1), np.uint32)
    tot = np.zeros(1, np.float32)
    n = lib().or_pool_tables(_p(lam, ctypes.c_float), lam.size, _p(idx, ctypes.c_uint32),
                             _p(thr, ctypes.c_uint32), _p(tot, ctypes.c_float))
    return idx[:n].copy(), thr[:n].copy(), float(tot[0])


def psf(image: np.ndarray, kernel: np.ndarray, n_im: int) -> np.ndarray:
    """Periodic PSF convolution per band, FP64.  kernel [B][S][S], or [16][B][S][S] for the 4x4
    grid of sub-pixel PSFs (Section 2.2; region (4y/N, 4x/N) uses kernel 4 ry + rx)."""
    nb = image.shape[0]
    out = np.zeros_like(image)
    for b in range(nb):
        src = np.ascontiguousarray(image[b], np.float64)
        dst = np.zeros(n_im * n_im)
        if kernel.ndim == 4:
            k = np.ascontiguousarray(kernel[:, b], np.float32)
            lib().or_psf_grid(n_im, k.shape[-1], _p(k, ctypes.c_float), _p(src, ctypes.c_double),
                              _p(dst, ctypes.c_double))
        else:
            k = np.ascontiguousarray(kernel[b], np.float32)
            lib().or_psf(n_im, k.shape[0], _p(k, ctypes.c_float), _p(src, ctypes.c_double),
                         _p(dst, ctypes.c_double))
        out[b] = dst
    return out


def noise_mags(w, image: np.ndarray, n_im: int, set_id: int):
    nb = w.n_bands
    npix = n_im * n_im
    img = np.ascontiguousarray(image, np.float64)
    sky = np.ascontiguousarray(w.sky[:nb], np.float64)
    zp = np.ascontiguousarray(w.zeropoint[:nb], np.float64)
    et = np.ascontiguousarray(w.exptime[:nb], np.float64)
    mag = np.zeros(npix, np.float32)
    col = np.zeros(npix, np.float32)
    valid = np.zeros(npix, np.uint8)
    fl = np.zeros((nb, npix))
    lib().or_noise_mags(n_im, nb, _p(img, ctypes.c_double), int(bool(w.flags & FLAG_NOISE)),
                        _p(sky, ctypes.c_double), _p(zp, ctypes.c_double), _p(et, ctypes.c_double),
                        set_id, w.seed, _p(mag, ctypes.c_float), _p(col, ctypes.c_float),
                        _p(valid, ctypes.c_uint8), _p(fl, ctypes.c_double))
    return mag, col, valid, fl


def hess(w, mag: np.ndarray, colour: np.ndarray, valid: np.ndarray):
    """(hist[ny, nx] uint32, counters[2] = (overflow, invalid), moments[3] = (sum colour,
    sum mag, n_valid))."""
    mag = np.ascontiguousarray(mag, np.float32)
    colour = np.ascontiguousarray(colour, np.float32)
    valid = np.ascontiguousarray(valid, np.uint8)
    hist = np.zeros((w.hess_ny, w.hess_nx), np.uint32)
    ctr = np.zeros(2, np.uint32)
    mom = np.zeros(3)
    lib().or_hess(mag.size, _p(mag, ctypes.c_float), _p(colour, ctypes.c_float),
                  _p(valid, ctypes.c_uint8), w.hess_nx, w.hess_ny, w.hess_c_lo, w.hess_m_lo,
                  w.hess_width, _p(hist, ctypes.c_uint32), _p(ctr, ctypes.c_uint32),
                  _p(mom, ctypes.c_double))
    return hist, ctr, mom


def model(w, set_index: int = 0, set_id: Optional[int] = None, n_threads: int = 1):
    """The whole forward model of one parameter set: dict with raw image, post-PSF image,
    noisy fluxes, magnitudes, colours, valid mask, Hess and moments."""
    set_id = set_index if set_id is None else set_id
    n_im = w.n_ims[set_index]
    raw = simulate(w, set_index, set_id, n_threads=n_threads)
    conv = psf(raw, w.psf, n_im) if w.psf is not None else raw
    mag, col, valid, fl = noise_mags(w, conv, n_im, set_id)
    hist, ctr, mom = hess(w, mag, col, valid)
    return dict(raw=raw, conv=conv, flux=fl, mag=mag, colour=col, valid=valid, hist=hist,
                counters=ctr, moments=mom, n_pix=n_im * n_im)


# ----------------------------------------------------------------------------------------
# likelihood (Section 2.5, Eq. 2-4) and the Poisson alternative
# ----------------------------------------------------------------------------------------

def loglike(model_hist, model_moments, n_m, data_hist, data_moments, n_d,
            mode: int = LL_PAPER, sigma_sqrtsum: bool = False) -> float:
    """Eq. 2: sum_i -(d_i/N_d - m_i/N_m)^2 / (2 sigma_i^2) + C, Eq. 3: sigma_i =
    max(sqrt(d_i^2 + m_i^2), 2) (or max(sqrt(d_i + m_i), 2) with sigma_sqrtsum), Eq. 4:
    C = -(C_d - C_m)^2 / (2 0.05^2) - (M_d - M_m)^2 / (2 0.05^2) with C, M the mean colour
    and magnitude of the valid pixels.  N_d, N_m are the total pixel counts of the images.
    POISSON mode: sum_i d_i ln mh_i - mh_i - ln Gamma(d_i + 1), mh_i = max(m_i, 0.5) N_d/N_m."""
    d = np.asarray(data_hist, np.float64).reshape(-1)
    m = np.asarray(model_hist, np.float64).reshape(-1)
    n_d = float(n_d)
    n_m = float(n_m)
    if mode == LL_POISSON:
        mh = np.maximum(m, 0.5) * (n_d / n_m)
        lg = np.array([math.lgamma(x + 1.0) for x in d])
        return float(np.sum(d * np.log(mh) - mh - lg))
    if model_moments[2] <= 0 or data_moments[2] <= 0:
        return -math.inf
    if sigma_sqrtsum:
        sig = np.maximum(np.sqrt(d + m), 2.0)
    else:
        sig = np.maximum(np.sqrt(d * d + m * m), 2.0)
    g = -((d / n_d - m / n_m) ** 2) / (2.0 * sig * sig)
    c_d = data_moments[0] / data_moments[2]
    m_d = data_moments[1] / data_moments[2]
    c_m = model_moments[0] / model_moments[2]
    m_m = model_moments[1] / model_moments[2]
    cterm = -((c_d - c_m) ** 2) / (2 * 0.05 ** 2) - ((m_d - m_m) ** 2) / (2 * 0.05 ** 2)
    return float(np.sum(g) + cterm)


# ----------------------------------------------------------------------------------------
# parametric star-formation histories (Section 2.2, S1-S4)
# ----------------------------------------------------------------------------------------

SFH_SSP, SFH_CONSTANT, SFH_TAU, SFH_DELAYED_TAU = 1, 2, 3, 4


def sfh_bins(model: int, theta, log_age_edges) -> np.ndarray:
    """log10 stars per pixel formed in each age bin [e_j, e_j+1) (log10 years), summing to
    Npix = 10^theta[0].  Star formation starts at the oldest edge T0; a star of age a formed at
    t = T0 - a.  S1: all stars in the bin holding age 10^theta[1]; S2: constant rate; S3: rate
    exp(-t/tau); S4: rate t exp(-t/tau), tau = theta[1] Gyr.  The mass of a bin is the integral
    of the rate over its formation times, evaluated here in closed form (FP64); empty bins -30."""
    e = np.asarray(log_age_edges, np.float64)
    ages = 10.0 ** e
    t0 = ages[-1]
    n = e.size - 1
    mass = np.zeros(n)
    if model == SFH_SSP:
        j = np.nonzero((theta[1] >= e[:-1]) & (theta[1] < e[1:]))[0]
        mass[j[0]] = 1.0
    elif model == SFH_CONSTANT:
        mass = ages[1:] - ages[:-1]
    else:
        tau = theta[1] * 1e9
        early, late = t0 - ages[1:], t0 - ages[:-1]      # formation-time bounds of each bin
        if model == SFH_TAU:
            prim = lambda t: -tau * np.exp(-t / tau)                 # noqa: E731
        else:
            prim = lambda t: -tau * np.exp(-t / tau) * (t + tau)     # noqa: E731
        mass = prim(late) - prim(early)
    v = 10.0 ** theta[0] * mass / mass.sum()
    with np.errstate(divide="ignore"):
        out = np.where(v > 0, np.log10(np.where(v > 0, v, 1.0)), -30.0)
    return np.maximum(out, -30.0)
