"""Pins of the oracle's forward model (weights, fluxes, simulation, dust, PSF, noise,
magnitudes, Hess, likelihood) to closed forms, quadrature, FFT, brute-force enumeration and
hand-computed values (CPU only)."""
import dataclasses
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O
from paper_1904_00011_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _iso(masses, mags, log_age=10.0, feh=-0.5):
    m = np.asarray(masses, np.float64).reshape(1, 1, -1)
    a = np.asarray(mags, np.float64).reshape(1, 1, m.shape[2], -1)
    return W.Isochrones(np.array([log_age]), np.array([feh]), m, a)


def _wl(iso, npix, n_im=64, **kw):
    p = W.Params(log_sfh=np.array([math.log10(npix)]), feh_mean=-0.5, feh_sigma=0.0,
                 log_ebv=kw.pop("log_ebv", -1.0), dust_sigma=kw.pop("dust_sigma", 0.0),
                 dmod=kw.pop("dmod", 25.0))
    base = dict(name="t", iso=iso, n_bands=iso.abs_mag.shape[-1], n_im=n_im, params=[p],
                n_ims=[n_im], psf=None, hess_c_lo=-1.0, hess_m_lo=21.0, seed=kw.pop("seed", 5))
    base.update(kw)
    return W.Workload(**base)


# ------------------------------------------------------------------------------- weights

def test_weights_sum_to_npix_and_imf_cells_match_quadrature():
    w = W.full(log_npix=3.0)
    lam = O.weights(w, w.params[0])
    assert abs(lam.sum() - 1000.0) < 1e-9
    # IMF: ratio of two points of one isochrone = ratio of integrals of m^-2.35 over cells
    m = w.iso.mass[3, 2]
    e = np.sqrt(m[1:] * m[:-1])
    lo = np.concatenate([[m[0] ** 2 / e[0]], e])
    hi = np.concatenate([e, [m[-1] ** 2 / e[-1]]])
    q = np.array([integrate.quad(lambda x: x ** -2.35, a, b, epsabs=0, epsrel=1e-12)[0]
                  for a, b in zip(lo, hi)])
    got = lam[3, 2] / lam[3, 2].sum()
    assert np.allclose(got, q / q.sum(), rtol=1e-9, atol=0)
    # SFH: age-bin totals equal 10^log_sfh
    assert np.allclose(lam.sum(axis=(1, 2)), 10.0 ** w.params[0].log_sfh, rtol=1e-12)


def test_mdf_gaussian_weights_and_cut():
    w = W.full()
    p = dataclasses.replace(w.params[0], feh_mean=-0.45, feh_sigma=0.12)
    lam = O.weights(w, p)
    per_feh = lam.sum(axis=(0, 2)) / lam.sum()
    g = stats.norm.pdf(np.asarray(W.FULL_FEH), -0.45, 0.12)
    g = g / g.sum()
    keep = g >= 0.01
    ref = np.where(keep, g, 0.0)
    ref = ref / ref.sum()
    assert keep.sum() < len(g)          # the cut removes something here
    assert np.allclose(per_feh, ref, rtol=1e-12, atol=1e-15)
    # zero width -> M1: every star in one slot (grid -0.4, holding the isochrone at -0.33)
    p0 = dataclasses.replace(w.params[0], feh_mean=-0.33, feh_sigma=0.0)
    per0 = O.weights(w, p0).sum(axis=(0, 2))
    assert per0[4] == pytest.approx(per0.sum()) and np.count_nonzero(per0) == 1


def test_flux_zero_point_closed_form():
    w = _wl(_iso([1.0], [[25.94 - 25.0, 26.05 - 25.0]]), 10.0)
    f = O.fluxes(w, w.params[0])
    # a star at apparent magnitude = ZP gives exactly t_exp electrons
    assert f[0, 0] == pytest.approx(3235.0, rel=1e-13)
    assert f[0, 1] == pytest.approx(3620.0, rel=1e-13)
    f2 = O.fluxes(w, dataclasses.replace(w.params[0], dmod=27.5))
    assert f2[0, 0] / f[0, 0] == pytest.approx(10 ** (-1.0), rel=1e-13)


def test_halves_split_lambda_by_dust_fraction():
    w = W.full()
    lam = O.weights(w, w.params[0])
    h = O.halves(w, lam)
    flat = lam.reshape(-1)
    assert np.array_equal(h[0], (flat * 0.5).astype(np.float32))
    assert np.array_equal(h[1], (flat * 0.5).astype(np.float32))
    w1 = dataclasses.replace(w, f_dust=1.0)
    h1 = O.halves(w1, lam)
    assert not h1[0].any() and np.array_equal(h1[1], flat.astype(np.float32))
    w0 = dataclasses.replace(w, flags=0)
    h0 = O.halves(w0, lam)
    assert not h0[1].any()


# ------------------------------------------------------------------------------- simulation

def test_one_point_isochrone_brute_force():
    """One isochrone point: each pixel holds n ~ Poisson(Npix) stars of one flux, so the
    pixel flux is exactly n f; the empirical law of n matches the Poisson pmf."""
    w = _wl(_iso([1.0], [[4.0, 5.0]]), 3.0, n_im=128)
    img, cnt = O.simulate(w, counts=True)
    f = O.fluxes(w, w.params[0])[0]
    n = cnt[:, 0, 0].astype(np.int64)
    assert np.array_equal(img[0], n * f[0]) and np.array_equal(img[1], n * f[1])
    ks = np.arange(0, 12)
    obs = np.bincount(n, minlength=12)[:12]
    exp_ = stats.poisson.pmf(ks, 3.0) * n.size
    sel = exp_ > 5
    chi2 = (((obs - exp_) ** 2) / exp_)[sel].sum()
    assert stats.chi2.sf(chi2, sel.sum() - 1) > 1e-4


def test_two_point_enumeration_of_pixel_fluxes():
    """Two points: enumerate (n1, n2), the exact probabilities of every pixel-flux value,
    and compare with the simulated frequencies (chi-square)."""
    masses = [0.5, 1.5]
    w = _wl(_iso(masses, [[6.0, 7.0], [3.0, 3.4]]), 1.3, n_im=256, seed=9)
    # independent IMF split of Npix by quadrature over the geometric-midpoint cells
    e1 = math.sqrt(masses[0] * masses[1])
    cells = [(masses[0] ** 2 / e1, e1), (e1, masses[1] ** 2 / e1)]
    q = [integrate.quad(lambda x: x ** -2.35, a, b)[0] for a, b in cells]
    lam = [1.3 * qi / sum(q) for qi in q]
    f = O.fluxes(w, w.params[0])
    img = O.simulate(w)
    vals = {}
    for n1 in range(12):
        for n2 in range(8):
            key = round(n1 * f[0, 0] + n2 * f[1, 0], 6)
            vals[key] = vals.get(key, 0.0) + stats.poisson.pmf(n1, lam[0]) * stats.poisson.pmf(n2, lam[1])
    got = {}
    for v in np.round(img[0], 6):
        got[v] = got.get(v, 0) + 1
    assert set(got) <= set(vals)
    keys = [k for k in vals if vals[k] * img.shape[1] > 5]
    obs = np.array([got.get(k, 0) for k in keys], float)
    exp_ = np.array([vals[k] for k in keys]) * img.shape[1]
    chi2 = ((obs - exp_) ** 2 / exp_).sum()
    assert stats.chi2.sf(chi2, len(keys) - 1) > 1e-4


def test_total_star_count_is_poisson_npix():
    """Sum of Poisson counts over all points of a pixel is Poisson(Npix) (Section 2.1 footnote)."""
    w = W.tiny()
    _, cnt = O.simulate(w, counts=True)
    tot = cnt.sum(axis=(1, 2)).astype(np.int64)
    lam = 100.0
    assert abs(tot.mean() - lam) < 4 * math.sqrt(lam / tot.size)
    assert abs(tot.var() - lam) < 4 * lam * math.sqrt(2.0 / tot.size) + 1.0
    ks = np.arange(60, 141)
    obs = np.histogram(tot, bins=np.concatenate([[-0.5], ks[1:] - 0.5, [1e9]]))[0]
    cdf = stats.poisson.cdf(ks, lam)
    exp_ = np.diff(np.concatenate([[0.0], cdf[:-1], [1.0]])) * tot.size
    sel = exp_ > 5
    chi2 = ((obs - exp_) ** 2 / exp_)[sel].sum()
    assert stats.chi2.sf(chi2, sel.sum() - 1) > 1e-4


def test_compound_poisson_flux_moments():
    """E[F_b] = sum_i lambda_i f_ib, Var[F_b] = sum_i lambda_i f_ib^2 (no dust, PSF, noise)."""
    w = W.tiny(n_im=128)
    lam_h, flux, lam = O.tables(w)
    img = O.simulate(w)
    lam64 = lam_h[0].astype(np.float64)
    for b in range(2):
        mu = (lam64 * flux[:, b]).sum()
        var = (lam64 * flux[:, b] ** 2).sum()
        m4 = (lam64 * flux[:, b] ** 4).sum() + 3 * var ** 2
        n = img.shape[1]
        assert abs(img[b].mean() - mu) < 4.5 * math.sqrt(var / n)
        assert abs(img[b].var() - var) < 4.5 * math.sqrt((m4 - var ** 2) / n)


def test_dust_screen_factor_moments():
    """E1 fixed screen: the behind half is dimmed by exactly 10^(-0.4 R_b E(B-V)); E2 log-normal:
    E[factor] equals its Gaussian-quadrature expectation."""
    iso = _iso([1.0], [[4.0, 5.0]])
    wf = _wl(iso, 2.0, n_im=128, flags=W.FLAG_DUST, f_dust=1.0, log_ebv=-0.5)
    img, cnt = O.simulate(wf, counts=True)
    f = O.fluxes(wf, wf.params[0])[0]
    fac = [10 ** (-0.4 * W.R_EXT[b] * 10 ** -0.5) for b in range(2)]
    n = cnt[:, 1, 0].astype(np.float64)
    for b in range(2):
        assert np.allclose(img[b], n * f[b] * fac[b], rtol=1e-13, atol=0)
    # log-normal screen, all stars behind: E[F_b] = Npix f_b E[factor_b]
    sig = 0.4
    wl = _wl(iso, 2.0, n_im=256, flags=W.FLAG_DUST, f_dust=1.0, log_ebv=-0.3, dust_sigma=sig)
    img2, cnt2 = O.simulate(wl, counts=True)
    n2 = cnt2[:, 1, 0].astype(np.float64)
    for b in range(2):
        ratio = img2[b][n2 > 0] / (n2[n2 > 0] * f[b])
        ef = integrate.quad(lambda z: stats.norm.pdf(z) *
                            10 ** (-0.4 * W.R_EXT[b] * 10 ** -0.3 * math.exp(sig * z)), -9, 9)[0]
        ef2 = integrate.quad(lambda z: stats.norm.pdf(z) *
                             10 ** (-0.8 * W.R_EXT[b] * 10 ** -0.3 * math.exp(sig * z)), -9, 9)[0]
        assert abs(ratio.mean() - ef) < 4.5 * math.sqrt((ef2 - ef * ef) / ratio.size)


def test_integrated_light_limit():
    """At large Npix pixel colours converge on the integrated-light colour and the spread
    shrinks like Npix^-1/2."""
    spreads = []
    for npix in (1e4, 1e6):
        w = W.tiny(n_im=24, npix=npix)
        lam_h, flux, lam = O.tables(w)
        r = O.model(w)
        col = r["colour"][r["valid"] > 0].astype(np.float64)
        L = (lam.reshape(-1)[:, None] * flux).sum(axis=0)
        m_int = [W.ZEROPOINT[b] - 2.5 * math.log10(L[b] / W.EXPTIME[b]) for b in range(2)]
        c_int = m_int[1] - m_int[0]
        spreads.append(col.std())
        if npix == 1e6:
            assert abs(np.median(col) - c_int) < 0.01
    assert 5.0 < spreads[0] / spreads[1] < 20.0


# ------------------------------------------------------------------------------- PSF / noise / mags

def test_psf_is_circular_convolution():
    rng = np.random.default_rng(3)
    n = 40
    img = rng.exponential(size=(1, n * n))
    k = rng.uniform(size=(1, 7, 7)).astype(np.float32)  # deliberately asymmetric
    got = O.psf(img, k, n)[0].reshape(n, n)
    kk = np.zeros((n, n))
    R = 3
    for u in range(7):
        for v in range(7):
            kk[(u - R) % n, (v - R) % n] = k[0, u, v]
    ref = np.real(np.fft.ifft2(np.fft.fft2(img[0].reshape(n, n)) * np.fft.fft2(kk)))
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-10)


def test_noise_is_sqrt_counts_gaussian():
    w = W.tiny(n_im=128)
    w = dataclasses.replace(w, flags=W.FLAG_NOISE, sky=(50.0, 20.0, 0, 0))
    raw = O.simulate(w)
    _, _, _, fl = O.noise_mags(w, raw, 128, 0)
    for b, sky in enumerate((50.0, 20.0)):
        z = (fl[b] - raw[b]) / np.sqrt(raw[b] + sky)
        assert abs(z.mean()) < 4.5 / math.sqrt(z.size)
        assert abs(z.var() - 1.0) < 4.5 * math.sqrt(2.0 / z.size)
        assert stats.kstest(z, "norm").pvalue > 1e-4


def test_magnitudes_of_single_star_pixels():
    w = _wl(_iso([1.0], [[4.0, 5.0]]), 2.0, n_im=64)
    img, cnt = O.simulate(w, counts=True)
    mag, col, valid, _ = O.noise_mags(w, img, 64, 0)
    n = cnt[:, 0, 0]
    sel = n > 0
    assert np.array_equal(valid > 0, sel)
    ref_m = (4.0 + 25.0 - 2.5 * np.log10(n[sel])).astype(np.float32)
    assert np.allclose(mag[sel], ref_m, atol=2e-6)
    assert np.allclose(col[sel], 1.0, atol=4e-6)


def test_distance_shifts_bins_only_vertically():
    """A distance-modulus change of 10 bin widths moves every valid pixel by exactly 10 bins
    in magnitude and none in colour (Section 2.3), PSF and noise off."""
    w = W.tiny(n_im=96)
    r1 = O.model(w)
    w2 = dataclasses.replace(w, params=[dataclasses.replace(w.params[0], dmod=25.5)])
    r2 = O.model(w2)
    v = r1["valid"] > 0
    iy1 = np.floor((r1["mag"][v] - np.float32(21.0)) * np.float32(20.0))
    iy2 = np.floor((r2["mag"][v] - np.float32(21.0)) * np.float32(20.0))
    ix1 = np.floor((r1["colour"][v] - np.float32(-1.0)) * np.float32(20.0))
    ix2 = np.floor((r2["colour"][v] - np.float32(-1.0)) * np.float32(20.0))
    assert np.mean(iy2 - iy1 == 10) > 0.999
    assert np.mean(ix2 == ix1) > 0.999


def test_hess_conserves_pixels_and_bin_rule():
    w = W.full(n_im=32)
    r = O.model(w)
    assert r["hist"].sum() + r["counters"].sum() == 32 * 32
    # bin rule on hand-picked FP32 values (c_lo = -1, m_lo = 21.5, width 0.05)
    # 21.75 - 21.5 = 0.25 exactly, times 20 = 5: a lower bin edge belongs to its bin
    mag = np.float32([21.5, 21.56, 21.75, 26.5, 26.49, 21.4999, 23.0])
    col = np.float32([-1.0, -0.94, 3.99, 4.0, 0.0, 0.0, 0.0])
    valid = np.uint8([1, 1, 1, 1, 1, 1, 0])
    h, c, m = O.hess(w, mag, col, valid)
    assert h[0, 0] == 1 and h[1, 1] == 1 and h[5, 99] == 1 and h[99, 20] == 1
    assert h.sum() == 4
    assert c[0] == 2 and c[1] == 1 and m[2] == 6


# ------------------------------------------------------------------------------- likelihood

def _golden_ll():
    out = {}
    with open(os.path.join(GOLDEN, "loglike_toy.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def test_loglike_hand_computed():
    g = _golden_ll()
    d = np.array([[0, 1, 2], [3, 0, 0], [0, 0, 4]])
    m = np.array([[1, 1, 0], [2, 0, 0], [0, 1, 3]])
    md = (6.0, 120.0, 10.0)
    mm = (5.5, 121.0, 10.0)
    assert O.loglike(m, mm, 10, d, md, 12) == pytest.approx(g["paper"], rel=1e-12)
    assert O.loglike(m, mm, 10, d, md, 12, sigma_sqrtsum=True) == pytest.approx(
        g["paper_sqrtsum"], rel=1e-12)
    assert O.loglike(m, mm, 10, d, md, 12, mode=O.LL_POISSON) == pytest.approx(
        g["poisson"], rel=1e-12)
    # identical diagrams and moments: the Gaussian term and C vanish
    assert O.loglike(d, md, 12, d, md, 12) == 0.0


# ------------------------------------------------------------------- sub-pixel PSF grid

def test_psf_grid_of_identical_kernels_is_the_single_psf():
    rng = np.random.default_rng(21)
    img = rng.uniform(0, 5, size=(2, 40 * 40))
    k = W.moffat_psf(7, (2.0, 1.6))
    grid = np.repeat(k[None], 16, axis=0)
    assert np.array_equal(O.psf(img, grid, 40), O.psf(img, k, 40))


@pytest.mark.parametrize("n_im", [32, 37])
def test_psf_grid_uses_each_regions_kernel(n_im):
    """Region (4y/N, 4x/N) of the output equals the whole-image convolution with that region's
    kernel, for every region (ragged N puts uneven regions on the grid)."""
    rng = np.random.default_rng(22)
    img = rng.uniform(0, 5, size=(2, n_im * n_im))
    grid = W.subpixel_psf_grid(9, (2.0, 1.7))
    out = O.psf(img, grid, n_im).reshape(2, n_im, n_im)
    y, x = np.mgrid[0:n_im, 0:n_im]
    region = (4 * y // n_im) * 4 + (4 * x // n_im)
    for r in range(16):
        whole = O.psf(img, grid[r], n_im).reshape(2, n_im, n_im)
        m = region == r
        assert m.any()
        assert np.array_equal(out[:, m], whole[:, m])


def test_subpixel_psfs_are_shifted_moffats():
    """Kernel 4 ry + rx is centred at ((rx + 1/2)/4 - 1/2, (ry + 1/2)/4 - 1/2) pixels: its
    first moments, unit sum."""
    grid = W.subpixel_psf_grid(25, (2.0, 1.8))
    r = 12
    yy, xx = np.mgrid[-r:r + 1, -r:r + 1]
    for ry in range(4):
        for rx in range(4):
            k = grid[4 * ry + rx, 0].astype(np.float64)
            assert abs(k.sum() - 1.0) < 1e-6
            # the Moffat's wings are truncated by the grid, so the centroid is only close
            assert abs((k * xx).sum() - ((rx + 0.5) / 4 - 0.5)) < 0.05
            assert abs((k * yy).sum() - ((ry + 0.5) / 4 - 0.5)) < 0.05
