"""The total-count (pool) sampler of the oracle (the Poisson additivity of the Section 2.1
footnote, used in reverse as the splitting property): per pixel and half the
points below lambda 640 get N ~ Poisson(sum lambda) stars assigned by their weights.  Pins: the
per-point counts are independent Poisson(lambda_i) (means, variances, zero fractions, pairwise
covariances, a joint chi-square), the total is Poisson, the image mean equals the per-point
sampler's (CPU)."""
import dataclasses
import math

import numpy as np
from scipy import stats

import oracle as O
from paper_1904_00011_gb300 import workloads as W


def _two_point_w(masses, n_im=128):
    m = np.asarray(masses, np.float64)
    k = m.size
    mags = np.stack([10.0 - 2.0 * np.log10(m), 10.3 - 2.0 * np.log10(m)], axis=-1)
    iso = W.Isochrones(np.array([10.0]), np.array([-0.5]), m.reshape(1, 1, k), mags.reshape(1, 1, k, 2))
    p = W.Params(log_sfh=np.array([math.log10(1.2)]), feh_mean=-0.5, feh_sigma=0.0, log_ebv=-1.0,
                 dust_sigma=0.0, dmod=25.0)
    return W.Workload("pool", iso, 2, n_im, [p], [n_im], psf=None, hess_c_lo=-1.0,
                      hess_m_lo=21.0, seed=11, flags=W.FLAG_POOL)


def test_pool_counts_are_independent_poisson():
    w = W.tiny(npix=20.0)
    w = dataclasses.replace(w, flags=W.FLAG_POOL, n_im=96, n_ims=[96])
    lam_h, _, _ = O.tables(w)
    _, cnt = O.simulate(w, 0, 3, counts=True, n_im=96, n_threads=8)
    c = cnt[:, 0, :].astype(np.float64)            # half 0 (no dust: all stars in half 0)
    lam = lam_h[0].astype(np.float64)
    n = c.shape[0]
    se = np.sqrt(lam / n)
    assert np.all(np.abs(c.mean(axis=0) - lam) < 5 * se + 1e-9)
    top = np.argsort(lam)[-5:]                     # the best-measured points
    for i in top:
        assert abs(c[:, i].var() / lam[i] - 1.0) < 0.15
        assert abs((c[:, i] == 0).mean() - math.exp(-lam[i])) < 5 * math.sqrt(math.exp(-lam[i]) / n) + 1e-3
    cov = np.cov(c[:, top].T)
    norm = np.sqrt(np.outer(lam[top], lam[top]))
    off = (cov / norm)[~np.eye(5, dtype=bool)]
    assert np.abs(off).max() < 0.1                 # independent
    tot = c.sum(axis=1)
    assert abs(tot.mean() - lam.sum()) < 5 * math.sqrt(lam.sum() / n)
    assert abs(tot.var() / lam.sum() - 1.0) < 0.1  # the total is Poisson


def test_two_point_pool_joint_distribution():
    """Two points: per pixel (n0, n1) ~ Poisson(l0) x Poisson(l1) jointly; chi-square on the
    joint table over 16 384 pixels."""
    w = _two_point_w([0.6, 1.4])
    lam_h, _, _ = O.tables(w)
    l0, l1 = float(lam_h[0][0]), float(lam_h[0][1])
    _, cnt = O.simulate(w, 0, 5, counts=True, n_threads=8)
    n0, n1 = cnt[:, 0, 0].astype(int), cnt[:, 0, 1].astype(int)
    kmax = 4
    obs = np.zeros((kmax + 1, kmax + 1))
    for a, b in zip(np.minimum(n0, kmax), np.minimum(n1, kmax)):
        obs[a, b] += 1
    pa = np.append(stats.poisson.pmf(np.arange(kmax), l0), stats.poisson.sf(kmax - 1, l0))
    pb = np.append(stats.poisson.pmf(np.arange(kmax), l1), stats.poisson.sf(kmax - 1, l1))
    exp = np.outer(pa, pb) * n0.size
    keep = exp > 5
    chi = ((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    assert stats.chi2.sf(chi, keep.sum() - 1) > 1e-4


def test_pool_image_mean_matches_the_per_point_sampler():
    w = W.full(n_im=48, psf=False)
    wp = dataclasses.replace(w, flags=w.flags | W.FLAG_POOL)
    a = O.simulate(w, 0, 2, n_threads=8)
    b = O.simulate(wp, 0, 2, n_threads=8)
    for band in range(2):
        ma, mb = a[band].mean(), b[band].mean()
        sd = math.sqrt(0.5 * (a[band].var() + b[band].var()) / a.shape[1])
        assert abs(ma - mb) < 5 * math.sqrt(2) * sd


def test_pool_without_pool_points_draws_nothing_from_it():
    """Points at or above lambda 640 (transformed rejection) keep their own draws in pool mode:
    their counts equal the per-point sampler's; the points below differ by construction."""
    w = W.large(log_npix=6.5, n_im=4)
    wp = dataclasses.replace(w, flags=w.flags | W.FLAG_POOL)
    lam_h, _, _ = O.tables(w)
    big = lam_h >= 640
    assert big.any() and np.any((lam_h > 0) & (lam_h < 640))
    _, ca = O.simulate(w, 0, 1, counts=True, pix_end=4, n_threads=8)
    _, cb = O.simulate(wp, 0, 1, counts=True, pix_end=4, n_threads=8)
    for h in range(2):
        assert np.array_equal(ca[:, h, big[h]], cb[:, h, big[h]])


def test_pool_tables_assign_stars_in_proportion_to_lambda():
    """Star-assignment thresholds: entry j takes the words in [T_{j-1}, T_j), so its probability
    (T_j - T_{j-1}) / 2^32 is lambda_j / sum(lambda) up to the 2^-32 grid and the 2^-40 weights;
    the pool is exactly the points with 0 < lambda < 640 (and lambda >= 2^-40), in point order."""
    rng = np.random.default_rng(5)
    lam = np.concatenate([rng.gamma(0.3, 0.5, 3000), [0.0, 70.0, 640.0, 639.99, 192.0, 700.0, 12.0, 1e-13, 3e-12],
                          10.0 ** rng.uniform(-9, 0.9, 2000)]).astype(np.float32)
    rng.shuffle(lam)
    idx, thr, tot = O.pool_tables(lam)
    keep = np.flatnonzero((lam > 0) & (lam < 640) & (lam.astype(np.float64) >= 2.0 ** -40))
    assert np.array_equal(idx, keep)
    l64 = lam[idx].astype(np.float64)
    assert abs(tot / l64.sum() - 1.0) < 1e-6
    prev = np.concatenate([[0], thr[:-1].astype(np.int64)])
    p = (thr.astype(np.int64) - prev) / 2.0 ** 32
    p[-1] = 1.0 - prev[-1] / 2.0 ** 32                 # the last entry takes the rest
    assert np.all(np.diff(thr[:-1].astype(np.int64)) >= 0)
    assert np.all(np.abs(p - l64 / l64.sum()) <= 2.0 ** -31)


def test_pool_tables_small_cases_are_exact():
    """lambda = (1, 3): T_0 = 2^32 / 4 exactly; one entry: it takes every star; nothing below
    2^-40 or at 640: an empty pool."""
    idx, thr, tot = O.pool_tables(np.array([1.0, 3.0], np.float32))
    assert list(idx) == [0, 1] and int(thr[0]) == 2 ** 30 and int(thr[1]) == 2 ** 32 - 1 and tot == 4.0
    idx, thr, tot = O.pool_tables(np.array([0.0, 0.25, 700.0], np.float32))
    assert list(idx) == [1] and tot == 0.25
    idx, thr, tot = O.pool_tables(np.array([1e-13, 640.0, 0.0], np.float32))
    assert idx.size == 0


def test_pool_counts_of_both_dust_halves_have_their_own_poisson_means():
    """Full model with the dust screen (F_dust = 0.5): each half's pool gets N ~ Poisson(its
    Lambda); per point the counts of half h average lambda_h,i and the per-pixel totals of
    each half have Poisson mean and variance."""
    w = dataclasses.replace(W.full(n_im=64, psf=False), flags=W.full().flags | W.FLAG_POOL)
    lam_h, _, _ = O.tables(w)
    n_pix = 1500
    _, cnt = O.simulate(w, 0, 9, counts=True, pix_end=n_pix, n_threads=8)
    for h in range(2):
        lam = lam_h[h].astype(np.float64)
        pool = (lam > 0) & (lam < 64)
        c = cnt[:, h, :].astype(np.float64)
        top = np.argsort(np.where(pool, lam, 0.0))[-8:]
        se = np.sqrt(lam[top] / n_pix)
        assert np.all(np.abs(c[:, top].mean(axis=0) - lam[top]) < 5 * se)
        tot = c[:, pool].sum(axis=1)
        lt = lam[pool].sum()
        assert abs(tot.mean() - lt) < 5 * math.sqrt(lt / n_pix)
        assert abs(tot.var() / lt - 1.0) < 0.15
