"""Pins of the oracle's RNG and Poisson sampler to published vectors, libm, scipy and exact
probabilities (CPU only)."""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = O.philox(r[0:4], r[4:6])
        assert [int(v) for v in out] == r[6:10]


def test_uniform_mapping_is_exact_and_open():
    for w in [0, 1, 255, 256, 0x7FFFFFFF, 0x80000000, 0xFFFFFF00, 0xFFFFFFFF]:
        u = O.uniform(w)
        assert 0.0 < u < 1.0
        assert u == (((w >> 8) | 1) / 2.0 ** 24)
    assert O.uniform(0) == 2.0 ** -24
    assert O.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24


def _ulp32(x):
    x = np.float32(x)
    return float(np.spacing(np.abs(x)))


def test_lnf_against_libm():
    rng = np.random.default_rng(0)
    xs = np.concatenate([
        np.float32(2.0) ** rng.uniform(-120, 120, 4000).astype(np.float32),
        rng.uniform(0.5, 2.0, 4000).astype(np.float32),
        np.float32([1.0, 2.0, 0.5, 10.0, 1e-5, 3.3e4, 1.4142135, 1.4142137, 0.70710677,
                    2.0 ** -24, 1.0 - 2.0 ** -24, 1e9, 3.4e38, 1.2e-38])])
    worst = 0.0
    for x in xs:
        ref = math.log(float(x))
        got = O.lnf(float(x))
        err = abs(got - ref) / max(_ulp32(ref), 2.0 ** -149)
        worst = max(worst, err)
    assert worst <= 2.0, worst
    assert O.lnf(1.0) == 0.0


def test_inversion_boundaries_are_the_poisson_cdf():
    """The inversion is monotone in the 32-bit word x; its k -> k+1 boundaries, found by
    bisection, must sit at 2^32 * CDF(k) of the exact Poisson law within quantisation."""
    for lam in [1e-4, 0.1, 1.0, 4.5, 9.99, 27.3, 63.9, 120.25, 191.9, 310.5, 639.9]:
        cdf = stats.poisson.cdf(np.arange(0, 1025), lam)
        kmax = int(stats.poisson.ppf(1 - 1e-9, lam))
        for k in range(0, kmax + 1):
            # smallest x with n(x) > k
            lo, hi = 0, 2 ** 32
            while lo < hi:
                mid = (lo + hi) // 2
                if O.poisson_inversion(lam, mid) > k:
                    hi = mid
                else:
                    lo = mid + 1
            frac = lo / 2.0 ** 32
            # lambda is used as its FP32 value
            ref = stats.poisson.cdf(k, float(np.float32(lam)))
            assert abs(frac - ref) <= 2.0 ** -31 + 1e-13 * k, (lam, k, frac, ref)
        assert cdf[-1] > 0.999999


def test_inversion_is_zero_iff_below_e_minus_lambda():
    lam = np.float32(0.37)
    p0 = math.exp(-float(lam))
    x0 = int(math.floor(p0 * 2 ** 32 - 0.5))
    assert O.poisson_inversion(float(lam), x0 - 1) == 0
    assert O.poisson_inversion(float(lam), x0 + 2) >= 1


@pytest.mark.parametrize("lam", [10.0, 37.5, 1000.0, 1e5])
def test_ptrs_matches_poisson_law(lam):
    n = 60000
    seed = 0x1234ABCD5678
    draws = np.array([O.poisson_ptrs(lam, seed, p, 7, 3, p & 1)[0] for p in range(n)])
    assert draws.max() < 2 ** 31
    mean, var = draws.mean(), draws.var()
    se_mean = math.sqrt(lam / n)
    assert abs(mean - lam) < 4.5 * se_mean
    se_var = lam * math.sqrt(2.0 / n)
    assert abs(var - lam) < 4.5 * se_var + 1e-3 * lam
    # chi-square over bins of >= 50 expected counts
    lo = int(stats.poisson.ppf(1e-5, lam))
    hi = int(stats.poisson.ppf(1 - 1e-5, lam))
    ks = np.arange(lo, hi + 1)
    pmf = stats.poisson.pmf(ks, lam)
    edges = [lo]
    acc = 0.0
    for k, p in zip(ks, pmf):
        acc += p
        if acc * n >= 50:
            edges.append(k + 1)
            acc = 0.0
    edges[-1] = hi + 1
    obs = np.histogram(draws, bins=np.array(edges) - 0.5)[0]
    exp_ = np.array([stats.poisson.cdf(b - 1, lam) - stats.poisson.cdf(a - 1, lam)
                     for a, b in zip(edges[:-1], edges[1:])]) * n
    chi2 = float(((obs - exp_) ** 2 / exp_).sum())
    dof = len(obs) - 1
    assert stats.chi2.sf(chi2, dof) > 1e-4, (chi2, dof)


def test_ptrs_attempts_mostly_one():
    att = [O.poisson_ptrs(500.0, 99, p, 0, 0, 0)[1] for p in range(5000)]
    assert np.mean(np.array(att) == 1) > 0.85
    assert max(att) < 20


def test_log_pmf_against_scipy():
    for lam in [10.0, 13.7, 100.0, 2500.0, 1e5, 3e6]:
        lam32 = float(np.float32(lam))
        s = math.sqrt(lam)
        ks = sorted({0, 1, 2, 5, 15, 16, 17} | {int(max(0, lam + t * s)) for t in
                                                (-8, -4, -2, -1, -0.3, 0, 0.3, 1, 2, 4, 8)})
        for k in ks:
            ref = stats.poisson.logpmf(k, lam32)
            got = O.log_pmf(float(k), lam32)
            tol = 2e-5 + 2e-6 * abs(ref)
            assert abs(got - ref) <= tol, (lam, k, got, ref)


def test_draw_switches_sampler_at_640():
    seed = 77
    # below 640: identical to inversion on the draw word; at/above: PTRS stream
    below = float(np.nextafter(np.float32(640.0), np.float32(0.0)))
    for p in range(50):
        x = O.draw_word(seed, p, 5, 1, 0)
        assert O.draw(below, seed, p, 5, 1, 0) == O.poisson_inversion(below, x)
        assert O.draw(12.0, seed, p, 5, 1, 0) == O.poisson_inversion(12.0, x)
        assert O.draw(64.0, seed, p, 5, 1, 0) == O.poisson_inversion(64.0, x)
        assert O.draw(192.0, seed, p, 5, 1, 0) == O.poisson_inversion(192.0, x)
        assert O.draw(640.0, seed, p, 5, 1, 0) == O.poisson_ptrs(640.0, seed, p, 5, 1, 0)[0]
    assert O.draw(0.0, seed, 3, 3, 3, 1) == 0


def test_inversion_cap_never_binds_below_640():
    """The largest word (v = 1 - 2^-33) stops the walk where the CDF first exceeds 1 - 2^-33,
    below the cap of 1024 for every mean under 640: the cap never truncates the law."""
    below = float(np.nextafter(np.float32(640.0), np.float32(0.0)))
    k = O.poisson_inversion(below, 0xFFFFFFFF)
    first = min(j for j in range(1200) if stats.poisson.sf(j, below) < 2.0 ** -33)
    assert k < 1024 and abs(k - first) <= 1, (k, first)
    # the smallest word: the CDF's lower tail, n0 always-exceeded thresholds and the first
    # count whose CDF reaches 2^-33
    k0 = O.poisson_inversion(below, 0)
    first0 = min(j for j in range(1200) if stats.poisson.cdf(j, below) > 2.0 ** -33)
    assert abs(k0 - first0) <= 1, (k0, first0)


@pytest.mark.parametrize("lam", [12.5, 40.0, 63.5, 150.0, 300.0, 639.5])
def test_inversion_matches_poisson_law_at_large_means(lam):
    """Draws of the inversion branch over Philox words at means between the old and new
    boundary follow the Poisson law (chi-square, mean and variance)."""
    n = 60000
    seed = 0x5EED
    draws = np.array([O.draw(lam, seed, p, 11, 2, p & 1) for p in range(n)])
    assert abs(draws.mean() - lam) < 4.5 * math.sqrt(lam / n)
    assert abs(draws.var() - lam) < 4.5 * lam * math.sqrt(2.0 / n) + 1e-3 * lam
    lo = int(stats.poisson.ppf(1e-5, lam))
    hi = int(stats.poisson.ppf(1 - 1e-5, lam))
    edges = [lo]
    acc = 0.0
    for k in range(lo, hi + 1):
        acc += stats.poisson.pmf(k, lam)
        if acc * n >= 50:
            edges.append(k + 1)
            acc = 0.0
    edges[-1] = hi + 1
    obs = np.histogram(draws, bins=np.array(edges) - 0.5)[0]
    exp_ = np.array([stats.poisson.cdf(b - 1, lam) - stats.poisson.cdf(a - 1, lam)
                     for a, b in zip(edges[:-1], edges[1:])]) * n
    chi2 = float(((obs - exp_) ** 2 / exp_).sum())
    assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-4, chi2


def test_draw_word_layout():
    """x = b << 24 | l >> 8: b byte i & 3 of word (i & 15) >> 2 of the HI call of group i >> 4,
    l word i & 3 of the LO call of quad i >> 2."""
    seed = (0xDEADBEEF << 32) | 0x01234567
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for (pix, i, s, h) in [(0, 0, 0, 0), (17, 9, 4, 1), (65535, 199, 511, 0), (3, 7, 2, 1), (8, 31, 1, 0)]:
        whi = O.philox([pix, i >> 4, s, (1 << 28) | (h << 27)], key)
        wlo = O.philox([pix, i >> 2, s, (2 << 28) | (h << 27)], key)
        b = (int(whi[(i & 15) >> 2]) >> (8 * (i & 3))) & 0xFF
        assert O.draw_word(seed, pix, i, s, h) == (b << 24) | (int(wlo[i & 3]) >> 8)


def test_draw_words_are_uniform_and_distinct_across_points():
    """Every point of a group has its own byte and its own low bits: over many pixels the words
    of the 16 points of one group are uniform (chi-square on the top 4 bits) and pairwise
    uncorrelated."""
    from scipy import stats
    seed = 12345
    W = np.array([[O.draw_word(seed, p, i, 2, 0) for i in range(16)] for p in range(4000)], np.float64)
    top = (W.astype(np.uint64) >> np.uint64(28)).astype(int)
    for i in range(16):
        cnt = np.bincount(top[:, i], minlength=16)
        assert stats.chisquare(cnt).pvalue > 1e-4
    c = np.corrcoef(W.T)
    off = c[~np.eye(16, dtype=bool)]
    assert np.abs(off).max() < 0.08