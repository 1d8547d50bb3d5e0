"""Appendix A post-processing: the L_max ceiling (median of the best fit's recomputed
likelihoods) and the nested-sampling weights recomputed with capped likelihoods (CPU)."""
import math

import numpy as np

from paper_1904_00011_gb300 import sampler as S


def _prior(k, rng):
    return rng.uniform(-3.0, 3.0, size=(k, 2))


def test_uncapped_weights_reproduce_the_run_and_sum_to_one():
    r = S.nested_sampling(lambda t: -np.sum(t ** 2, axis=1), _prior, n_live=32, n_iter=300, seed=1)
    w, log_z = S.capped_weights(r.dead_log_l, r.dead_log_x, 32, np.inf)
    assert abs(log_z - r.log_evidence) < 1e-12
    assert abs(w.sum() - 1.0) < 1e-12
    # the dead points' volumes shrink by e^{-1/n_live} per iteration
    assert np.allclose(np.diff(r.dead_log_x), -1.0 / 32)


def test_evidence_converges_to_the_closed_form():
    """Z = (1/36) int exp(-|t|^2) over [-3,3]^2 = pi erf(3)^2 / 36; the dead points plus the live
    remainder approach it (dead points alone at 1500 iterations leave < 1 % of the mass)."""
    r = S.nested_sampling(lambda t: -np.sum(t ** 2, axis=1), _prior, n_live=64, n_iter=1500, seed=2)
    exact = math.log(math.pi * math.erf(3.0) ** 2 / 36.0)
    assert abs(r.log_evidence - exact) < 0.35


def test_capping_moves_weight_off_the_fluctuations():
    rng = np.random.default_rng(5)

    def noisy(t):   # a stochastic likelihood: the truth plus a fluctuation per call
        return -np.sum(t ** 2, axis=1) + rng.normal(0.0, 0.5, size=len(t))

    r = S.nested_sampling(noisy, _prior, n_live=32, n_iter=400, seed=3)
    best = r.dead_theta[np.argmax(r.dead_log_l)]
    l_max = S.lmax_from_repeats(noisy(np.repeat(best[None, :], 100, axis=0)))
    assert l_max < r.dead_log_l.max()                 # the best point was a positive fluctuation
    w0, z0 = S.capped_weights(r.dead_log_l, r.dead_log_x, 32, np.inf)
    w1, z1 = S.capped_weights(r.dead_log_l, r.dead_log_x, 32, l_max)
    assert z1 <= z0
    capped = r.dead_log_l >= l_max
    assert capped.sum() >= 1
    # capped points weigh by prior volume alone: ratios of their weights = ratios of dX
    i = np.nonzero(capped)[0]
    if len(i) >= 2:
        assert np.isclose(w1[i[1]] / w1[i[0]], math.exp(r.dead_log_x[i[1]] - r.dead_log_x[i[0]]))
    # the posterior mass on the capped points shrinks (their unnormalised weights fell, the
    # others' did not)
    assert w1[capped].sum() < w0[capped].sum()


def test_lmax_is_the_median():
    assert S.lmax_from_repeats([3.0, 1.0, 2.0]) == 2.0
    assert S.lmax_from_repeats([4.0, 1.0, 2.0, 3.0]) == 2.5
