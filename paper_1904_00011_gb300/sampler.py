"""A minimal nested sampler (Skilling 2004) over a box prior, with an optional surrogate
pre-screen.

Section 2.5 fits pCMDs with nested sampling; each replacement of the worst live point needs a
new prior draw whose likelihood exceeds the current threshold L_min, and with plain rejection
from the prior every trial costs one exact simulation.  With a surrogate, prior draws are first
scored by the network and only those whose surrogate likelihood exceeds L_min - margin go to the
exact simulator, in the order they were drawn; the exact simulator alone decides acceptance, so
the replacement is still the first draw with L > L_min among the draws the filter keeps (a
uniform draw from the constrained prior when the margin covers the surrogate's error).  The
statistic reported is the number of exact likelihood calls per accepted replacement.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class RunStats:
    iterations: int
    exact_calls: int
    surrogate_calls: int
    log_evidence: float
    l_min_final: float
    dead_theta: Optional[np.ndarray] = None     # [iterations][d] replaced (dead) points
    dead_log_l: Optional[np.ndarray] = None     # their log-likelihoods
    dead_log_x: Optional[np.ndarray] = None     # log prior volume at each death

    @property
    def exact_calls_per_replacement(self) -> float:
        return self.exact_calls / max(1, self.iterations)


def nested_sampling(exact_ll: Callable[[np.ndarray], np.ndarray],
                    prior_draw: Callable[[int, np.random.Generator], np.ndarray],
                    n_live: int, n_iter: int, seed: int,
                    surrogate_ll: Optional[Callable[[np.ndarray], np.ndarray]] = None,
                    margin: float = 0.0, batch: int = 1024, max_exact: int = 200000) -> RunStats:
    """Run n_iter replacements.  exact_ll maps rows of parameters to log-likelihoods (one exact
    simulation per row) and is called one row at a time during replacements; surrogate_ll scores
    whole batches of prior draws."""
    rng = np.random.default_rng(seed)
    live = prior_draw(n_live, rng)
    live_ll = exact_ll(live)
    calls = 0
    s_calls = 0
    log_z = -np.inf
    log_x = 0.0
    it = 0
    d_theta, d_ll, d_lx = [], [], []
    for it in range(n_iter):
        worst = int(np.argmin(live_ll))
        l_min = float(live_ll[worst])
        log_w = log_x + np.log1p(-np.exp(-1.0 / n_live))
        log_z = np.logaddexp(log_z, log_w + l_min)
        d_theta.append(np.array(live[worst]))
        d_ll.append(l_min)
        d_lx.append(log_x)
        log_x -= 1.0 / n_live
        new = None
        while new is None and calls < max_exact:
            pool = prior_draw(batch if surrogate_ll is not None else 64, rng)
            if surrogate_ll is not None:
                s = surrogate_ll(pool)
                s_calls += len(pool)
                pool = pool[s > l_min - margin]
            for row in pool:
                ll = float(exact_ll(row[None, :])[0])
                calls += 1
                if ll > l_min:
                    new = (row, ll)
                    break
                if calls >= max_exact:
                    break
        if new is None:
            break
        live[worst], live_ll[worst] = new
    return RunStats(it + 1, calls, s_calls, float(log_z), float(np.min(live_ll)),
                    np.array(d_theta), np.array(d_ll), np.array(d_lx))


def lmax_from_repeats(log_l_repeats: Sequence[float]) -> float:
    """Appendix A: the ceiling is the median of the best fit's recomputed log-likelihoods."""
    return float(np.median(np.asarray(log_l_repeats, np.float64)))


def capped_weights(dead_log_l: np.ndarray, dead_log_x: np.ndarray, n_live: int, l_max: float):
    """Recompute the nested-sampling weights with every log-likelihood capped at l_max: dead point
    i (at log prior volume log X_i) gets log w_i = log(X_i - X_{i+1}) + min(L_i, L_max), with
    X_{i+1} = X_i e^{-1/n_live}.  Returns (normalised posterior weights, log evidence)."""
    ll = np.minimum(np.asarray(dead_log_l, np.float64), l_max)
    log_dx = np.asarray(dead_log_x, np.float64) + np.log1p(-np.exp(-1.0 / n_live))
    log_w = log_dx + ll
    log_z = float(np.logaddexp.reduce(log_w)) if log_w.size else -np.inf
    return np.exp(log_w - log_z), log_z
