"""Pins of the FP64 surrogate-network reference: gradients against central finite differences,
GELU against its closed-form limits, the surrogate likelihood against scipy's Poisson pmf."""
import numpy as np
import pytest

from oracle import mlp as M


def _net(seed, dims):
    rng = np.random.default_rng(seed)
    Ws = [rng.normal(0, 1 / np.sqrt(dims[l]), size=(dims[l + 1], dims[l])) for l in range(len(dims) - 1)]
    bs = [rng.normal(0, 0.1, size=dims[l + 1]) for l in range(len(dims) - 1)]
    return Ws, bs


def test_gelu_limits():
    assert M.gelu(0.0) == 0.0
    assert abs(M.gelu(8.0) - 8.0) < 1e-12 and abs(M.gelu(-8.0)) < 1e-12
    assert abs(M.gelu(1.0) - 0.8413447460685429) < 1e-15      # Phi(1)
    z = np.linspace(-4, 4, 41)
    fd = (M.gelu(z + 1e-6) - M.gelu(z - 1e-6)) / 2e-6
    assert np.allclose(M.gelu_grad(z), fd, atol=1e-8)


@pytest.mark.parametrize("poisson", [False, True])
def test_gradients_match_finite_differences(poisson):
    dims = [5, 7, 6, 4]
    Ws, bs = _net(1, dims)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(9, dims[0]))
    y = rng.poisson(2.0, size=(9, dims[-1])).astype(float) if poisson else rng.normal(size=(9, dims[-1]))
    lg = lambda W, b: M.loss_and_grads(W, b, x, y, poisson)  # noqa: E731
    loss, gW, gb = lg(Ws, bs)
    h = 1e-6
    for l in range(len(Ws)):
        for (i, j) in [(0, 0), (dims[l + 1] - 1, dims[l] - 1), (1, 2)]:
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[l][i, j] += h
            Wm[l][i, j] -= h
            fd = (lg(Wp, bs)[0] - lg(Wm, bs)[0]) / (2 * h)
            assert abs(fd - gW[l][i, j]) < 1e-7 * max(1.0, abs(fd))
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[l][0] += h
        bm[l][0] -= h
        fd = (lg(Ws, bp)[0] - lg(Ws, bm)[0]) / (2 * h)
        assert abs(fd - gb[l][0]) < 1e-7 * max(1.0, abs(fd))


def test_adam_first_step_moves_by_lr():
    w, m, v = np.ones(3), np.zeros(3), np.zeros(3)
    g = np.array([0.5, -2.0, 1e-3])
    w2, m2, v2 = M.adam(w, m, v, g, 1, 0.01)
    # with bias correction the first step is lr * sign(g) (up to eps)
    assert np.allclose(w2, w - 0.01 * np.sign(g), atol=1e-6)


@pytest.mark.parametrize("poisson", [True, False])
def test_surrogate_loglike_is_poisson_logpmf_sum(poisson):
    from scipy import stats
    rng = np.random.default_rng(5)
    y = rng.normal(0.0, 1.5, size=(3, 50))
    d = rng.poisson(2.0, size=50)
    scale, ratio = 3.0, 0.25
    got = M.surrogate_loglike(y, d, scale, ratio, poisson)
    rate = np.exp(y) if poisson else np.expm1(y)
    mh = np.maximum(rate * scale, 0.5) * ratio
    ref = stats.poisson.logpmf(d[None, :], mh).sum(axis=1)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-9)
    # the floor: a rate far below 1/2 contributes as 1/2
    low = M.surrogate_loglike(np.full((1, 50), -30.0), d, 1.0, 1.0, True)
    assert np.isclose(low[0], stats.poisson.logpmf(d, 0.5).sum())
