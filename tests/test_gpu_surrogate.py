"""The learned surrogate on the exact simulator's own output: it must beat the prior-mean
predictor on held-out parameters, rank likelihoods like the simulator, and cut the exact
simulations a nested sampler spends per accepted replacement."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_00011_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def trained():
    from paper_1904_00011_gb300.surrogate import Surrogate
    S = Surrogate(batch=512, seed=0)
    info = S.train(n_sims=512 * 96)
    return S, info


def _mock(S):
    theta0 = S.box.mean(axis=1).astype(np.float32)
    return S.exact_mock(theta0)


def test_surrogate_beats_prior_mean_and_ranks_likelihoods(trained):
    S, info = trained
    assert info["final_loss"] < S.history[0][1]
    # prior-mean predictor: the average ln(1 + m) of 512 fresh simulations
    th = S.sample_theta(512, np.random.default_rng(5)).astype(np.float32)
    h, _ = S.simulate(th)
    mean_pred = torch.log1p(h.reshape(512, -1).float()).mean(0, keepdim=True)
    d_mock, mom, npix = _mock(S)
    err = S.errors(n_test=256, seed=42, d_mock=d_mock, mock_moments=mom, mock_n_pix=npix)
    th2 = S.sample_theta(256, np.random.default_rng(42)).astype(np.float32)
    h2, _ = S.simulate(th2, set_id0=7 << 26)
    y2 = torch.log1p(h2.reshape(256, -1).float())
    rms_mean = float(((mean_pred - y2) ** 2).mean().sqrt())
    assert err["rms_log_bin"] < 0.85 * rms_mean, (err, rms_mean)
    assert err["ll_spearman"] > 0.9, err


def test_prescreen_cuts_exact_calls(trained):
    from paper_1904_00011_gb300.sampler import nested_sampling
    S, _ = trained
    d_mock, mom, npix = _mock(S)
    err = S.errors(n_test=256, seed=43, d_mock=d_mock, mock_moments=mom, mock_n_pix=npix)
    offset, margin = err["ll_offset"], 2.0 * err["ll_spread_p90"]

    def exact(th):
        return S.exact_loglike(th, d_mock, mom, npix)

    def sur(th):
        return S.loglike(th, d_mock, npix) + offset

    def prior(n, rng):
        return S.sample_theta(n, rng).astype(np.float32)

    plain = nested_sampling(exact, prior, n_live=32, n_iter=96, seed=3)
    fast = nested_sampling(exact, prior, n_live=32, n_iter=96, seed=3, surrogate_ll=sur,
                           margin=margin)
    assert fast.iterations == plain.iterations == 96
    # the filtered chain explores the same constrained prior: its final threshold is comparable
    assert fast.l_min_final > plain.l_min_final - 4 * margin, (plain, fast, margin)
    assert fast.exact_calls_per_replacement * 1.5 < plain.exact_calls_per_replacement, (plain, fast, err)
