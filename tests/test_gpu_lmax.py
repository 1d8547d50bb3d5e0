"""Appendix A on the GPU: the best fit recomputed 100 times in one batched call (100 RNG set ids)
equals 100 single evaluations with the same set ids, and its median is the ceiling L_max."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_1904_00011_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_00011_gb300 import build
    build.build()


@pytest.mark.parametrize("psf", [True, False])
def test_batched_repeats_equal_single_evaluations(psf):
    import paper_1904_00011_gb300 as P
    from paper_1904_00011_gb300 import sampler as S
    n_im, reps = 64, 24
    w = W.full(n_im=n_im, psf=psf)
    sim = P.Simulator(w, max_sets=100)
    sim.simulate(w.params, [n_im], 123_456)
    h, m, _, _ = sim.hess(1, [n_im])
    torch.cuda.synchronize()
    mock, mom = h[0].clone(), m[0].cpu().numpy().copy()
    p = w.params[0]
    ll_b = sim.evaluate([p] * reps, [n_im] * reps, mock, mom, n_im * n_im, W.LL_PAPER, first_set_id=500)
    ll_s = np.array([sim.evaluate([p], [n_im], mock, mom, n_im * n_im, W.LL_PAPER, first_set_id=500 + k)[0]
                     for k in range(reps)])
    assert np.allclose(ll_b, ll_s, rtol=1e-12, atol=0.0), np.abs(ll_b - ll_s).max()
    assert np.std(ll_b) > 0.0                       # the likelihood is stochastic
    l_max = S.lmax_from_repeats(ll_b)
    assert ll_b.min() <= l_max <= ll_b.max()


@pytest.mark.parametrize("psf", [True, False])
def test_repeats_match_oracle(psf):
    """Five of the batched repeats (set ids 500-504) against the oracle's forward model and
    likelihood (Eq. 2-4) on the same set ids, with the oracle's own realisation as the data."""
    import oracle as O
    import paper_1904_00011_gb300 as P
    O.build()
    n_im, reps = 64, 24
    w = W.full(n_im=n_im, psf=psf)
    mock = O.model(w, 0, 123_456, n_threads=16)
    d_mock = torch.from_numpy(mock["hist"].view(np.int32)).cuda()
    sim = P.Simulator(w, max_sets=100)
    p = w.params[0]
    ll_b = sim.evaluate([p] * reps, [n_im] * reps, d_mock, mock["moments"], n_im * n_im, W.LL_PAPER,
                        first_set_id=500)
    for k in range(5):
        ref = O.model(w, 0, 500 + k, n_threads=16)
        ll_o = O.loglike(ref["hist"], ref["moments"], n_im * n_im, mock["hist"], mock["moments"],
                         n_im * n_im, O.LL_PAPER)
        assert ll_b[k] == pytest.approx(ll_o, rel=1e-4), (k, ll_b[k], ll_o)
