"""The total-count (pool) sampler through the C ABI against the oracle's pool mode: star counts
bit-exact (sparse, full, large with transformed-rejection totals, ragged isochrone) and the
fused batched path (end to end: test_gpu_parity's "pool" case)."""
import dataclasses

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1904_00011_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_00011_gb300 import build
    build.build()


def _pool(w):
    return dataclasses.replace(w, flags=w.flags | W.FLAG_POOL)


def _counts(w, n_im, set_id, pixels):
    import paper_1904_00011_gb300 as P
    s = P.Simulator(w, max_sets=1, max_im=n_im)
    for (p0, n) in pixels:
        got = s.counts(w.params[0], n_im, set_id, p0, n).cpu().numpy().view(np.uint32)
        _, ref = O.simulate(w, 0, set_id, pix_begin=p0, pix_end=p0 + n, counts=True, n_im=n_im, n_threads=8)
        bad = np.argwhere(got != ref)
        assert bad.size == 0, (bad[:5], got[tuple(bad[0])], ref[tuple(bad[0])])


def test_pool_counts_tiny_whole_image():
    _counts(_pool(W.tiny()), 64, 0, [(0, 64 * 64)])


def test_pool_counts_full_sampled_pixels():
    _counts(_pool(W.full()), 256, 7, [(0, 96), (33000, 64), (65536 - 70, 70)])


@pytest.mark.parametrize("log_npix", [3.0, 5.0])
def test_pool_counts_with_large_totals_and_ptrs_points(log_npix):
    w = _pool(W.large(log_npix=log_npix, n_im=64))
    _counts(w, 64, 3, [(5, 32), (64 * 64 - 32, 32)])


def test_pool_counts_ragged_isochrone():
    iso = W.make_isochrones(seed=31, log_ages=[9.0], fehs=[-0.5], n_mass=13, n_bands=2)
    w = dataclasses.replace(W.tiny(n_im=40), iso=iso)
    _counts(_pool(w), 40, 2, [(0, 40 * 40)])


def test_pool_fused_batch_equals_per_set_path():
    import paper_1904_00011_gb300 as P
    w = _pool(W.batch(n_sets=6, n_min=32, n_max=64, step=16))
    s = P.Simulator(w, max_sets=w.n_sets)
    mp = W.batch_mock_params()
    wm = W.with_params(w, [mp], [64])
    ms = P.Simulator(wm, max_sets=1, max_im=64)
    ms.simulate([mp], [64], 99)
    h, m, _, _ = ms.hess(1, [64])
    torch.cuda.synchronize()
    mock, mom = h[0].clone(), m[0].cpu().numpy().copy()
    ll_b = s.evaluate(w.params, w.n_ims, mock, mom, 64 * 64, W.LL_POISSON, first_set_id=70)
    ll_1 = [s.evaluate([w.params[k]], [w.n_ims[k]], mock, mom, 64 * 64, W.LL_POISSON, first_set_id=70 + k)[0]
            for k in range(w.n_sets)]
    assert np.allclose(ll_b, ll_1, rtol=1e-12, atol=0.0)
