"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element on the
same seeded inputs.  Bars: star counts and bins from identical FP32 magnitudes bit-exact;
fluxes within 1e-5 relative; fewer than 1e-4 of pixels changing Hess bin; log-likelihood within
1e-4 relative."""
import dataclasses
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1904_00011_gb300 import workloads as W  # noqa: E402

FLUX_RTOL = 1e-5
LL_RTOL = 1e-4
BIN_CHANGE_MAX = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_00011_gb300 import build
    build.build()
    O.build()


def _sim(w, **kw):
    import paper_1904_00011_gb300 as P
    return P.Simulator(w, **kw)


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


# ------------------------------------------------------------------------------ tables

def _parametric_full():
    """The full model with a Kroupa IMF and a delayed-tau SFH (Section 2.2 S4) on its age bins."""
    import paper_1904_00011_gb300 as P
    w = W.full()
    edges = np.array(W._edges(W.FULL_LOG_AGES))
    sfh = P.sfh_bins(P.PCMD_SFH_DELAYED_TAU, [2.5, 3.0], edges)
    p = dataclasses.replace(w.params[0], log_sfh=sfh)
    return dataclasses.replace(w, imf=1, params=[p])


@pytest.mark.parametrize("name", ["tiny", "full", "large", "kroupa_tau"])
def test_tables_match_oracle(name):
    w = {"tiny": W.tiny, "full": W.full, "large": lambda: W.large(log_npix=6.5),
         "kroupa_tau": _parametric_full}[name]()
    s = _sim(w)
    lam, flux, z0 = s.tables(w.params[0])
    lam_o, flux_o, _ = O.tables(w)
    assert np.array_equal(lam, lam_o)                       # FP32 means bit-exact
    # FP32 rounding of the FP64 fluxes; the library applies distance as one factor, so the FP64
    # values may differ in the last bit and the FP32 table by at most one unit in the last place
    f32 = flux_o.astype(np.float32)
    assert np.all(np.abs(flux.view(np.int32) - f32.view(np.int32)) <= 1)
    rng = np.random.default_rng(0)
    for h in range(2):
        # below a mean of ~22 some word gives zero stars: Z_0 >= 0 is exported
        idx = np.nonzero((lam[h] > 0) & (lam[h] < 22))[0]
        for i in rng.choice(idx, size=min(60, idx.size), replace=False):
            # z0 is the largest word with zero stars under the oracle's inversion
            assert O.poisson_inversion(float(lam[h, i]), int(z0[h, i])) == 0
            if z0[h, i] < 0xFFFFFFFF:
                assert O.poisson_inversion(float(lam[h, i]), int(z0[h, i]) + 1) >= 1
        # from ~22.9 to 640 even the smallest word gives a star (e^-lambda 2^32 < 1/2): no Z_0
        big = np.nonzero((lam[h] > 22.9) & (lam[h] < 640))[0]
        for i in big[:20]:
            assert z0[h, i] == 0xFFFFFFFF
            assert O.poisson_inversion(float(lam[h, i]), 0) >= 1


# ------------------------------------------------------------------------------ counts

def _counts_case(w, n_im, set_id, pixels):
    s = _sim(w, max_im=n_im)
    p = w.params[0]
    for (p0, n) in pixels:
        got = _u32(s.counts(p, n_im, set_id, p0, n))
        _, ref = O.simulate(w, 0, set_id, pix_begin=p0, pix_end=p0 + n, counts=True, n_im=n_im, n_threads=8)
        assert got.shape == ref.shape
        bad = np.argwhere(got != ref)
        assert bad.size == 0, (bad[:5], got[tuple(bad[0])], ref[tuple(bad[0])])


def test_counts_bit_exact_tiny_whole_image():
    _counts_case(W.tiny(), 64, 0, [(0, 64 * 64)])


def test_counts_bit_exact_full_sampled_pixels():
    w = W.full()
    _counts_case(w, 256, 7, [(0, 96), (33000, 64), (65536 - 70, 70)])


def test_counts_bit_exact_kroupa_delayed_tau():
    _counts_case(_parametric_full(), 256, 9, [(100, 64), (40000, 64)])


@pytest.mark.parametrize("log_npix", [4.0, 6.5])
def test_counts_bit_exact_large_npix(log_npix):
    w = W.large(log_npix=log_npix)
    _counts_case(w, 1024, 3, [(5, 16), (1024 * 1024 - 16, 16)])


def test_counts_ragged_isochrone_not_multiple_of_8():
    iso = W.make_isochrones(seed=3, log_ages=[9.0], fehs=[-0.5], n_mass=13, n_bands=2)
    w = dataclasses.replace(W.tiny(n_im=40), iso=iso)
    w.params[0].log_sfh = np.array([2.3])
    _counts_case(w, 40, 2, [(0, 1600)])


# ------------------------------------------------------------------------------ raw flux

@pytest.mark.parametrize("name", ["tiny", "full", "large"])
def test_raw_flux_full_size_sampled(name):
    """Raw images of the full-size launch (the bench's launch shape) at sampled pixels."""
    w = {"tiny": W.tiny, "full": W.full, "large": lambda: W.large(log_npix=6.0)}[name]()
    n = w.n_im
    s = _sim(w)
    img = s.image(w.params, [n]).cpu().numpy().reshape(w.n_bands, n * n).astype(np.float64)
    rng = np.random.default_rng(1)
    picks = sorted(set(rng.integers(0, n * n, size=24).tolist()) | {0, n * n - 1})
    ref = np.zeros((w.n_bands, len(picks)))
    for k, p in enumerate(picks):
        ref[:, k] = O.simulate(w, 0, 0, pix_begin=p, pix_end=p + 1)[:, p]
    got = img[:, picks]
    rel = np.abs(got - ref) / np.where(ref != 0.0, np.abs(ref), 1.0)
    assert np.all(rel <= FLUX_RTOL), rel.max()


# ------------------------------------------------------------------------------ end to end

def _end_to_end(w, n_threads=16):
    n = w.n_im
    s = _sim(w)
    s.simulate(w.params, [n], 0)
    h, m, c, px = s.hess(1, [n], pixels=True)
    torch.cuda.synchronize()
    ref = O.model(w, 0, 0, n_threads=n_threads)
    return s, h, m, c, px, ref


@pytest.mark.parametrize("name", ["tiny", "full_small", "full", "psf_grid", "psf_grid_ragged", "pool",
                                  "large_physics"])
def test_end_to_end_fluxes_bins_loglike(name):
    # large_physics: the large-Npix model (3 bands, log10 Npix 6.5: sparse, dense and
    # transformed-rejection draws, Kahan sums, dust, 25x25 PSF, noise) on a 128x128 image
    w = {"tiny": W.tiny, "full_small": lambda: W.full(n_im=128, sky=40.0),
         "large_physics": lambda: W.large(n_im=128, log_npix=6.5),
         "full": W.full, "psf_grid": lambda: W.full(n_im=128, psf_grid=True),
         "psf_grid_ragged": lambda: W.full(n_im=100, psf_grid=True, sky=10.0),
         "pool": lambda: dataclasses.replace(W.full(n_im=128, sky=20.0),
                                             flags=W.full().flags | W.FLAG_POOL)}[name]()
    n = w.n_im
    npix = n * n
    s, h, m, c, px, ref = _end_to_end(w)
    B = w.n_bands
    px = px.cpu().numpy().reshape(B + 2, npix)
    # noisy fluxes (post PSF and noise)
    fl = px[:B].astype(np.float64)
    # every pixel within 1e-5 relative of the FP64 oracle (no pixel exempt); a pixel whose
    # noisy flux is exactly zero in the oracle may only be zero on the GPU too
    rel = np.abs(fl - ref["flux"]) / np.where(ref["flux"] != 0.0, np.abs(ref["flux"]), 1.0)
    print("%s: max relative error of the noisy fluxes %.3g over %d values" % (name, rel.max(), rel.size))
    assert np.all(rel <= FLUX_RTOL), (rel.max(), np.unravel_index(np.argmax(rel), rel.shape))
    # bins: pixels whose (ix, iy) differ
    valid = ref["valid"] > 0
    gv = ~np.isnan(px[B])
    assert np.mean(gv != valid) < BIN_CHANGE_MAX

    def bins(mag, col):
        ix = np.floor((col.astype(np.float32) - np.float32(w.hess_c_lo)) * np.float32(1 / w.hess_width))
        iy = np.floor((mag.astype(np.float32) - np.float32(w.hess_m_lo)) * np.float32(1 / w.hess_width))
        return ix, iy

    both = valid & gv
    gx, gy = bins(px[B][both], px[B + 1][both])
    ox, oy = bins(ref["mag"][both], ref["colour"][both])
    changed = np.mean((gx != ox) | (gy != oy)) if both.any() else 0.0
    assert changed < BIN_CHANGE_MAX, changed
    # histogram and counters
    gh = _u32(h)[0]
    assert gh.sum() + _u32(c)[0].sum() == npix
    diff = np.abs(gh.astype(np.int64) - ref["hist"].astype(np.int64)).sum()
    assert diff <= 2 * max(1, int(BIN_CHANGE_MAX * npix)), diff
    # moments
    mm = m.cpu().numpy()[0]
    assert mm[2] == pytest.approx(ref["moments"][2], abs=2)
    assert mm[0] / mm[2] == pytest.approx(ref["moments"][0] / ref["moments"][2], rel=1e-6, abs=1e-6)
    assert mm[1] / mm[2] == pytest.approx(ref["moments"][1] / ref["moments"][2], rel=1e-7)
    # likelihood against a mock (the oracle's own realisation with another set id)
    mock = O.model(w, 0, 1000, n_threads=16)
    d_mock = torch.from_numpy(mock["hist"].view(np.int32)).cuda()
    for mode in (O.LL_PAPER, O.LL_POISSON):
        ll = s.loglike(1, d_mock, mock["moments"], npix, mode)[0]
        ll_o = O.loglike(ref["hist"], ref["moments"], npix, mock["hist"], mock["moments"], npix, mode)
        assert ll == pytest.approx(ll_o, rel=LL_RTOL), (mode, ll, ll_o)


def test_bins_bit_exact_from_identical_fp32_magnitudes():
    w = W.full()
    s = _sim(w)
    rng = np.random.default_rng(5)
    n = 200000
    mag = rng.uniform(21.0, 27.0, n).astype(np.float32)
    col = rng.uniform(-1.5, 4.5, n).astype(np.float32)
    # values on and next to bin edges
    edges_m = (np.float32(21.5) + np.arange(0, 100, dtype=np.float32) * np.float32(0.05)).astype(np.float32)
    mag[:100] = edges_m
    mag[100:200] = np.nextafter(edges_m, np.float32(-np.inf))
    mag[200:300] = np.nextafter(edges_m, np.float32(np.inf))
    col[300:400] = (np.float32(-1.0) + np.arange(100, dtype=np.float32) * np.float32(0.05))
    valid = (rng.uniform(size=n) > 0.01).astype(np.uint8)
    h, c, m = s.bin_mags(torch.from_numpy(mag).cuda(), torch.from_numpy(col).cuda(),
                         torch.from_numpy(valid).cuda())
    oh, oc, om = O.hess(w, mag, col, valid)
    assert np.array_equal(_u32(h), oh)
    assert np.array_equal(_u32(c), oc)


# ------------------------------------------------------------------------------ batching

def test_fused_batch_matches_per_set_path_and_oracle():
    w = W.batch(n_sets=12, n_min=32, n_max=96, step=16)
    mp = W.batch_mock_params()
    wm = W.with_params(w, [mp], [96])
    mock = O.model(wm, 0, 999, n_threads=16)
    d_mock = torch.from_numpy(mock["hist"].view(np.int32)).cuda()
    s = _sim(w, max_sets=w.n_sets)
    ll = s.evaluate(w.params, w.n_ims, d_mock, mock["moments"], 96 * 96, W.LL_POISSON, first_set_id=50)
    hb = _u32(torch.from_numpy(np.zeros(1)))  # placeholder to keep API symmetric
    del hb
    # per-set path (image + Hess kernel), same set ids
    s.simulate(w.params, w.n_ims, 50)
    h, m, c, _ = s.hess(w.n_sets, w.n_ims)
    ll2 = s.loglike(w.n_sets, d_mock, mock["moments"], 96 * 96, W.LL_POISSON)
    assert np.allclose(ll, ll2, rtol=1e-12, atol=1e-9)
    for k in range(w.n_sets):
        ref = O.model(w, k, 50 + k, n_threads=16)
        gh = _u32(h)[k]
        n2 = w.n_ims[k] ** 2
        assert gh.sum() + _u32(c)[k].sum() == n2
        assert np.abs(gh.astype(np.int64) - ref["hist"].astype(np.int64)).sum() <= 2
        ll_o = O.loglike(ref["hist"], ref["moments"], n2, mock["hist"], mock["moments"], 96 * 96,
                         O.LL_POISSON)
        assert ll[k] == pytest.approx(ll_o, rel=LL_RTOL)


def test_batch_of_full_size_sets_matches_oracle():
    """The batched workload at its own sizes: 20 of its sets (images 128..512, log10 Npix 1..6)
    plus three 512x512 sets at log10 Npix 5.5, 5.8 and 6.0 (transformed rejection and dense groups),
    all in one fused persistent launch.  Every set's likelihood against the oracle's; the big
    sets' counts at sampled pixels bit for bit; every set's Hess diagram (per-set path, same
    set ids) within the bin-change bar."""
    w0 = W.batch()
    params = list(w0.params[:20])
    sizes = list(w0.n_ims[:20])
    for lg in (5.5, 5.8, 6.0):
        params.append(dataclasses.replace(w0.params[0], log_sfh=np.array([lg])))
        sizes.append(512)
    w = W.with_params(w0, params, sizes)
    mp = W.batch_mock_params()
    mock = O.model(W.with_params(w0, [mp], [256]), 0, 999, n_threads=16)
    d_mock = torch.from_numpy(mock["hist"].view(np.int32)).cuda()
    s = _sim(w, max_sets=w.n_sets, max_im=512)
    first = 7000
    ll = s.evaluate(w.params, w.n_ims, d_mock, mock["moments"], 256 * 256, W.LL_POISSON,
                    first_set_id=first)
    s.simulate(w.params, w.n_ims, first)
    h, m, c, _ = s.hess(w.n_sets, w.n_ims)
    gh_all, gc_all = _u32(h), _u32(c)
    for k in range(w.n_sets):
        n2 = w.n_ims[k] ** 2
        ref = O.model(w, k, first + k, n_threads=16)
        gh = gh_all[k]
        assert gh.sum() + gc_all[k].sum() == n2
        assert np.abs(gh.astype(np.int64) - ref["hist"].astype(np.int64)).sum() <= \
            2 * max(1, int(BIN_CHANGE_MAX * n2)), k
        ll_o = O.loglike(ref["hist"], ref["moments"], n2, mock["hist"], mock["moments"], 256 * 256,
                         O.LL_POISSON)
        assert ll[k] == pytest.approx(ll_o, rel=LL_RTOL), (k, ll[k], ll_o)
    big = _sim(w, max_im=512)
    for k in range(20, 23):
        got = _u32(big.counts(w.params[k], 512, first + k, 131000, 48))
        _, ref = O.simulate(w, k, first + k, pix_begin=131000, pix_end=131048, counts=True, n_threads=16)
        assert np.array_equal(got, ref), k


def test_launch_shape_does_not_change_counts():
    w = W.full(n_im=96)
    s = _sim(w)
    ref = _u32(s.counts(w.params[0], 96, 4, 0, 96 * 96))
    for (block, split, chunk) in [(256, 1, 64), (128, 2, 17), (64, 2, 256), (256, 8, 1)]:
        s.set_launch(block, split, chunk)
        got = _u32(s.counts(w.params[0], 96, 4, 0, 96 * 96))
        assert np.array_equal(got, ref), (block, split, chunk)


# ------------------------------------------------------------------------------ edges

def test_single_pixel_and_ragged_images():
    w = W.full(n_im=37, psf=True)
    for n in (1, 5, 37):
        w2 = dataclasses.replace(w, n_im=n, n_ims=[n])
        s, h, m, c, px, ref = _end_to_end(w2)
        gh = _u32(h)[0]
        assert gh.sum() + _u32(c)[0].sum() == n * n
        assert np.abs(gh.astype(np.int64) - ref["hist"].astype(np.int64)).sum() <= 2


def test_nearly_empty_pixels_are_invalid():
    w = W.tiny(npix=1e-3)
    s, h, m, c, px, ref = _end_to_end(w)
    assert _u32(c)[0][1] == ref["counters"][1] and ref["counters"][1] > 4000


@pytest.mark.parametrize("fused", [False, True])
def test_sampler_limit_is_latched_and_reported(fused):
    """A transformed-rejection draw that reaches the attempt cap latches PCMD_ERR_SAMPLER_LIMIT in
    the device error word; the next synchronising call returns it, and once the cap is restored
    the same context evaluates normally and equals a fresh context.  fused: the graph-replayed
    batched path (no PSF), else the image + PSF path."""
    import paper_1904_00011_gb300 as P
    w = W.large(n_im=64, log_npix=6.5)
    if fused:
        w = dataclasses.replace(w, psf=None)
    s = _sim(w)
    n = w.n_im
    s.simulate(w.params, [n], 31)
    h, m, _, _ = s.hess(1, [n])
    torch.cuda.synchronize()
    mock, mom = h[0].clone(), m[0].cpu().numpy().copy()
    ll0 = s.evaluate(w.params, [n], mock, mom, n * n, W.LL_PAPER, first_set_id=40)[0]
    s.set_attempt_cap(1)           # about one draw in seven needs a second attempt
    with pytest.raises(P.PcmdError) as e:
        s.evaluate(w.params, [n], mock, mom, n * n, W.LL_PAPER, first_set_id=40)
    assert e.value.code == 4       # PCMD_ERR_SAMPLER_LIMIT
    s.set_attempt_cap(0)
    ll1 = s.evaluate(w.params, [n], mock, mom, n * n, W.LL_PAPER, first_set_id=40)[0]
    assert ll1 == ll0
    fresh = _sim(w)
    assert fresh.evaluate(w.params, [n], mock, mom, n * n, W.LL_PAPER, first_set_id=40)[0] == ll0
    with pytest.raises(P.PcmdError) as e:
        s.set_attempt_cap(1025)
    assert e.value.code == 1


def test_argument_and_state_errors():
    import paper_1904_00011_gb300 as P
    w = W.tiny()
    s = _sim(w, max_im=64, max_sets=2)
    with pytest.raises(P.PcmdError) as e:
        s.simulate(w.params, [65])
    assert e.value.code == 1
    with pytest.raises(P.PcmdError) as e:
        s.simulate(w.params * 3, [8, 8, 8])
    assert e.value.code == 1
    bad = dataclasses.replace(w.params[0], dust_sigma=float("nan"))
    with pytest.raises(P.PcmdError):
        s.simulate([bad], [8])
    s2 = _sim(w)
    with pytest.raises(P.PcmdError) as e:
        s2.hess(1, [64])
    assert e.value.code == 5
