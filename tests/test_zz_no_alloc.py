"""The allocation-free Hess stage (pcmd_hess_noalloc) against the context-based pcmd_hess.

pcmd_hess_noalloc serves callers that may not allocate GPU memory (a host application whose
pool owns the device, or a loop where cudaMalloc would stall other streams).  It keeps its
working memory in one fixed device array shared by all calls, so this test calls it twice in a
row on the same image and checks both results against pcmd_hess: histogram and counters
identical, moments within the tolerance of the other tests.  The file is named so that pytest
collects it last."""
import ctypes

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


def _pixel_config(w, set_id, psf):
    import paper_1904_00011_gb300 as P
    c = P.pcmd_pixel_config()
    c.n_bands = w.n_bands
    for b in range(P.PCMD_MAX_BANDS):
        c.exptime[b] = w.exptime[b]
        c.zeropoint[b] = w.zeropoint[b]
        c.sky[b] = w.sky[b]
    c.noise = 1 if (w.flags & P.PCMD_FLAG_NOISE) else 0
    c.seed = w.seed
    c.set_id = set_id
    if psf is not None:
        c.psf = psf.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        c.psf_size = psf.shape[-1]
    c.hess_nx, c.hess_ny = w.hess_nx, w.hess_ny
    c.hess_c_lo, c.hess_m_lo, c.hess_width = w.hess_c_lo, w.hess_m_lo, w.hess_width
    return c


@pytest.mark.parametrize("psf_size", [25, 9, 0])
def test_no_alloc_hess_matches_pcmd_hess_twice(psf_size):
    import dataclasses
    import paper_1904_00011_gb300 as P
    from paper_1904_00011_gb300 import workloads as W

    w = W.full(n_im=96, sky=25.0)
    if psf_size == 0:
        w = dataclasses.replace(w, psf=None)
    elif psf_size != 25:
        w = dataclasses.replace(w, psf=W.moffat_psf(psf_size, (2.0, 1.8)))
    n = w.n_im
    set_id = 5
    sim = P.Simulator(w)
    image = sim.image(w.params, [n], first_set_id=set_id)     # raw fluxes in a caller buffer
    h_ref, m_ref, c_ref, _ = sim.hess(1, [n])                  # the context-based Hess stage
    torch.cuda.synchronize()
    psf = None if w.psf is None else np.ascontiguousarray(w.psf[:w.n_bands], np.float32)
    cfg = _pixel_config(w, set_id, psf)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        h = torch.full((w.hess_ny, w.hess_nx), 7, dtype=torch.int32, device="cuda")
        m = torch.zeros(3, dtype=torch.float64, device="cuda")
        c = torch.full((2,), 7, dtype=torch.int32, device="cuda")
        P.pcmd_hess_noalloc(cfg, image.data_ptr(), n, h.data_ptr(), m.data_ptr(), c.data_ptr(), stream)
        torch.cuda.synchronize()
        assert torch.equal(h, h_ref[0]), call
        assert torch.equal(c, c_ref[0]), call
        assert np.allclose(m.cpu().numpy(), m_ref[0].cpu().numpy(), rtol=1e-12, atol=0), call
        assert int(h.sum()) + int(c.sum()) == n * n


def test_no_alloc_rejects_oversized_image():
    import paper_1904_00011_gb300 as P
    from paper_1904_00011_gb300 import workloads as W
    w = W.tiny()
    cfg = _pixel_config(w, 0, None)
    buf = torch.zeros(16, device="cuda")
    with pytest.raises(P.PcmdError) as e:
        P.pcmd_hess_noalloc(cfg, buf.data_ptr(), 8193, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), None)
    assert e.value.code == 1


def test_no_alloc_rejects_non_finite_settings():
    import paper_1904_00011_gb300 as P
    from paper_1904_00011_gb300 import workloads as W
    w = W.tiny()
    buf = torch.zeros(16, device="cuda")
    for field, value in (("sky", float("inf")), ("exptime", float("inf")), ("zeropoint", float("nan")),
                         ("hess_c_lo", float("nan")), ("hess_width", float("inf"))):
        cfg = _pixel_config(w, 0, None)
        if field in ("sky", "exptime", "zeropoint"):
            getattr(cfg, field)[0] = value
        else:
            setattr(cfg, field, value)
        with pytest.raises(P.PcmdError) as e:
            P.pcmd_hess_noalloc(cfg, buf.data_ptr(), 8, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), None)
        assert e.value.code == 1, field
