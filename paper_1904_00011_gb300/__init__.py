"""GB300-native pCMD forward model: Python binding of libpcmd (include/pcmd.h).

Argument marshalling only: every step of the forward model runs in the library's CUDA kernels.
PyTorch provides device memory and the stream.  The functions ``pcmd_*`` mirror the C ABI one to
one; ``Simulator`` wraps a context built from a ``workloads.Workload``.

There is no CPU fallback: importing the library on a machine where it cannot be loaded, or
calling into it without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

from . import workloads

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpcmd.so")

PCMD_MAX_BANDS = 4
PCMD_MAX_SFH = 32

STATUS = {0: "PCMD_OK", 1: "PCMD_ERR_ARG", 2: "PCMD_ERR_CUDA", 3: "PCMD_ERR_OOM",
          4: "PCMD_ERR_SAMPLER_LIMIT", 5: "PCMD_ERR_STATE", 6: "PCMD_ERR_TIMEOUT"}
PCMD_FLAG_DUST, PCMD_FLAG_NOISE, PCMD_FLAG_KAHAN, PCMD_FLAG_SIGMA_SQRTSUM, PCMD_FLAG_POOL = 1, 2, 4, 8, 16
PCMD_LL_PAPER, PCMD_LL_POISSON = 0, 1
PCMD_IMF_POWER, PCMD_IMF_KROUPA = 0, 1
PCMD_SFH_SSP, PCMD_SFH_CONSTANT, PCMD_SFH_TAU, PCMD_SFH_DELAYED_TAU = 1, 2, 3, 4


class PcmdError(RuntimeError):
    def __init__(self, code: int, where: str, text: str = ""):
        super().__init__("%s failed: %s %s" % (where, STATUS.get(code, code), text))
        self.code = code


class pcmd_config(ctypes.Structure):
    _fields_ = [
        ("n_bands", ctypes.c_int), ("n_ages", ctypes.c_int), ("n_feh", ctypes.c_int),
        ("n_mass", ctypes.c_int),
        ("log_age", ctypes.POINTER(ctypes.c_double)), ("feh_grid", ctypes.POINTER(ctypes.c_double)),
        ("mass", ctypes.POINTER(ctypes.c_double)), ("abs_mag", ctypes.POINTER(ctypes.c_double)),
        ("imf_slope", ctypes.c_double),
        ("exptime", ctypes.c_double * PCMD_MAX_BANDS), ("zeropoint", ctypes.c_double * PCMD_MAX_BANDS),
        ("sky", ctypes.c_double * PCMD_MAX_BANDS), ("r_ext", ctypes.c_double * PCMD_MAX_BANDS),
        ("f_dust", ctypes.c_double), ("mdf_cut", ctypes.c_double),
        ("psf", ctypes.POINTER(ctypes.c_float)), ("psf_size", ctypes.c_int),
        ("hess_nx", ctypes.c_int), ("hess_ny", ctypes.c_int),
        ("hess_c_lo", ctypes.c_double), ("hess_m_lo", ctypes.c_double),
        ("hess_width", ctypes.c_double),
        ("max_im", ctypes.c_int), ("max_sets", ctypes.c_int),
        ("seed", ctypes.c_uint64), ("flags", ctypes.c_uint), ("stream", ctypes.c_void_p),
        ("imf", ctypes.c_int), ("psf_grid", ctypes.c_int),
    ]


class pcmd_params(ctypes.Structure):
    _fields_ = [("log_sfh", ctypes.c_double * PCMD_MAX_SFH), ("feh_mean", ctypes.c_double),
                ("feh_sigma", ctypes.c_double), ("log_ebv", ctypes.c_double),
                ("dust_sigma", ctypes.c_double), ("dmod", ctypes.c_double)]


class pcmd_pixel_config(ctypes.Structure):
    _fields_ = [("n_bands", ctypes.c_int), ("exptime", ctypes.c_double * PCMD_MAX_BANDS),
                ("zeropoint", ctypes.c_double * PCMD_MAX_BANDS), ("sky", ctypes.c_double * PCMD_MAX_BANDS),
                ("noise", ctypes.c_int), ("seed", ctypes.c_uint64), ("set_id", ctypes.c_uint32),
                ("psf", ctypes.POINTER(ctypes.c_float)), ("psf_size", ctypes.c_int),
                ("hess_nx", ctypes.c_int), ("hess_ny", ctypes.c_int), ("hess_c_lo", ctypes.c_double),
                ("hess_m_lo", ctypes.c_double), ("hess_width", ctypes.c_double)]


_lib = None


def lib():
    """Load libpcmd.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libpcmd.so is not built: run paper_1904_00011_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, u32, u64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
        cfgp = ctypes.POINTER(pcmd_config)
        parp = ctypes.POINTER(pcmd_params)
        ip = ctypes.POINTER(ctypes.c_int)
        dp = ctypes.POINTER(ctypes.c_double)
        L.pcmd_create.argtypes = [cfgp, ctypes.POINTER(vp)]
        L.pcmd_destroy.argtypes = [vp]
        L.pcmd_destroy.restype = None
        L.pcmd_last_error.argtypes = [vp]
        L.pcmd_last_error.restype = ctypes.c_char_p
        L.pcmd_simulate.argtypes = [vp, parp, i, ip, u32, vp]
        L.pcmd_hess.argtypes = [vp, vp, vp, vp, vp]
        L.pcmd_loglike.argtypes = [vp, vp, dp, d, i, dp]
        L.pcmd_evaluate.argtypes = [vp, parp, i, ip, u32, vp, dp, d, i, dp]
        L.pcmd_sync.argtypes = [vp]
        L.pcmd_n_points.argtypes = [vp]
        L.pcmd_set_launch.argtypes = [vp, i, i, i]
        L.pcmd_set_attempt_cap.argtypes = [vp, i]
        L.pcmd_get_tables.argtypes = [vp, parp, vp, vp, vp]
        L.pcmd_sfh_bins.argtypes = [ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp, vp]
        L.pcmd_sfh_bins.restype = ctypes.c_int
        L.pcmd_counts.argtypes = [vp, parp, i, u32, u32, u32, vp]
        L.pcmd_bin_mags.argtypes = [vp, vp, vp, vp, u32, vp, vp, vp]
        L.pcmd_profile.argtypes = [vp, i]
        L.pcmd_hess_noalloc.argtypes = [ctypes.POINTER(pcmd_pixel_config), vp, i, vp, vp, vp, vp]
        L.pcmd_gemm_bf16.argtypes = [vp, i, vp, i, vp, i, vp, vp, i, i, i, i, vp, vp]
        L.pcmd_kernel_times.argtypes = [vp, dp, ip]
        for name in ["pcmd_create", "pcmd_simulate", "pcmd_hess", "pcmd_loglike", "pcmd_evaluate",
                     "pcmd_sync", "pcmd_n_points", "pcmd_set_launch", "pcmd_set_attempt_cap",
                     "pcmd_get_tables",
                     "pcmd_counts", "pcmd_bin_mags", "pcmd_profile", "pcmd_kernel_times",
                     "pcmd_hess_noalloc", "pcmd_gemm_bf16"]:
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int, where: str, ctx=None):
    if rc != 0:
        text = ""
        if ctx:
            text = lib().pcmd_last_error(ctx).decode(errors="replace")
        raise PcmdError(rc, where, text)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(p: "workloads.Params") -> pcmd_params:
    out = pcmd_params()
    sfh = np.asarray(p.log_sfh, np.float64)
    for j, v in enumerate(sfh):
        out.log_sfh[j] = float(v)
    out.feh_mean, out.feh_sigma = float(p.feh_mean), float(p.feh_sigma)
    out.log_ebv, out.dust_sigma, out.dmod = float(p.log_ebv), float(p.dust_sigma), float(p.dmod)
    return out


def params_array(ps):
    """pcmd_params[n] from a list of workloads.Params, or (no per-set Python work) from a float64
    matrix [n][PCMD_MAX_SFH + 5] laid out as the struct: log SFH bins, [Fe/H] mean and width,
    log E(B-V), dust width, distance modulus."""
    if isinstance(ps, np.ndarray):
        a = np.ascontiguousarray(ps, np.float64)
        if a.ndim != 2 or a.shape[1] != PCMD_MAX_SFH + 5:
            raise ValueError("parameter matrix must be [n][%d]" % (PCMD_MAX_SFH + 5))
        return (pcmd_params * a.shape[0]).from_buffer(a)
    arr = (pcmd_params * len(ps))()
    for k, p in enumerate(ps):
        arr[k] = make_params(p)
    return arr


# ------------------------------------------------------------------------------------------
# one-to-one wrappers of the C ABI
# ------------------------------------------------------------------------------------------

def pcmd_create(cfg: pcmd_config):
    ctx = ctypes.c_void_p()
    _check(lib().pcmd_create(ctypes.byref(cfg), ctypes.byref(ctx)), "pcmd_create")
    return ctx


def pcmd_destroy(ctx) -> None:
    lib().pcmd_destroy(ctx)


def pcmd_simulate(ctx, params, n_sets: int, n_im, first_set_id: int, d_image=None) -> None:
    _check(lib().pcmd_simulate(ctx, params, n_sets, n_im, first_set_id, d_image), "pcmd_simulate", ctx)


def pcmd_hess(ctx, d_hess=None, d_moments=None, d_counters=None, d_pixels=None) -> None:
    _check(lib().pcmd_hess(ctx, d_hess, d_moments, d_counters, d_pixels), "pcmd_hess", ctx)


def pcmd_loglike(ctx, d_mock_hess, mock_moments: np.ndarray, mock_n_pix: float, mode: int,
                 h_ll: np.ndarray) -> None:
    _check(lib().pcmd_loglike(ctx, d_mock_hess, _dptr(mock_moments), mock_n_pix, mode, _dptr(h_ll)),
           "pcmd_loglike", ctx)


def pcmd_evaluate(ctx, params, n_sets, n_im, first_set_id, d_mock_hess, mock_moments, mock_n_pix,
                  mode, h_ll) -> None:
    _check(lib().pcmd_evaluate(ctx, params, n_sets, n_im, first_set_id, d_mock_hess,
                               _dptr(mock_moments), mock_n_pix, mode, _dptr(h_ll)), "pcmd_evaluate", ctx)


def sfh_bins(model: int, theta, log_age_edges) -> np.ndarray:
    """Parametric SFH (Section 2.2 S1-S4) as log10 stars per age bin (host computation in the
    library; see pcmd_sfh_bins)."""
    th = np.ascontiguousarray(theta, np.float64)
    ed = np.ascontiguousarray(log_age_edges, np.float64)
    out = np.zeros(ed.size - 1, np.float64)
    _check(lib().pcmd_sfh_bins(int(model), th.ctypes.data, th.size, out.size, ed.ctypes.data,
                               out.ctypes.data), "pcmd_sfh_bins")
    return out


def pcmd_sync(ctx) -> None:
    _check(lib().pcmd_sync(ctx), "pcmd_sync", ctx)


def pcmd_hess_noalloc(cfg: pcmd_pixel_config, d_image, n_im: int, d_hess, d_moments, d_counters,
                      stream=None) -> None:
    """The Hess stage of one image without a context and without any device allocation (see
    include/pcmd.h); all arguments are device pointers except ``cfg``."""
    _check(lib().pcmd_hess_noalloc(ctypes.byref(cfg), d_image, n_im, d_hess, d_moments, d_counters,
                                   stream), "pcmd_hess_noalloc")


PCMD_GEMM_F32, PCMD_GEMM_BIAS_F32, PCMD_GEMM_BIAS_GELU_BF16, PCMD_GEMM_BIAS_BF16 = 0, 1, 2, 3


def pcmd_gemm_bf16(d_a, lda, d_b, ldb, d_c, ldc, d_bias, d_aux, m, n, k, epilogue, d_err,
                   stream=None) -> None:
    _check(lib().pcmd_gemm_bf16(d_a, lda, d_b, ldb, d_c, ldc, d_bias, d_aux, m, n, k, epilogue,
                                d_err, stream), "pcmd_gemm_bf16")


def gemm(a, b, bias=None, epilogue=PCMD_GEMM_F32, err=None, want_aux=True):
    """C = epilogue(a @ b.T) for BF16 CUDA tensors a [m, k], b [n, k] (row strides multiples of
    8 elements); returns (C, aux).  want_aux=False skips the pre-activation output of the GELU
    epilogue."""
    import torch
    m, k = a.shape
    n = b.shape[0]
    bf16_out = epilogue in (PCMD_GEMM_BIAS_GELU_BF16, PCMD_GEMM_BIAS_BF16)
    c = torch.empty((m, n), dtype=torch.bfloat16 if bf16_out else torch.float32, device=a.device)
    aux = torch.empty_like(c) if epilogue == PCMD_GEMM_BIAS_GELU_BF16 and want_aux else None
    if err is None:
        err = torch.zeros(1, dtype=torch.int32, device=a.device)
    pcmd_gemm_bf16(a.data_ptr(), a.stride(0), b.data_ptr(), b.stride(0), c.data_ptr(), c.stride(0),
                   _ptr(bias), _ptr(aux), m, n, k, epilogue, err.data_ptr(),
                   torch.cuda.current_stream().cuda_stream)
    return c, aux


KERNEL_KINDS = ["draw", "hess", "finalize", "loglike", "graph", "gemm", "tables", "spare"]


def pcmd_profile(ctx, enable: bool) -> None:
    _check(lib().pcmd_profile(ctx, int(bool(enable))), "pcmd_profile", ctx)


def pcmd_kernel_times(ctx):
    ms = np.zeros(8)
    cnt = (ctypes.c_int * 8)()
    _check(lib().pcmd_kernel_times(ctx, _dptr(ms), cnt), "pcmd_kernel_times", ctx)
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_KINDS)}


def pcmd_set_launch(ctx, block: int, split: int, chunk: int) -> None:
    _check(lib().pcmd_set_launch(ctx, block, split, chunk), "pcmd_set_launch", ctx)


def pcmd_set_attempt_cap(ctx, cap: int) -> None:
    _check(lib().pcmd_set_attempt_cap(ctx, cap), "pcmd_set_attempt_cap", ctx)


# ------------------------------------------------------------------------------------------
# Simulator: a context built from a Workload
# ------------------------------------------------------------------------------------------

class Simulator:
    """One library context for a workload's isochrones and hyper-parameters."""

    def __init__(self, w: "workloads.Workload", max_sets: Optional[int] = None,
                 max_im: Optional[int] = None, stream=None, device: Optional[int] = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the pCMD library needs a CUDA device (no CPU fallback)")
        self.torch = torch
        if device is not None:
            torch.cuda.set_device(device)
        self.w = w
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        iso = w.iso
        na, nf, nm = iso.mass.shape
        self._keep = []
        cfg = pcmd_config()
        cfg.n_bands, cfg.n_ages, cfg.n_feh, cfg.n_mass = w.n_bands, na, nf, nm

        def dbl(a):
            a = np.ascontiguousarray(a, np.float64)
            self._keep.append(a)
            return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

        cfg.log_age = dbl(iso.log_age)
        cfg.feh_grid = dbl(iso.feh)
        cfg.mass = dbl(iso.mass)
        cfg.abs_mag = dbl(iso.abs_mag[..., :w.n_bands])
        cfg.imf_slope = w.imf_slope
        cfg.imf = int(getattr(w, "imf", PCMD_IMF_POWER))
        for b in range(PCMD_MAX_BANDS):
            cfg.exptime[b] = w.exptime[b]
            cfg.zeropoint[b] = w.zeropoint[b]
            cfg.sky[b] = w.sky[b]
            cfg.r_ext[b] = w.r_ext[b]
        cfg.f_dust, cfg.mdf_cut = w.f_dust, w.mdf_cut
        if w.psf is not None:
            if w.psf.ndim == 4:       # sub-pixel grid [16][B][S][S]
                psf = np.ascontiguousarray(w.psf[:, :w.n_bands], np.float32)
                cfg.psf_grid = 4
            else:
                psf = np.ascontiguousarray(w.psf[:w.n_bands], np.float32)
            self._keep.append(psf)
            cfg.psf = psf.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
            cfg.psf_size = psf.shape[-1]
        cfg.hess_nx, cfg.hess_ny = w.hess_nx, w.hess_ny
        cfg.hess_c_lo, cfg.hess_m_lo, cfg.hess_width = w.hess_c_lo, w.hess_m_lo, w.hess_width
        cfg.max_im = int(max_im or max(w.n_ims))
        cfg.max_sets = int(max_sets or w.n_sets)
        cfg.seed = int(w.seed)
        cfg.flags = int(w.flags)
        cfg.stream = ctypes.c_void_p(self.stream.cuda_stream)
        self.cfg = cfg
        self.ctx = pcmd_create(cfg)
        self.n_points = lib().pcmd_n_points(self.ctx)
        self.nbins = w.hess_nx * w.hess_ny

    def close(self):
        if getattr(self, "ctx", None):
            pcmd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_launch(self, block: int, split: int, chunk: int):
        pcmd_set_launch(self.ctx, block, split, chunk)

    def set_attempt_cap(self, cap: int):
        pcmd_set_attempt_cap(self.ctx, cap)

    def profile(self, enable: bool = True):
        pcmd_profile(self.ctx, enable)

    def kernel_times(self):
        return pcmd_kernel_times(self.ctx)

    # ---- forward model -------------------------------------------------------------------
    def simulate(self, params: Sequence["workloads.Params"], n_ims: Sequence[int],
                 first_set_id: int = 0, out=None):
        ps = params_array(params)
        ni = (ctypes.c_int * len(n_ims))(*[int(v) for v in n_ims])
        pcmd_simulate(self.ctx, ps, len(params), ni, first_set_id, _ptr(out))
        return out

    def image(self, params, n_ims, first_set_id: int = 0):
        """Raw images as one float32 CUDA tensor, sets packed one after the other."""
        t = self.torch
        total = sum(self.w.n_bands * n * n for n in n_ims)
        out = t.empty(total, dtype=t.float32, device="cuda")
        self.simulate(params, n_ims, first_set_id, out)
        return out

    def hess(self, n_sets: int, n_ims: Sequence[int], pixels: bool = False):
        t = self.torch
        h = t.zeros((n_sets, self.w.hess_ny, self.w.hess_nx), dtype=t.int32, device="cuda")
        m = t.zeros((n_sets, 3), dtype=t.float64, device="cuda")
        c = t.zeros((n_sets, 2), dtype=t.int32, device="cuda")
        px = None
        if pixels:
            px = t.empty(sum((self.w.n_bands + 2) * n * n for n in n_ims), dtype=t.float32, device="cuda")
        pcmd_hess(self.ctx, _ptr(h), _ptr(m), _ptr(c), _ptr(px))
        return h, m, c, px

    def loglike(self, n_sets: int, mock_hess, mock_moments, mock_n_pix: float, mode: int) -> np.ndarray:
        ll = np.zeros(n_sets)
        mom = np.ascontiguousarray(mock_moments, np.float64)
        pcmd_loglike(self.ctx, _ptr(mock_hess), mom, float(mock_n_pix), mode, ll)
        return ll

    def evaluate(self, params, n_ims, mock_hess, mock_moments, mock_n_pix, mode,
                 first_set_id: int = 0) -> np.ndarray:
        ps = params_array(params)
        ni = (ctypes.c_int * len(n_ims))(*[int(v) for v in n_ims])
        ll = np.zeros(len(params))
        mom = np.ascontiguousarray(mock_moments, np.float64)
        pcmd_evaluate(self.ctx, ps, len(params), ni, first_set_id, _ptr(mock_hess), mom,
                      float(mock_n_pix), mode, ll)
        return ll

    def sync(self):
        pcmd_sync(self.ctx)

    # ---- inspection ----------------------------------------------------------------------
    def tables(self, p: "workloads.Params"):
        P = self.n_points
        lam = np.zeros((2, P), np.float32)
        flux = np.zeros((P, self.w.n_bands), np.float32)
        z0 = np.zeros((2, P), np.uint32)
        pp = make_params(p)
        _check(lib().pcmd_get_tables(self.ctx, ctypes.byref(pp), lam.ctypes.data, flux.ctypes.data,
                                     z0.ctypes.data), "pcmd_get_tables", self.ctx)
        return lam, flux, z0

    def counts(self, p: "workloads.Params", n_im: int, set_id: int, pix_begin: int, n_pix: int):
        t = self.torch
        out = t.zeros((n_pix, 2, self.n_points), dtype=t.int32, device="cuda")
        pp = make_params(p)
        _check(lib().pcmd_counts(self.ctx, ctypes.byref(pp), n_im, set_id, pix_begin, n_pix,
                                 out.data_ptr()), "pcmd_counts", self.ctx)
        return out

    def bin_mags(self, mag, colour, valid):
        t = self.torch
        h = t.zeros((self.w.hess_ny, self.w.hess_nx), dtype=t.int32, device="cuda")
        c = t.zeros(2, dtype=t.int32, device="cuda")
        m = t.zeros(3, dtype=t.float64, device="cuda")
        _check(lib().pcmd_bin_mags(self.ctx, mag.data_ptr(), colour.data_ptr(), valid.data_ptr(),
                                   int(mag.numel()), h.data_ptr(), c.data_ptr(), m.data_ptr()),
               "pcmd_bin_mags", self.ctx)
        return h, c, m
