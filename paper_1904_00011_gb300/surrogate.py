"""Learned surrogate of the pCMD forward model (binding of include/pcmd_mlp.h).

``Mlp`` wraps the library's network object: every forward and backward product is the library's
tcgen05 BF16 GEMM, training is its own Adam kernel.  ``Surrogate`` trains such a network on
Hess diagrams the exact simulator produces (targets ln(1 + m)) and scores parameter points with
the predicted diagrams; the exact simulator stays the judge (``sampler.py``).

The network maps the 12 free parameters of the full model (7 log SFH bins, mean and width of
the [Fe/H] distribution, dust median and width, distance modulus; Table 1) to the 100 x 100 log
Hess diagram of a 64 x 64 image (Section 2.5).
"""
from __future__ import annotations

import ctypes
import time
from typing import Optional, Sequence

import numpy as np

from . import _check, _ptr, lib, workloads

HIDDEN = 1024
N_HIDDEN = 4


def _setup_types():
    L = lib()
    if getattr(L, "_mlp_types", False):
        return L
    vp, i, d, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
    ip = ctypes.POINTER(ctypes.c_int)
    fp = ctypes.POINTER(ctypes.c_float)
    dp = ctypes.POINTER(ctypes.c_double)
    L.pcmd_mlp_create.argtypes = [ip, i, i, fp, fp, i, u64, vp, ctypes.POINTER(vp)]
    L.pcmd_mlp_destroy.argtypes = [vp]
    L.pcmd_mlp_destroy.restype = None
    L.pcmd_mlp_last_error.argtypes = [vp]
    L.pcmd_mlp_last_error.restype = ctypes.c_char_p
    L.pcmd_mlp_forward.argtypes = [vp, vp, i, i, vp]
    L.pcmd_mlp_output.argtypes = [vp]
    L.pcmd_mlp_output.restype = ctypes.c_void_p
    L.pcmd_mlp_targets.argtypes = [vp, vp, i]
    L.pcmd_mlp_set_targets.argtypes = [vp, vp, i]
    L.pcmd_mlp_train_step.argtypes = [vp, vp, i, i, ctypes.c_float, i]
    L.pcmd_mlp_loss.argtypes = [vp, dp]
    L.pcmd_mlp_loglike.argtypes = [vp, i, vp, d, d, dp]
    L.pcmd_mlp_forward_loglike.argtypes = [vp, vp, i, i, vp, d, d, dp]
    L.pcmd_mlp_get_layer.argtypes = [vp, i, vp, vp, vp, vp]
    L.pcmd_mlp_set_loss.argtypes = [vp, i]
    L.pcmd_mlp_set_layer.argtypes = [vp, i, vp, vp]
    for n in ["pcmd_mlp_create", "pcmd_mlp_forward", "pcmd_mlp_targets", "pcmd_mlp_set_targets",
              "pcmd_mlp_train_step", "pcmd_mlp_loss", "pcmd_mlp_loglike", "pcmd_mlp_get_layer",
              "pcmd_mlp_set_layer", "pcmd_mlp_set_loss", "pcmd_mlp_forward_loglike"]:
        getattr(L, n).restype = ctypes.c_int
    L._mlp_types = True
    return L


class Mlp:
    """One network object of the library (device-resident weights, Adam state, activations)."""

    def __init__(self, dims: Sequence[int], n_in: int, in_lo, in_hi, max_batch: int, seed: int = 0,
                 stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the surrogate needs a CUDA device (no CPU fallback)")
        self.torch = torch
        L = _setup_types()
        self.dims = [int(v) for v in dims]
        self.n_layers = len(self.dims) - 1
        self.n_in = n_in
        self.max_batch = max_batch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        d = (ctypes.c_int * len(self.dims))(*self.dims)
        lo = (ctypes.c_float * n_in)(*[float(v) for v in in_lo])
        hi = (ctypes.c_float * n_in)(*[float(v) for v in in_hi])
        self.h = ctypes.c_void_p()
        _check(L.pcmd_mlp_create(d, self.n_layers, n_in, lo, hi, max_batch, seed,
                                 ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.h)),
               "pcmd_mlp_create")
        self.L = L

    def close(self):
        if getattr(self, "h", None):
            self.L.pcmd_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc, where):
        if rc:
            from . import PcmdError
            raise PcmdError(rc, where, self.L.pcmd_mlp_last_error(self.h).decode(errors="replace"))

    def _theta(self, theta):
        t = self.torch
        if isinstance(theta, t.Tensor):
            theta = theta.to(device="cuda", dtype=t.float32).contiguous()
            return theta, 1, theta
        arr = np.ascontiguousarray(theta, np.float32)
        return arr, 0, arr.ctypes.data

    def forward(self, theta, out=None):
        keep, on_dev, ptr = self._theta(theta)
        B = keep.shape[0]
        self._chk(self.L.pcmd_mlp_forward(self.h, ptr if not on_dev else ptr.data_ptr(), on_dev, B,
                                          _ptr(out)), "pcmd_mlp_forward")
        return out

    def predict(self, theta):
        """Forward pass into a new CUDA tensor [B][d_out]."""
        t = self.torch
        B = len(theta)
        out = t.empty((B, self.dims[-1]), dtype=t.float32, device="cuda")
        self.forward(theta, out)
        return out

    def set_loss(self, poisson: bool):
        self._chk(self.L.pcmd_mlp_set_loss(self.h, int(bool(poisson))), "pcmd_mlp_set_loss")
        self.poisson = bool(poisson)

    def targets_from_hess(self, d_hess, B: int):
        self._chk(self.L.pcmd_mlp_targets(self.h, d_hess.data_ptr(), B), "pcmd_mlp_targets")

    def set_targets(self, y, B: int):
        self._chk(self.L.pcmd_mlp_set_targets(self.h, y.data_ptr(), B), "pcmd_mlp_set_targets")

    def train_step(self, theta, lr: float, update: bool = True):
        keep, on_dev, ptr = self._theta(theta)
        B = keep.shape[0]
        self._chk(self.L.pcmd_mlp_train_step(self.h, ptr if not on_dev else ptr.data_ptr(), on_dev, B,
                                             float(lr), int(bool(update))), "pcmd_mlp_train_step")

    def loss(self) -> float:
        v = ctypes.c_double(0.0)
        self._chk(self.L.pcmd_mlp_loss(self.h, ctypes.byref(v)), "pcmd_mlp_loss")
        return float(v.value)

    def loglike(self, B: int, d_data_hess, scale: float, ratio: float) -> np.ndarray:
        out = np.zeros(B)
        self._chk(self.L.pcmd_mlp_loglike(self.h, B, d_data_hess.data_ptr(), float(scale), float(ratio),
                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                  "pcmd_mlp_loglike")
        return out

    def forward_loglike(self, theta, d_data_hess, scale: float, ratio: float) -> np.ndarray:
        """Forward pass and likelihood in one call; the predicted diagrams are not written."""
        keep, on_dev, ptr = self._theta(theta)
        B = keep.shape[0]
        out = np.zeros(B)
        self._chk(self.L.pcmd_mlp_forward_loglike(self.h, ptr if not on_dev else ptr.data_ptr(), on_dev, B,
                                                  d_data_hess.data_ptr(), float(scale), float(ratio),
                                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                  "pcmd_mlp_forward_loglike")
        return out

    def get_layer(self, l: int):
        N, K = self.dims[l + 1], self.dims[l]
        w = np.zeros((N, K), np.float32)
        b = np.zeros(N, np.float32)
        gw = np.zeros((N, K), np.float32)
        gb = np.zeros(N, np.float32)
        self._chk(self.L.pcmd_mlp_get_layer(self.h, l, w.ctypes.data, b.ctypes.data, gw.ctypes.data,
                                            gb.ctypes.data), "pcmd_mlp_get_layer")
        return w, b, gw, gb

    def set_layer(self, l: int, w: np.ndarray, b: np.ndarray):
        w = np.ascontiguousarray(w, np.float32)
        b = np.ascontiguousarray(b, np.float32)
        self._chk(self.L.pcmd_mlp_set_layer(self.h, l, w.ctypes.data, b.ctypes.data), "pcmd_mlp_set_layer")


def surrogate_dims(n_out: int = 10000, hidden: int = HIDDEN, n_hidden: int = N_HIDDEN):
    return [64] + [hidden] * n_hidden + [n_out]


class Surrogate:
    """An MLP from the 12 free parameters of the full model to the log Hess diagram of a
    64 x 64 image, trained on diagrams the exact simulator produces on the GPU."""

    def __init__(self, n_im: int = 64, batch: int = 512, seed: int = 0, hidden: int = HIDDEN,
                 n_hidden: int = N_HIDDEN, infer_batch: int = 4096, exact_n_im: int = 256):
        import torch
        from . import Simulator
        self.torch = torch
        self.n_im = n_im
        self.batch = batch
        self.box = workloads.SURROGATE_BOX.copy()
        self.base = workloads.surrogate(n_sets=1, n_im=n_im)
        self.sim = Simulator(self.base, max_sets=batch, max_im=n_im)
        # the judge: the exact simulator on larger images (expected Hess counts scale with the
        # number of pixels, so the network's 64x64 rates are rescaled, not retrained)
        self.exact_n_im = exact_n_im
        self.exact_sim = Simulator(self.base, max_sets=8, max_im=exact_n_im)
        self.nbins = self.base.hess_nx * self.base.hess_ny
        self.net = Mlp(surrogate_dims(self.nbins, hidden, n_hidden), 12, self.box[:, 0],
                       self.box[:, 1], max_batch=max(batch, infer_batch), seed=seed)
        # the output is the log expected count of every bin (Poisson deviance on the counts)
        self.net.set_loss(True)
        self.calib = {"offset": 0.0, "spread": 0.0}
        self.rng = np.random.default_rng(seed + 17)
        self.set_counter = 1 << 24
        self.history = []

    # -- data --------------------------------------------------------------------------------
    def sample_theta(self, n: int, rng: Optional[np.random.Generator] = None) -> np.ndarray:
        rng = rng or self.rng
        u = rng.uniform(size=(n, 12))
        return self.box[:, 0] + u * (self.box[:, 1] - self.box[:, 0])

    def param_matrix(self, theta: np.ndarray) -> np.ndarray:
        """The parameter rows as the library's pcmd_params layout (float64 [n][MAX_SFH + 5]):
        7 log SFH bins (offsets from the constant-SFR history), [Fe/H] mean and width, log
        E(B-V), dust width, distance modulus."""
        from . import PCMD_MAX_SFH
        th = np.asarray(theta, np.float64)
        m = np.zeros((th.shape[0], PCMD_MAX_SFH + 5))
        m[:, :7] = np.asarray(self.base.params[0].log_sfh, np.float64)[None, :] + th[:, :7]
        m[:, PCMD_MAX_SFH:] = th[:, 7:12]
        return m

    def simulate(self, theta: np.ndarray, set_id0: Optional[int] = None):
        """Exact Hess diagrams [n][ny][nx] (int32 CUDA tensor) of the parameter rows."""
        n = len(theta)
        if set_id0 is None:
            set_id0 = self.set_counter
            self.set_counter += n
        self.sim.simulate(self.param_matrix(theta), [self.n_im] * n, set_id0)
        h, m, c, _ = self.sim.hess(n, [self.n_im] * n)
        return h, m

    # -- training -----------------------------------------------------------------------------
    def train(self, n_sims: int, lr: float = 1e-3, lr_min: float = 2e-5, log_every: int = 50):
        """Fresh simulations every step (no sample is seen twice); cosine learning-rate decay."""
        steps = max(1, n_sims // self.batch)
        t0 = time.perf_counter()
        t_sim = 0.0
        for s in range(steps):
            theta = self.sample_theta(self.batch).astype(np.float32)
            ts = time.perf_counter()
            h, _ = self.simulate(theta)
            self.torch.cuda.synchronize()
            t_sim += time.perf_counter() - ts
            if s == 0:
                # start the output layer at the log mean count of every bin
                last = self.net.n_layers - 1
                w, _, _, _ = self.net.get_layer(last)
                mean = h.reshape(self.batch, -1).float().mean(0).cpu().numpy()
                self.net.set_layer(last, w * 0.1, np.log(mean + 1e-2).astype(np.float32))
            self.net.targets_from_hess(h, self.batch)
            a = lr_min + 0.5 * (lr - lr_min) * (1 + np.cos(np.pi * s / steps))
            self.net.train_step(theta, a)
            if s % log_every == 0 or s == steps - 1:
                self.history.append((s, self.net.loss()))
        self.torch.cuda.synchronize()
        return {"steps": steps, "sims": steps * self.batch, "seconds": time.perf_counter() - t0,
                "simulation_seconds": t_sim, "final_loss": self.history[-1][1]}

    # -- inference -----------------------------------------------------------------------------
    def predict(self, theta: np.ndarray):
        """Predicted ln(1 + m) [n][nbins] as a CUDA tensor (n a multiple of 8)."""
        return self.net.predict(np.asarray(theta, np.float32))

    def loglike(self, theta: np.ndarray, d_mock_hess, mock_n_pix: float) -> np.ndarray:
        """Surrogate Poisson log-likelihood of every parameter row against the data diagram, for
        a model image of exact_n_im (the judge's image size)."""
        n = len(theta)
        pad = (-n) % 8
        th = np.asarray(theta, np.float32)
        if pad:
            th = np.concatenate([th, np.repeat(th[-1:], pad, axis=0)])
        scale = float(self.exact_n_im ** 2) / float(self.n_im ** 2)
        ll = self.net.forward_loglike(th, d_mock_hess.reshape(-1), scale,
                                      mock_n_pix / float(self.exact_n_im ** 2))
        return ll[:n]

    def exact_loglike(self, theta: np.ndarray, d_mock_hess, mock_moments, mock_n_pix: float,
                      set_id0: Optional[int] = None) -> np.ndarray:
        """The exact simulator's Poisson log-likelihood (the judge) on exact_n_im images."""
        n = len(theta)
        if set_id0 is None:
            set_id0 = self.set_counter
            self.set_counter += n
        out = np.zeros(n)
        for k in range(0, n, 8):
            th = theta[k:k + 8]
            w = workloads.surrogate_from_theta(th, n_im=self.exact_n_im, base=self.base)
            out[k:k + len(th)] = self.exact_sim.evaluate(
                w.params, [self.exact_n_im] * len(th), d_mock_hess, mock_moments, mock_n_pix,
                workloads.LL_POISSON, first_set_id=set_id0 + k)
        return out

    def exact_mock(self, theta: np.ndarray, set_id: int = 123456789):
        """Data diagram: one exact realisation at theta on an exact_n_im image."""
        w = workloads.surrogate_from_theta(np.atleast_2d(theta), n_im=self.exact_n_im, base=self.base)
        self.exact_sim.simulate(w.params, [self.exact_n_im], set_id)
        h, m, c, _ = self.exact_sim.hess(1, [self.exact_n_im])
        return h[0].contiguous(), m[0].cpu().numpy(), float(self.exact_n_im ** 2)

    def errors(self, n_test: int = 512, seed: int = 99, d_mock=None, mock_moments=None,
               mock_n_pix: float = 0.0):
        """Held-out accuracy: RMS of ln(1 + m) per bin against one exact realisation, the same
        between two exact realisations (the simulator's own noise floor), and, with a mock,
        the log-likelihood difference surrogate - exact."""
        t = self.torch
        rng = np.random.default_rng(seed)
        n_test = max(8, n_test - n_test % 8)
        theta = self.sample_theta(n_test, rng).astype(np.float32)
        pred = self.torch.log1p(self.torch.exp(self.predict(theta)))
        h1, _ = self.simulate(theta, set_id0=7 << 26)
        y1 = t.log1p(h1.reshape(n_test, -1).float())
        h2, _ = self.simulate(theta, set_id0=9 << 26)
        y2 = t.log1p(h2.reshape(n_test, -1).float())
        out = {"n_test": n_test,
               "rms_log_bin": float(((pred - y1) ** 2).mean().sqrt()),
               "rms_log_bin_noise_floor": float(((y2 - y1) ** 2).mean().sqrt() / np.sqrt(2.0))}
        if d_mock is not None:
            ll_s = self.loglike(theta, d_mock, mock_n_pix)
            ll_e = self.exact_loglike(theta, d_mock, mock_moments, mock_n_pix, set_id0=11 << 26)
            d = ll_s - ll_e
            off = float(np.median(ll_e - ll_s))
            spread = float(np.percentile(np.abs(ll_e - ll_s - off), 90))
            self.calib = {"offset": off, "spread": spread}
            out.update({"ll_offset": off, "ll_spread_p90": spread,
                        "ll_abs_err_median": float(np.median(np.abs(d))),
                        "ll_abs_err_p90": float(np.percentile(np.abs(d), 90)),
                        "ll_rel_err_median": float(np.median(np.abs(d) / np.abs(ll_e))),
                        "ll_spearman": float(_spearman(ll_s, ll_e))})
        return out


    def scatter_calibration(self, d_mock, mock_moments, mock_n_pix: float, n_theta: int = 32,
                            n_rep: int = 16, seed: int = 77) -> dict:
        """The surrogate's likelihood error next to the exact simulator's own scatter (Appendix A:
        the likelihood of one parameter point is itself stochastic).  For n_theta held-out points,
        the exact likelihood at n_rep RNG set ids gives a mean and a standard deviation; the
        surrogate's likelihood plus the held-out offset is compared with that mean.  Returns the
        median over points of |surrogate + offset - exact mean| / exact scatter, and the parts."""
        rng = np.random.default_rng(seed)
        theta = self.sample_theta(n_theta, rng).astype(np.float32)
        reps = np.repeat(theta, n_rep, axis=0)
        ll = self.exact_loglike(reps, d_mock, mock_moments, mock_n_pix, set_id0=13 << 26)
        ll = ll.reshape(n_theta, n_rep)
        mean, sd = ll.mean(axis=1), ll.std(axis=1, ddof=1)
        sur = self.loglike(theta, d_mock, mock_n_pix) + self.calib["offset"]
        err = np.abs(sur - mean)
        ratio = err / np.maximum(sd, 1e-12)
        return {"n_theta": n_theta, "n_rep": n_rep,
                "ll_err_over_exact_scatter": float(np.median(ratio)),
                "ll_err_over_exact_scatter_p90": float(np.percentile(ratio, 90)),
                "surrogate_abs_err_median": float(np.median(err)),
                "exact_scatter_median": float(np.median(sd)),
                "exact_ll_median": float(np.median(mean))}


def _spearman(a, b):
    ra = np.argsort(np.argsort(a))
    rb = np.argsort(np.argsort(b))
    return np.corrcoef(ra, rb)[0, 1]
