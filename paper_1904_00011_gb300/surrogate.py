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
    L.pcmd_mlp_loglike.argtypes = [vp, i, vp, d, dp]
    L.pcmd_mlp_get_layer.argtypes = [vp, i, vp, vp, vp, vp]
    L.pcmd_mlp_set_layer.argtypes = [vp, i, vp, vp]
    for n in ["pcmd_mlp_create", "pcmd_mlp_forward", "pcmd_mlp_targets", "pcmd_mlp_set_targets",
              "pcmd_mlp_train_step", "pcmd_mlp_loss", "pcmd_mlp_loglike", "pcmd_mlp_get_layer",
              "pcmd_mlp_set_layer"]:
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

    def loglike(self, B: int, d_data_hess, ratio: float) -> np.ndarray:
        out = np.zeros(B)
        self._chk(self.L.pcmd_mlp_loglike(self.h, B, d_data_hess.data_ptr(), float(ratio),
                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                  "pcmd_mlp_loglike")
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
