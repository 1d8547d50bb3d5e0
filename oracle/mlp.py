"""FP64 reference of the surrogate network -- test infrastructure only.

A plain numpy restatement of the multilayer perceptron the library trains: hidden layers
z = x W^T + b followed by the exact GELU 0.5 z (1 + erf(z / sqrt 2)), a linear output layer,
loss sum((yhat - y)^2) / (2 B), gradients by the chain rule, Adam with bias correction.  Pinned by
finite differences (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np
from scipy.special import erf


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def normalise(theta, lo, hi, width):
    """Inputs as the library packs them: 2 (theta - lo) / (hi - lo) - 1, zero-padded to width."""
    theta = np.asarray(theta, np.float64)
    x = np.zeros((theta.shape[0], width))
    x[:, :theta.shape[1]] = 2.0 * (theta - lo) / (hi - lo) - 1.0
    return x


def forward(Ws: List[np.ndarray], bs: List[np.ndarray], x: np.ndarray):
    """Returns (yhat, zs, xs): pre-activations and layer inputs."""
    xs, zs = [x], []
    a = x
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = a @ W.T + b
        zs.append(z)
        if l < len(Ws) - 1:
            a = gelu(z)
            xs.append(a)
        else:
            a = z
    return a, zs, xs


def loss_and_grads(Ws, bs, x, y, poisson: bool = False) -> Tuple[float, list, list]:
    """Squared error sum((yhat - y)^2) / (2B), or with poisson the deviance of a log-rate output
    against counts y: sum(exp(yhat) - y yhat) / B."""
    B = x.shape[0]
    yhat, zs, xs = forward(Ws, bs, x)
    if poisson:
        r = np.exp(yhat)
        loss = float(np.sum(r - y * yhat)) / B
        dz = (r - y) / B
    else:
        d = yhat - y
        loss = 0.5 * float(np.sum(d * d)) / B
        dz = d / B
    gW, gb = [None] * len(Ws), [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        gW[l] = dz.T @ xs[l]
        gb[l] = dz.sum(axis=0)
        if l > 0:
            da = dz @ Ws[l]
            dz = da * gelu_grad(zs[l - 1])
    return loss, gW, gb


def adam(w, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def surrogate_loglike(yhat, data, scale: float, ratio: float, poisson: bool = True) -> np.ndarray:
    """Poisson log-likelihood of each predicted diagram (Section 2.5's alternative likelihood),
    FP64: rate = exp(y) (log-rate output) or expm1(y) (ln(1 + m) output), mh = max(rate * scale,
    1/2) * ratio, sum over bins of d ln mh - mh - ln Gamma(d + 1)."""
    y = np.asarray(yhat, np.float64)
    d = np.asarray(data, np.float64).reshape(-1)
    rate = np.exp(y) if poisson else np.expm1(y)
    mh = np.maximum(rate * scale, 0.5) * ratio
    lg = np.array([math.lgamma(v + 1.0) for v in d])
    return (d * np.log(mh) - mh).sum(axis=-1) - lg.sum()
