"""FP64 reference of the learned continuous-pole-expansion seed (test infrastructure).

Not in the paper: a multilayer perceptron maps the Matsubara self-energy of one
(k, n) problem to non-negative pole weights on the CPE real-frequency grid, which
warm-start the CPE least-squares fit (Sec. III.B.6). Plain numpy, FP64.

Network (sizes nin -> nh -> ... -> nout):
    h_0 = x,  z_l = W_l h_{l-1} + b_l,  h_l = gelu(z_l) (hidden),  out = softplus(z_L)
    gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2,  softplus(z) = log(1 + e^z)
Input x: [Re s(i w_0..w_63), Im s(i w_0..w_63)] / scale; output: weights b_hat >= 0 so that
the CPE model A b_hat fits x, A = real-stacked Phi_m(i w_n) (the CPE kernel).
Loss (unsupervised, no labels): L = (1/B) sum_b ||A b_hat_b - x_b||^2.
"""
from __future__ import annotations

import math

import numpy as np

_SQRT2 = math.sqrt(2.0)
_INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def _erf(z):
    v = np.vectorize(math.erf, otypes=[float])
    return v(z)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / _SQRT2))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + _erf(z / _SQRT2)) + z * _INV_SQRT_2PI * np.exp(-0.5 * z * z)


def softplus(z):
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(params, x):
    """params: list of (W [out, in], b [out]); x [B, nin]. Returns (out [B, nout], cache)."""
    h = x
    cache = [(None, h)]
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = h @ W.T + b[None, :]
        h = softplus(z) if l == L - 1 else gelu(z)
        cache.append((z, h))
    return h, cache


def loss_and_grad(params, x, A):
    """L = (1/B) sum_b ||A b_hat_b - x_b||^2 and dL/dparams (same structure as params)."""
    B = x.shape[0]
    out, cache = forward(params, x)
    r = out @ A.T - x                     # [B, 2 nw]
    loss = float((r * r).sum() / B)
    d = (2.0 / B) * (r @ A)               # dL/d out  [B, nout]
    grads = [None] * len(params)
    L = len(params)
    for l in range(L - 1, -1, -1):
        z, _ = cache[l + 1]
        hin = cache[l][1]
        dz = d * (sigmoid(z) if l == L - 1 else gelu_grad(z))
        W, _ = params[l]
        grads[l] = (dz.T @ hin, dz.sum(0))
        d = dz @ W
    return loss, grads


def init_params(sizes, rng):
    """He-style normal init for the hidden layers, small output layer."""
    params = []
    for i, (nin, nout) in enumerate(zip(sizes[:-1], sizes[1:])):
        s = math.sqrt(2.0 / nin) if i < len(sizes) - 2 else 0.1 / math.sqrt(nin)
        params.append((rng.standard_normal((nout, nin)) * s, np.zeros(nout)))
    return params
