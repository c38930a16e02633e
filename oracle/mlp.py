"""FP64 reference of the warm-start network — test infrastructure.

The paper has no learned component; this network (input r = W^T a, two hidden
layers of width 256 with GELU, softplus output of size K) is an addition
whose definition is fixed here so that the GPU kernels can be checked:

* GELU(x) = x * Phi(x) = 0.5 x (1 + erf(x / sqrt 2))   (exact erf form);
* softplus(x) = log(1 + e^x) for x <= 20, else x;
* loss = mean over batch and outputs of (y - h*)^2;
* Adam (Kingma & Ba 2015) with bias correction:
  m <- b1 m + (1-b1) g;  v <- b2 v + (1-b2) g^2;
  theta <- theta - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Layer l maps x (B x n_in) to x @ Wl + bl with Wl stored n_in x n_out.

``operand_round`` (e.g. bf16.round_bf16) rounds the two operands of every
matrix product (three in the forward pass, six in the backward pass) before
they are multiplied exactly in FP64; biases, activations, their derivatives
and the bias gradients stay unrounded.  This defines the reduced-precision-
product form of the network that the tensor-core kernels compute.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SOFTPLUS_THRESHOLD = 20.0


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def softplus(x):
    out = np.where(x > SOFTPLUS_THRESHOLD, x, np.log1p(np.exp(np.minimum(x, SOFTPLUS_THRESHOLD))))
    return out


def softplus_grad(x):
    return np.where(x > SOFTPLUS_THRESHOLD, 1.0, 1.0 / (1.0 + np.exp(-x)))


def _ident(a):
    return a


def forward(params, x, operand_round=None):
    """params = [W1, b1, W2, b2, W3, b3]; returns (y, cache)."""
    r = operand_round or _ident
    W1, b1, W2, b2, W3, b3 = [np.asarray(p, dtype=np.float64) for p in params]
    x = np.asarray(x, dtype=np.float64)
    z1 = r(x) @ r(W1) + b1
    a1 = gelu(z1)
    z2 = r(a1) @ r(W2) + b2
    a2 = gelu(z2)
    z3 = r(a2) @ r(W3) + b3
    y = softplus(z3)
    return y, (x, z1, a1, z2, a2, z3)


def loss(params, x, target):
    y, _ = forward(params, x)
    return float(np.mean((y - np.asarray(target, dtype=np.float64)) ** 2))


def backward(params, cache, y, target, operand_round=None):
    """Gradients of the mean-squared loss w.r.t. [W1, b1, W2, b2, W3, b3]."""
    r = operand_round or _ident
    W1, b1, W2, b2, W3, b3 = [np.asarray(p, dtype=np.float64) for p in params]
    x, z1, a1, z2, a2, z3 = cache
    n = y.size
    dy = 2.0 * (y - np.asarray(target, dtype=np.float64)) / n
    dz3 = dy * softplus_grad(z3)
    gW3 = r(a2).T @ r(dz3)
    gb3 = dz3.sum(axis=0)
    da2 = r(dz3) @ r(W3).T
    dz2 = da2 * gelu_grad(z2)
    gW2 = r(a1).T @ r(dz2)
    gb2 = dz2.sum(axis=0)
    da1 = r(dz2) @ r(W2).T
    dz1 = da1 * gelu_grad(z1)
    gW1 = r(x).T @ r(dz1)
    gb1 = dz1.sum(axis=0)
    return [gW1, gb1, gW2, gb2, gW3, gb3]


def adam_step(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1).  Returns new (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    for p, g, mi, vi in zip(params, grads, m, v):
        mi = b1 * mi + (1 - b1) * g
        vi = b2 * vi + (1 - b2) * g * g
        mhat = mi / (1 - b1 ** t)
        vhat = vi / (1 - b2 ** t)
        out_p.append(p - lr * mhat / (np.sqrt(vhat) + eps))
        out_m.append(mi)
        out_v.append(vi)
    return out_p, out_m, out_v
