"""FP64 CPU reference of the surrogate MLP (forward, masked-MSE loss, backward).

TEST INFRASTRUCTURE: it checks the gradients of the GPU training kernels.  Plain numpy in
float64; the architecture follows the library's surrogate: layers W_l [out][in], b_l, GELU
(its tanh form, x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))) after every layer but the
last, loss = mean over non-NaN targets of
(y - t)^2.  Parameters use the library's flat layout: for each layer W (row-major) then b.

``quantize`` (optional, e.g. ``bf16_round``) is applied where the GPU stores a value in a
narrower type before its next use: every hidden activation GELU(z), the loss gradient
2 (y - t) / count and each back-propagated dZ = dA * GELU'(z).  The arithmetic between
those points stays FP64, so with the same inputs the two sides take the same rounding
decisions (up to values within FP32 rounding of a BF16 tie) and their gradients can be
compared element by element.
"""
from __future__ import annotations

import math

import numpy as np

GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def gelu(x):
    """GELU, tanh form: x/2 (1 + tanh(y)), y = sqrt(2/pi) (x + 0.044715 x^3)."""
    return 0.5 * x * (1.0 + np.tanh(GELU_C * (x + GELU_A * x ** 3)))


def gelu_grad(x):
    """d/dx of gelu: (1 + t)/2 + x (1 - t^2) sqrt(2/pi) (1 + 3 * 0.044715 x^2) / 2."""
    t = np.tanh(GELU_C * (x + GELU_A * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * x * x)


def unflatten(flat, dims):
    """dims = [in, h1, ..., out]; returns [(W, b), ...] views into float64 copies."""
    flat = np.asarray(flat, dtype=np.float64)
    out, k = [], 0
    for i in range(len(dims) - 1):
        n_in, n_out = dims[i], dims[i + 1]
        W = flat[k:k + n_in * n_out].reshape(n_out, n_in)
        k += n_in * n_out
        b = flat[k:k + n_out]
        k += n_out
        out.append((W, b))
    assert k == flat.size
    return out


def flatten(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64.  Values are first
    rounded to float32, as the GPU holds them."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _ident(a):
    return a


def forward(layers, x, quantize=None):
    q = quantize or _ident
    a, zs, acts = np.asarray(x, np.float64), [], []
    for i, (W, b) in enumerate(layers):
        acts.append(a)
        z = a @ W.T + b
        zs.append(z)
        a = q(gelu(z)) if i + 1 < len(layers) else z
    return a, zs, acts


def loss(layers, x, t):
    y, _, _ = forward(layers, x)
    m = ~np.isnan(t)
    d = np.where(m, y - np.nan_to_num(t), 0.0)
    return float(np.sum(d * d) / max(1, m.sum()))


def loss_and_grad(layers, x, t, quantize=None):
    """Masked mean squared error and its gradient (same flat layout as the parameters)."""
    q = quantize or _ident
    y, zs, acts = forward(layers, x, quantize)
    m = ~np.isnan(t)
    cnt = max(1, int(m.sum()))
    d = np.where(m, y - np.nan_to_num(t), 0.0)
    L = float(np.sum(d * d) / cnt)
    g = q(2.0 * d / cnt)
    grads = [None] * len(layers)
    for i in range(len(layers) - 1, -1, -1):
        W, _ = layers[i]
        grads[i] = (g.T @ acts[i], g.sum(axis=0))
        if i > 0:
            g = q((g @ W) * gelu_grad(zs[i - 1]))
    return L, flatten(grads)


def gradient_scale(layers, x, t, quantize=None):
    """For every gradient element, the sum of the absolute values of the terms that make it:
    the backward pass of loss_and_grad run on |.| of every factor (|2 (y - t)| / count, |W|,
    |GELU'(z)|, |activations|).  It bounds |gradient| elementwise (triangle inequality) and is
    the scale against which rounding differences of the terms are measured."""
    q = quantize or _ident
    y, zs, acts = forward(layers, x, quantize)
    m = ~np.isnan(t)
    cnt = max(1, int(m.sum()))
    d = np.where(m, y - np.nan_to_num(t), 0.0)
    g = np.abs(q(2.0 * d / cnt))
    out = [None] * len(layers)
    for i in range(len(layers) - 1, -1, -1):
        W, _ = layers[i]
        out[i] = (g.T @ np.abs(acts[i]), g.sum(axis=0))
        if i > 0:
            g = (g @ np.abs(W)) * np.abs(gelu_grad(zs[i - 1]))
    return flatten(out)
