"""FP64 numpy reference of the surrogate MLP -- test infrastructure only.

Same network as the CUDA surrogate: x -> depth x [Linear -> GELU] -> Linear, GELU in its
exact form 0.5 z (1 + erf(z / sqrt 2)), loss = mean(m (y - t)^2) with optional nonnegative
weights m. Parameters use the CUDA
library's flat layout: for each layer l = 0..depth, W_l [out][in] row-major then b_l [out].
Gradients come from the chain rule written out layer by layer (plain backpropagation).
Pinned in tests by central finite differences of the loss (tests/test_mlp_reference.py).
`grad_magnitudes` gives, per parameter, the sum of the magnitudes of the products its gradient
adds up (the scale of a rounding-error bound); `adamw_step` is one AdamW update (Adam's bias-
corrected moments, Kingma and Ba 2015, with decoupled weight decay, Loshchilov and Hutter 2019).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def layout(n_in, width, depth, n_out):
    """[(w_off, b_off, n_out_l, n_in_l)] per layer and the total parameter count."""
    out, off = [], 0
    for l in range(depth + 1):
        fi = n_in if l == 0 else width
        fo = n_out if l == depth else width
        out.append((off, off + fi * fo, fo, fi))
        off += fi * fo + fo
    return out, off


def unpack(params, n_in, width, depth, n_out):
    lay, _ = layout(n_in, width, depth, n_out)
    p = np.asarray(params, dtype=np.float64)
    return [(p[wo:wo + fo * fi].reshape(fo, fi), p[bo:bo + fo]) for (wo, bo, fo, fi) in lay]


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward(params, x, n_in, width, depth, n_out, keep=False):
    layers = unpack(params, n_in, width, depth, n_out)
    h = np.asarray(x, dtype=np.float64)
    zs, hs = [], [h]
    for (W, b) in layers[:-1]:
        z = h @ W.T + b
        h = gelu(z)
        zs.append(z)
        hs.append(h)
    W, b = layers[-1]
    y = h @ W.T + b
    return (y, zs, hs) if keep else y


def loss_and_grad(params, x, t, n_in, width, depth, n_out, mask=None):
    """(loss, flat gradient) of mean(mask (y - t)^2) over all batch x output elements."""
    layers = unpack(params, n_in, width, depth, n_out)
    y, zs, hs = forward(params, x, n_in, width, depth, n_out, keep=True)
    t = np.asarray(t, dtype=np.float64)
    m = np.ones_like(y) if mask is None else np.asarray(mask, dtype=np.float64)
    n = y.size
    loss = float(np.sum(m * (y - t) ** 2) / n)
    d = 2.0 * m * (y - t) / n
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        grads[l] = (d.T @ hs[l], d.sum(axis=0))
        if l > 0:
            d = (d @ W) * gelu_grad(zs[l - 1])
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for (gW, gb) in grads])
    return loss, flat


def grad_magnitudes(params, x, t, n_in, width, depth, n_out, mask=None):
    """Flat array (the gradient's layout) of sum_b |d_b,o| |h_b,i| for each weight and sum_b |d_b,o|
    for each bias, with the magnitudes |d| of the backpropagated errors (|W|^T |d| times |GELU'|)."""
    layers = unpack(params, n_in, width, depth, n_out)
    y, zs, hs = forward(params, x, n_in, width, depth, n_out, keep=True)
    t = np.asarray(t, dtype=np.float64)
    m = np.ones_like(y) if mask is None else np.asarray(mask, dtype=np.float64)
    d = np.abs(2.0 * m * (y - t) / y.size)
    mags = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        mags[l] = (d.T @ np.abs(hs[l]), d.sum(axis=0))
        if l > 0:
            d = (d @ np.abs(W)) * np.abs(gelu_grad(zs[l - 1]))
    return np.concatenate([np.concatenate([a.ravel(), b]) for (a, b) in mags])


def adamw_step(p, g, m, v, step, lr, beta1, beta2, eps, weight_decay):
    """(p, m, v) after AdamW step number `step` (1, 2, ...): moments m = beta1 m + (1 - beta1) g,
    v = beta2 v + (1 - beta2) g^2, bias-corrected by 1 - beta^step, then
    p - lr (m_hat / (sqrt(v_hat) + eps) + weight_decay p)."""
    p, g, m, v = (np.asarray(a, dtype=np.float64) for a in (p, g, m, v))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * (mh / (np.sqrt(vh) + eps) + weight_decay * p), m, v
