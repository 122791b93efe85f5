"""FP64 reference of the convolutional demag surrogate (test infrastructure).

The paper has no learned component; the surrogate is the benchmark's own
addition: a 4-layer CNN, 3 -> 32 -> 32 -> 32 -> 3 channels, 5x5 kernels,
zero "same" padding, ReLU after the first three layers, trained with the
mean-squared error and Adam.  Because the demagnetising field is linear in
m, the network is trained on increments: input dm = m - m_ref (scaled by
c_in), target dH = H_demag(dm) / Ms (scaled by c_in), where H_demag is the
exact FFT convolution.  Convolutions are cross-correlations:

    y[co, i, j] = b[co] + sum_ci sum_{p,q in -2..2} w[co, ci, p+2, q+2] x[ci, i+p, j+q]

Parity status: the operations are pinned (the forward pass against scipy's
correlate2d, the gradients against finite differences of the loss, Adam's
first step and BF16 rounding by their definitions).  A trained network's
predictions have no closed form: their error is measured against the exact
demagnetising field, not held to a parity bar.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (3, 32, 32, 32, 3)
KS = 5
PAD = KS // 2


def init_params(seed: int = 0, channels=CHANNELS):
    """He-style initial weights, zero biases."""
    rng = np.random.default_rng(seed)
    params = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        std = np.sqrt(2.0 / (cin * KS * KS))
        params.append({"w": rng.normal(0.0, std, size=(cout, cin, KS, KS)), "b": np.zeros(cout)})
    return params


def conv2d(x, w, b):
    """x (B, Cin, H, W) -> (B, Cout, H, W), zero padding PAD."""
    B, Cin, H, W = x.shape
    xp = np.zeros((B, Cin, H + 2 * PAD, W + 2 * PAD))
    xp[:, :, PAD:PAD + H, PAD:PAD + W] = x
    y = np.zeros((B, w.shape[0], H, W))
    for p in range(KS):
        for q in range(KS):
            y += np.einsum("oc,bchw->bohw", w[:, :, p, q], xp[:, :, p:p + H, q:q + W])
    return y + b[None, :, None, None]


def conv2d_backward(x, w, dy):
    """Gradients of conv2d: (dx, dw, db)."""
    B, Cin, H, W = x.shape
    xp = np.zeros((B, Cin, H + 2 * PAD, W + 2 * PAD))
    xp[:, :, PAD:PAD + H, PAD:PAD + W] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for p in range(KS):
        for q in range(KS):
            dw[:, :, p, q] = np.einsum("bohw,bchw->oc", dy, xp[:, :, p:p + H, q:q + W])
            dxp[:, :, p:p + H, q:q + W] += np.einsum("oc,bohw->bchw", w[:, :, p, q], dy)
    db = dy.sum(axis=(0, 2, 3))
    return dxp[:, :, PAD:PAD + H, PAD:PAD + W], dw, db


def forward(params, x):
    """Returns the output and the per-layer inputs/pre-activations."""
    cache = []
    h = x
    n = len(params)
    for li, P in enumerate(params):
        z = conv2d(h, P["w"], P["b"])
        cache.append((h, z))
        h = np.maximum(z, 0.0) if li < n - 1 else z
    return h, cache


def mse(y, t):
    """L = mean((y - t)^2) over every element; returns (L, dL/dy)."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(params, cache, dy):
    grads = [None] * len(params)
    g = dy
    n = len(params)
    for li in range(n - 1, -1, -1):
        h, z = cache[li]
        if li < n - 1:
            g = g * (z > 0)
        dx, dw, db = conv2d_backward(h, params[li]["w"], g)
        grads[li] = {"w": dw, "b": db}
        g = dx
    return grads, g


def adam_init(params):
    return {"t": 0, "m": [{k: np.zeros_like(v) for k, v in P.items()} for P in params],
            "v": [{k: np.zeros_like(v) for k, v in P.items()} for P in params]}


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """Kingma & Ba (2015) with bias correction."""
    state["t"] += 1
    t = state["t"]
    for P, G, M, V in zip(params, grads, state["m"], state["v"]):
        for k in P:
            M[k] = b1 * M[k] + (1 - b1) * G[k]
            V[k] = b2 * V[k] + (1 - b2) * G[k] * G[k]
            mh = M[k] / (1 - b1 ** t)
            vh = V[k] / (1 - b2 ** t)
            P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
