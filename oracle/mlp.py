"""FP64 numpy reference of the refinement-proposal network (test infrastructure).

Same architecture and parameter layout as the CUDA library's network
(32 -> 256 -> 256 -> 256 -> 256 -> 256, GELU after the four hidden layers,
parameters per layer l: W_l [K_l][256] row-major then b_l [256]), written
independently in plain numpy: forward pass, mean-squared-error loss and its
gradient by reverse-mode differentiation.  Pinned by central finite
differences in the CPU tests; the GPU BF16 gradients are compared with it.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

IN, HID, LAYERS = 32, 256, 5


def layer_shapes():
    return [(IN if l == 0 else HID, HID) for l in range(LAYERS)]


def param_count() -> int:
    return sum(k * n + n for k, n in layer_shapes())


def unpack(p):
    out, o = [], 0
    for k, n in layer_shapes():
        W = p[o:o + k * n].reshape(k, n)
        o += k * n
        b = p[o:o + n]
        o += n
        out.append((W, b))
    return out


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


def forward(p, x):
    """Returns the output [M][256] and the per-layer (input, pre-activation) cache."""
    h = np.asarray(x, dtype=np.float64)
    cache = []
    layers = unpack(np.asarray(p, dtype=np.float64))
    for l, (W, b) in enumerate(layers):
        a = h @ W + b
        cache.append((h, a))
        h = gelu(a) if l < LAYERS - 1 else a
    return h, cache


def loss_and_grad(p, x, t):
    """Mean over all M x 256 entries of (y - t)^2, and its gradient w.r.t. p."""
    y, cache = forward(p, x)
    t = np.asarray(t, dtype=np.float64)
    n = y.size
    loss = float(np.sum((y - t) ** 2) / n)
    d = 2.0 * (y - t) / n                       # dL/da of the last layer
    layers = unpack(np.asarray(p, dtype=np.float64))
    grads = [None] * LAYERS
    for l in range(LAYERS - 1, -1, -1):
        h_in, a = cache[l]
        if l < LAYERS - 1:
            d = d * gelu_grad(a)
        grads[l] = (h_in.T @ d, d.sum(axis=0))
        d = d @ layers[l][0].T
    g = np.concatenate([np.concatenate([gw.reshape(-1), gb]) for gw, gb in grads])
    return loss, g
