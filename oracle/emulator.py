"""Reference MLP of the lnL emulator (oracle; test infrastructure only).

The network (the learned part of the build, not in the paper): normalised
parameters x (padded with zeros to `in0` inputs) pass through `depth` hidden
layers z_l = W_l a_{l-1} + b_l, a_l = gelu(z_l) with gelu(z) = z Phi(z) =
z (1 + erf(z / sqrt 2)) / 2 (Hendrycks & Gimpel 2016), then a linear output
layer whose first component is the prediction.  Loss: mean squared error of
that component.  Gradients by the chain rule, dgelu/dz = Phi(z) + z phi(z).

Parameter layout (shared interface with the library): for each layer l in
order, W_l (out_l x in_l, row-major) then b_l (out_l).  The library stores
weights in bf16 for its tensor-core products and rounds each layer's input
activations to bf16; `forward(..., bf16_inputs=True)` reproduces those two
roundings so that its outputs and gradients are comparable.  In training the
library also rounds the back-propagated errors dL/dz to bf16 where they enter
a tensor-core product (the weight gradient dz^T a and the error of the layer
below, dz W), while the bias gradient sums the unrounded dz;
`loss_and_grad(..., bf16_grads=True)` reproduces that rounding too.
Everything else is float64.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def dims(in0: int, width: int, depth: int, out0: int):
    d = [in0] + [width] * depth + [out0]
    return [(d[i + 1], d[i]) for i in range(len(d) - 1)]


def unpack(params: np.ndarray, in0: int, width: int, depth: int, out0: int):
    layers, off = [], 0
    for (o, i) in dims(in0, width, depth, out0):
        W = params[off:off + o * i].reshape(o, i)
        off += o * i
        b = params[off:off + o]
        off += o
        layers.append((W, b))
    assert off == params.size
    return layers


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (round to nearest even) and back to float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def dgelu(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(params, X, in0, width, depth, out0, bf16_inputs=False):
    """Returns (prediction (B,), cache).  X: (B, in0)."""
    layers = unpack(params, in0, width, depth, out0)
    a = np.asarray(X, dtype=np.float64)
    cache = []
    for li, (W, b) in enumerate(layers):
        Wu = bf16_round(W) if bf16_inputs else W
        au = bf16_round(a) if bf16_inputs else a
        z = au @ Wu.T + b
        cache.append((au, z))
        a = gelu(z) if li < len(layers) - 1 else z
    return a[:, 0], cache


def loss_and_grad(params, X, t, in0, width, depth, out0, bf16_inputs=False, bf16_grads=False):
    """MSE of the first output and its gradient w.r.t. params (float64)."""
    layers = unpack(params, in0, width, depth, out0)
    pred, cache = forward(params, X, in0, width, depth, out0, bf16_inputs)
    B = X.shape[0]
    r = pred - t
    loss = float(np.mean(r * r))
    dz = np.zeros((B, out0))
    dz[:, 0] = 2.0 * r / B
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        au, z = cache[li]
        if li < len(layers) - 1:
            dz = dz * dgelu(z)
        dzu = bf16_round(dz) if bf16_grads else dz
        gW = dzu.T @ au
        gb = dz.sum(axis=0)
        grads.append((gW, gb))
        Wu = bf16_round(W) if bf16_inputs else W
        dz = dzu @ Wu
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat
