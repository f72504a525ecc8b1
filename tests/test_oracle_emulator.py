"""Pins for the oracle MLP (P15): gradients against central finite
differences in float64, gelu against its textbook values."""
import math

import numpy as np

from oracle import emulator as E


def test_gelu_values():
    # gelu(0) = 0, gelu(x) -> x for large x, gelu(-x) = gelu(x) - x
    assert E.gelu(np.array(0.0)) == 0.0
    assert abs(E.gelu(np.array(8.0)) - 8.0) < 1e-12
    x = np.linspace(-3, 3, 13)
    assert np.allclose(E.gelu(-x), E.gelu(x) - x, atol=1e-14)
    # Phi(1) = 0.841344746...
    assert abs(E.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    h = 1e-6
    assert np.allclose((E.gelu(x + h) - E.gelu(x - h)) / (2 * h), E.dgelu(x), atol=1e-8)


def test_gradient_finite_differences():
    rng = np.random.default_rng(0)
    in0, width, depth, out0 = 16, 12, 3, 16
    n = sum(o * i + o for o, i in E.dims(in0, width, depth, out0))
    p = rng.normal(size=n) * 0.3
    X = np.zeros((7, in0))
    X[:, :4] = rng.uniform(-1, 1, size=(7, 4))
    t = rng.normal(size=7)
    loss, g = E.loss_and_grad(p, X, t, in0, width, depth, out0)
    idx = rng.choice(n, 40, replace=False)
    for j in idx:
        e = np.zeros(n)
        e[j] = 1e-6
        lp, _ = E.loss_and_grad(p + e, X, t, in0, width, depth, out0)
        lm, _ = E.loss_and_grad(p - e, X, t, in0, width, depth, out0)
        fd = (lp - lm) / 2e-6
        assert abs(fd - g[j]) <= 1e-6 * max(1.0, abs(fd)), j


def test_bf16_round():
    assert E.bf16_round(np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8]))[1] == 1.0  # ties to even
    assert E.bf16_round(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    assert E.bf16_round(np.array([255.0]))[0] == 255.0


def test_bf16_error_rounding_option():
    """bf16_grads rounds the back-propagated errors where they enter a product
    (weight gradients, the error of the layer below) and nothing else: the
    output layer's bias gradient (a sum of unrounded errors) is unchanged, and
    every gradient moves by at most a few bf16 roundings (2^-8 relative)."""
    rng = np.random.default_rng(4)
    in0, width, depth, out0 = 16, 32, 3, 16
    dims = E.dims(in0, width, depth, out0)
    n = sum(o * i + o for o, i in dims)
    p = rng.normal(size=n) * 0.3
    X = np.zeros((24, in0))
    X[:, :4] = rng.uniform(-1, 1, size=(24, 4))
    t = rng.normal(size=24)
    _, g0 = E.loss_and_grad(p, X, t, in0, width, depth, out0, bf16_inputs=True)
    _, g1 = E.loss_and_grad(p, X, t, in0, width, depth, out0, bf16_inputs=True, bf16_grads=True)
    o, i = dims[-1]
    gb_last = slice(n - o, n)
    assert np.array_equal(g0[gb_last], g1[gb_last])
    d = np.abs(g1 - g0).max()
    assert 0 < d <= 4 * 2.0 ** -8 * np.abs(g0).max()
