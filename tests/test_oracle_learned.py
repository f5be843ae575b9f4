"""Pins of the learned-guess reference (``oracle/learned.py``), CPU only:
the convolution against scipy's correlation, adjoint identities of the
pooling and upsampling, analytic gradients against central finite
differences through the whole encoder-decoder, and Adam's first step."""
import numpy as np
import pytest
from scipy import signal

import oracle.learned as ol


def test_conv_matches_scipy_correlation():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 9, 13))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = ol.conv3x3(x, w, b)
    for o in range(4):
        ref = b[o] + sum(signal.correlate2d(x[i], w[o, i], mode="same", boundary="fill") for i in range(3))
        assert np.allclose(y[o], ref, atol=1e-12)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 8, 6))
    z = rng.normal(size=(2, 4, 3))
    assert np.isclose(np.sum(ol.pool2(x) * z), np.sum(x * ol.pool2_backward(z)))
    assert np.isclose(np.sum(ol.up2(z) * x), np.sum(z * ol.up2_backward(x)))
    # nearest upsampling then pooling is the identity
    assert np.allclose(ol.pool2(ol.up2(z)), z)


def test_conv_backward_by_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 5, 6))
    w = rng.normal(size=(3, 2, 3, 3))
    b = rng.normal(size=3)
    t = rng.normal(size=(3, 5, 6))
    loss = lambda x_, w_, b_: 0.5 * np.sum((ol.conv3x3(x_, w_, b_) - t) ** 2)
    dy = ol.conv3x3(x, w, b) - t
    dx, dw, db = ol.conv3x3_backward(x, w, dy)
    e = 1e-6
    for arr, grad in ((x, dx), (w, dw), (b, db)):
        for idx in list(np.ndindex(arr.shape))[::5]:
            old = arr[idx]
            arr[idx] = old + e
            lp = loss(x, w, b)
            arr[idx] = old - e
            lm = loss(x, w, b)
            arr[idx] = old
            assert abs((lp - lm) / (2 * e) - grad[idx]) <= 1e-6 * max(1.0, abs(grad[idx]))


def test_network_gradients_by_finite_differences():
    widths = (2, 3, 4, 5)
    p = ol.init_params(2, 3, widths, seed=3)
    rng = np.random.default_rng(4)
    for k in p:  # nonzero biases exercise the bias gradients and the ReLU masks
        p[k] = p[k] + 0.05 * rng.normal(size=p[k].shape)
    x = rng.normal(size=(2, 16, 16))
    t = rng.normal(size=(3, 16, 16))
    y, cache = ol.forward(p, x)
    assert y.shape == (3, 16, 16)
    g = ol.backward(p, cache, y, t)
    assert set(g) == set(p)
    e = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        gf = g[k].reshape(-1)
        for q in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[q]
            flat[q] = old + e
            lp = ol.mse(ol.forward(p, x)[0], t)
            flat[q] = old - e
            lm = ol.mse(ol.forward(p, x)[0], t)
            flat[q] = old
            fd = (lp - lm) / (2 * e)
            assert abs(fd - gf[q]) <= 1e-5 * max(1e-3, abs(gf[q])), (k, q, fd, gf[q])


def test_adam_first_step_and_training_reduces_the_loss():
    # first step: m_hat = g and v_hat = g^2, so every parameter moves by lr * sign(g)
    p = {"a": np.array([1.0, -2.0, 0.5])}
    g = {"a": np.array([0.3, -4.0, 1e-3])}
    ol.adam_step(p, g, {}, lr=0.01)
    assert np.allclose(p["a"], [1.0 - 0.01, -2.0 + 0.01, 0.5 - 0.01 * 1e-3 / (1e-3 + 1e-8)])
    # a few steps on one tiny example lower the loss
    widths = (2, 3, 4, 5)
    p = ol.init_params(1, 1, widths, seed=5)
    rng = np.random.default_rng(6)
    x = rng.normal(size=(1, 16, 16))
    t = 0.5 * x
    state = {}
    losses = []
    for _ in range(30):
        y, c = ol.forward(p, x)
        losses.append(ol.mse(y, t))
        ol.adam_step(p, ol.backward(p, c, y, t), state, lr=3e-3)
    assert losses[-1] < 0.5 * losses[0]
