"""FP64 reference of the learned initial guess -- TEST INFRASTRUCTURE ONLY
(same rules as the rest of ``oracle``).

A small convolutional encoder-decoder that maps a tile of I0 to a guess of
the solver's correction (I1 - I0 for AD, I2 - I0 for SP), to be used as the
solver's starting point; the multigrid solve still judges the residual.  The
paper has no such component; this module fixes what the network computes so
that GPU kernels for it can be checked element by element.

Layout: activations are ``[C][H][W]`` (one 2D tile; the slices of a z-tile
are channels), 3x3 convolutions with zero padding 1 and stride 1,
``y[o] = b[o] + sum_i sum_{dy,dx} w[o, i, dy, dx] x[i, y + dy - 1, x + dx - 1]``
(cross-correlation, as the GPU implicit-GEMM form computes it).

Network (``widths`` = (c1, c2, c3, c4), 16-32-64-128 by default):

  e1 = relu(conv(x,            c_in -> c1))           full size
  e2 = relu(conv(pool(e1),     c1 -> c2))              1/2
  e3 = relu(conv(pool(e2),     c2 -> c3))              1/4
  e4 = relu(conv(pool(e3),     c3 -> c4))              1/8
  d3 = relu(conv([up(e4), e3], c4 + c3 -> c3))         1/4
  d2 = relu(conv([up(d3), e2], c3 + c2 -> c2))         1/2
  d1 = relu(conv([up(d2), e1], c2 + c1 -> c1))         full
  y  =      conv(d1,           c1 -> c_out)            full

pool: 2x2 average; up: 2x nearest; [a, b]: channel concatenation.  Loss:
mean squared error.  The optimiser is Adam (Kingma & Ba 2015) with bias
correction.  Every function is plain numpy in FP64, written for reading, not
speed.
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------------------
# layers
# ---------------------------------------------------------------------------
def conv3x3(x, w, b):
    """x [Ci][H][W], w [Co][Ci][3][3], b [Co] -> [Co][H][W] (zero padding 1)."""
    ci, h, wd = x.shape
    co = w.shape[0]
    xp = np.zeros((ci, h + 2, wd + 2))
    xp[:, 1:-1, 1:-1] = x
    y = np.empty((co, h, wd))
    y[:] = b[:, None, None]
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, dy:dy + h, dx:dx + wd]  # [Ci][H][W]
            y += np.einsum("oi,ihw->ohw", w[:, :, dy, dx], patch)
    return y


def conv3x3_backward(x, w, dy):
    """Gradients of conv3x3 given dL/dy: (dx, dw, db)."""
    ci, h, wd = x.shape
    xp = np.zeros((ci, h + 2, wd + 2))
    xp[:, 1:-1, 1:-1] = x
    dw = np.empty_like(w)
    dxp = np.zeros_like(xp)
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, ky:ky + h, kx:kx + wd]
            dw[:, :, ky, kx] = np.einsum("ohw,ihw->oi", dy, patch)
            dxp[:, ky:ky + h, kx:kx + wd] += np.einsum("oi,ohw->ihw", w[:, :, ky, kx], dy)
    db = dy.sum(axis=(1, 2))
    return dxp[:, 1:-1, 1:-1], dw, db


def relu(x):
    return np.maximum(x, 0.0)


def relu_backward(x, dy):
    return dy * (x > 0.0)


def pool2(x):
    """2x2 average pooling (H, W even)."""
    c, h, w = x.shape
    return x.reshape(c, h // 2, 2, w // 2, 2).mean(axis=(2, 4))


def pool2_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) * 0.25


def up2(x):
    """2x nearest-neighbour upsampling."""
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_backward(dy):
    c, h, w = dy.shape
    return dy.reshape(c, h // 2, 2, w // 2, 2).sum(axis=(2, 4))


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------
LAYERS = ("e1", "e2", "e3", "e4", "d3", "d2", "d1", "y")


def layer_shapes(c_in, c_out, widths=(16, 32, 64, 128)):
    c1, c2, c3, c4 = widths
    return {"e1": (c1, c_in), "e2": (c2, c1), "e3": (c3, c2), "e4": (c4, c3),
            "d3": (c3, c4 + c3), "d2": (c2, c3 + c2), "d1": (c1, c2 + c1), "y": (c_out, c1)}


def init_params(c_in, c_out, widths=(16, 32, 64, 128), seed=0):
    """He-normal weights (std sqrt(2 / (9 Ci))), zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, (co, ci) in layer_shapes(c_in, c_out, widths).items():
        p[name + ".w"] = rng.normal(0.0, np.sqrt(2.0 / (9.0 * ci)), (co, ci, 3, 3))
        p[name + ".b"] = np.zeros(co)
    return p


def forward(p, x):
    """Returns (y, cache); x [C_in][H][W] with H, W multiples of 8."""
    c = {"x": x}
    c["a1"] = conv3x3(x, p["e1.w"], p["e1.b"]); c["e1"] = relu(c["a1"])
    c["p1"] = pool2(c["e1"])
    c["a2"] = conv3x3(c["p1"], p["e2.w"], p["e2.b"]); c["e2"] = relu(c["a2"])
    c["p2"] = pool2(c["e2"])
    c["a3"] = conv3x3(c["p2"], p["e3.w"], p["e3.b"]); c["e3"] = relu(c["a3"])
    c["p3"] = pool2(c["e3"])
    c["a4"] = conv3x3(c["p3"], p["e4.w"], p["e4.b"]); c["e4"] = relu(c["a4"])
    c["k3"] = np.concatenate([up2(c["e4"]), c["e3"]])
    c["b3"] = conv3x3(c["k3"], p["d3.w"], p["d3.b"]); c["d3"] = relu(c["b3"])
    c["k2"] = np.concatenate([up2(c["d3"]), c["e2"]])
    c["b2"] = conv3x3(c["k2"], p["d2.w"], p["d2.b"]); c["d2"] = relu(c["b2"])
    c["k1"] = np.concatenate([up2(c["d2"]), c["e1"]])
    c["b1"] = conv3x3(c["k1"], p["d1.w"], p["d1.b"]); c["d1"] = relu(c["b1"])
    y = conv3x3(c["d1"], p["y.w"], p["y.b"])
    return y, c


def mse(y, t):
    return float(np.mean((y - t) ** 2))


def backward(p, c, y, t):
    """Gradients of mse(y, t) with respect to every parameter."""
    g = {}
    dy = 2.0 * (y - t) / y.size
    dd1, g["y.w"], g["y.b"] = conv3x3_backward(c["d1"], p["y.w"], dy)
    dk1, g["d1.w"], g["d1.b"] = conv3x3_backward(c["k1"], p["d1.w"], relu_backward(c["b1"], dd1))
    n2 = c["d2"].shape[0]
    dd2, de1_skip = up2_backward(dk1[:n2]), dk1[n2:]
    dk2, g["d2.w"], g["d2.b"] = conv3x3_backward(c["k2"], p["d2.w"], relu_backward(c["b2"], dd2))
    n3 = c["d3"].shape[0]
    dd3, de2_skip = up2_backward(dk2[:n3]), dk2[n3:]
    dk3, g["d3.w"], g["d3.b"] = conv3x3_backward(c["k3"], p["d3.w"], relu_backward(c["b3"], dd3))
    n4 = c["e4"].shape[0]
    de4, de3_skip = up2_backward(dk3[:n4]), dk3[n4:]
    dp3, g["e4.w"], g["e4.b"] = conv3x3_backward(c["p3"], p["e4.w"], relu_backward(c["a4"], de4))
    de3 = pool2_backward(dp3) + de3_skip
    dp2, g["e3.w"], g["e3.b"] = conv3x3_backward(c["p2"], p["e3.w"], relu_backward(c["a3"], de3))
    de2 = pool2_backward(dp2) + de2_skip
    dp1, g["e2.w"], g["e2.b"] = conv3x3_backward(c["p1"], p["e2.w"], relu_backward(c["a2"], de2))
    de1 = pool2_backward(dp1) + de1_skip
    _, g["e1.w"], g["e1.b"] = conv3x3_backward(c["x"], p["e1.w"], relu_backward(c["a1"], de1))
    return g


def adam_step(p, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update in place; state holds m, v and the step count."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m." + k, np.zeros_like(p[k]))
        v = state.setdefault("v." + k, np.zeros_like(p[k]))
        m *= b1
        m += (1.0 - b1) * g[k]
        v *= b2
        v += (1.0 - b2) * g[k] * g[k]
        mh = m / (1.0 - b1 ** t)
        vh = v / (1.0 - b2 ** t)
        p[k] -= lr * mh / (np.sqrt(vh) + eps)
    return p
