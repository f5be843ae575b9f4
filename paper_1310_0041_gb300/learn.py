"""Python binding of the learned initial guess (``include/gd_learn.h``).

ctypes marshalling only, with the C names: every convolution, gradient,
optimiser step and tile transform runs in libgd's CUDA kernels.  Activations
are bfloat16 CUDA tensors, channels last ``(tiles, h, w, c)``; parameters and
gradients float32.  There is no CPU fallback: without libgd.so every call
raises.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import GD_OK, GdError, _default_stream, lib

LAYERS = ("e1", "e2", "e3", "e4", "d3", "d2", "d1", "y")


def _p(t, dtype=None):
    """Device pointer of a contiguous CUDA tensor (None passes through);
    `dtype` ("bf16" or "f32") is checked when given."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None:
        import torch
        want = torch.bfloat16 if dtype == "bf16" else torch.float32
        if t.dtype != want:
            raise ValueError("expected a %s tensor, got %s" % (want, t.dtype))
    return ctypes.c_void_p(t.data_ptr())


def _s(stream):
    if stream is None:
        stream = _default_stream()
    return ctypes.c_void_p(stream) if stream else None


def last_error(net=None) -> str:
    return (lib().gd_learn_last_error(net.handle if net is not None else None) or b"").decode()


def _ok(st, what):
    if st != GD_OK:
        raise GdError(st, "%s: %s" % (what, last_error()))
    return st


# ---------------------------------------------------------------------------
# layer-level calls
# ---------------------------------------------------------------------------
def gd_nn_conv3x3(xa, ca, up_a, xb, cb, ntiles, h, w, wt, bias, co, relu, mask=None, y=None,
                  yf=None, stream=None) -> int:
    return lib().gd_nn_conv3x3(_p(xa, "bf16"), ca, up_a, _p(xb, "bf16"), cb, ntiles, h, w,
                               _p(wt, "bf16"), _p(bias, "f32"), co, int(relu), _p(mask, "bf16"),
                               _p(y, "bf16"), _p(yf, "f32"), _s(stream))


def gd_nn_conv3x3_wgrad(xa, ca, up_a, xb, cb, ntiles, h, w, dy, co, dw, stream=None) -> int:
    return lib().gd_nn_conv3x3_wgrad(_p(xa, "bf16"), ca, up_a, _p(xb, "bf16"), cb, ntiles, h, w,
                                     _p(dy, "bf16"), co, _p(dw, "f32"), _s(stream))


def gd_nn_bias_grad(dy, npix, co, db, stream=None) -> int:
    return lib().gd_nn_bias_grad(_p(dy, "bf16"), npix, co, _p(db, "f32"), _s(stream))


def gd_nn_flip_weights(w, co, ci, w16=None, wf16=None, stream=None) -> int:
    return lib().gd_nn_flip_weights(_p(w, "f32"), co, ci, _p(w16, "bf16"), _p(wf16, "bf16"),
                                    _s(stream))


def gd_nn_pool2(x, ntiles, h, w, c, y, stream=None) -> int:
    return lib().gd_nn_pool2(_p(x, "bf16"), ntiles, h, w, c, _p(y, "bf16"), _s(stream))


def gd_nn_pool2_backward(dp, skip, skip_stride, skip_off, mask, ntiles, h, w, c, out,
                         stream=None) -> int:
    return lib().gd_nn_pool2_backward(_p(dp, "bf16"), _p(skip, "bf16"), skip_stride, skip_off,
                                      _p(mask, "bf16"), ntiles, h, w, c, _p(out, "bf16"), _s(stream))


def gd_nn_up2_backward(dk, ck, c, mask, ntiles, h, w, out, stream=None) -> int:
    return lib().gd_nn_up2_backward(_p(dk, "bf16"), ck, c, _p(mask, "bf16"), ntiles, h, w,
                                    _p(out, "bf16"), _s(stream))


def gd_nn_adam(p, g, m, v, lr, b1, b2, eps, t, stream=None) -> int:
    return lib().gd_nn_adam(_p(p, "f32"), _p(g, "f32"), _p(m, "f32"), _p(v, "f32"), p.numel(), lr,
                            b1, b2, eps, t, _s(stream))


def gd_learn_stack_tiles(I, I_sub, nx, ny, nz, th, tw, tc, tile0, ntiles, shift, scale, x=None,
                         xf=None, stream=None) -> int:
    return lib().gd_learn_stack_tiles(_p(I, "f32"), _p(I_sub, "f32"), nx, ny, nz, th, tw, tc, tile0,
                                      ntiles, shift, scale, _p(x, "bf16"), _p(xf, "f32"),
                                      _s(stream))


# ---------------------------------------------------------------------------
# the network
# ---------------------------------------------------------------------------
class Net:
    """Handle of a gd_learn network."""

    def __init__(self, handle, c_in, c_out, widths, tile_h, tile_w, max_batch):
        self.handle = handle
        self.c_in, self.c_out, self.widths = c_in, c_out, tuple(widths)
        self.tile_h, self.tile_w, self.max_batch = tile_h, tile_w, max_batch

    def shapes(self):
        """(co, ci) of every layer, in the flat parameter order."""
        c1, c2, c3, c4 = self.widths
        return [(c1, self.c_in), (c2, c1), (c3, c2), (c4, c3), (c3, c4 + c3), (c2, c3 + c2),
                (c1, c2 + c1), (self.c_out, c1)]


def gd_learn_create(c_in=16, c_out=16, widths=(16, 32, 64, 128), tile_h=256, tile_w=256,
                    max_batch=32, seed=0, stream=None) -> Net:
    h = ctypes.c_void_p()
    W = (ctypes.c_int * 4)(*widths)
    _ok(lib().gd_learn_create(ctypes.byref(h), c_in, c_out, W, tile_h, tile_w, max_batch, seed,
                              _s(stream)), "gd_learn_create")
    return Net(h, c_in, c_out, widths, tile_h, tile_w, max_batch)


def gd_learn_destroy(net: Net) -> int:
    st = lib().gd_learn_destroy(net.handle)
    net.handle = None
    return st


def gd_learn_param_count(net: Net) -> int:
    return int(lib().gd_learn_param_count(net.handle))


def gd_learn_set_params(net: Net, flat: np.ndarray) -> int:
    flat = np.ascontiguousarray(flat, dtype=np.float32)
    assert flat.size == gd_learn_param_count(net)
    return _ok(lib().gd_learn_set_params(net.handle, ctypes.c_void_p(flat.ctypes.data)),
               "gd_learn_set_params")


def gd_learn_get_params(net: Net) -> np.ndarray:
    out = np.empty(gd_learn_param_count(net), np.float32)
    _ok(lib().gd_learn_get_params(net.handle, ctypes.c_void_p(out.ctypes.data)), "gd_learn_get_params")
    return out


def gd_learn_get_grads(net: Net) -> np.ndarray:
    out = np.empty(gd_learn_param_count(net), np.float32)
    _ok(lib().gd_learn_get_grads(net.handle, ctypes.c_void_p(out.ctypes.data)), "gd_learn_get_grads")
    return out


def gd_learn_forward(net: Net, x, batch, yf) -> int:
    return _ok(lib().gd_learn_forward(net.handle, _p(x, "bf16"), batch, _p(yf, "f32")),
               "gd_learn_forward")


def gd_learn_train_step(net: Net, x_pool, t_pool, idx=None, batch=None, lr=1e-3) -> float:
    """One training step; returns the loss before it."""
    if idx is not None:
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        batch = idx.size
        ip = idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    else:
        ip = None
    loss = ctypes.c_double(0.0)
    pool = x_pool.shape[0]
    if t_pool.shape[0] != pool:
        raise ValueError("x_pool and t_pool hold different numbers of tiles")
    st = lib().gd_learn_train_step(net.handle, _p(x_pool, "bf16"), _p(t_pool, "f32"), int(pool), ip,
                                   int(batch), float(lr), ctypes.byref(loss))
    if st != GD_OK:
        raise GdError(st, (lib().gd_learn_last_error(net.handle) or b"").decode())
    return loss.value


def gd_learn_predict_stack(net: Net, I0, nx, ny, nz, in_shift, in_scale, out_scale, x0) -> int:
    return _ok(lib().gd_learn_predict_stack(net.handle, _p(I0, "f32"), nx, ny, nz, in_shift, in_scale,
                                            out_scale, _p(x0, "f32")), "gd_learn_predict_stack")


def gd_learn_lowmodes(net: Net, I0, x, nx, ny, nz, w, K) -> int:
    from . import _weights
    return _ok(lib().gd_learn_lowmodes(net.handle, _p(I0, "f32"), _p(x, "f32"), nx, ny, nz, _weights(w), K),
               "gd_learn_lowmodes")


def gd_learn_launch_count(net: Net) -> int:
    return int(lib().gd_learn_launch_count(net.handle))


# ---------------------------------------------------------------------------
# parameter layout conversions (the oracle's dict <-> the flat array)
# ---------------------------------------------------------------------------
def params_to_flat(net: Net, p: dict) -> np.ndarray:
    """{name.w: [co][ci][3][3], name.b: [co]} -> flat [co][9][ci] + bias per layer."""
    parts = []
    for name in LAYERS:
        w = np.asarray(p[name + ".w"])
        co, ci = w.shape[:2]
        parts.append(w.reshape(co, ci, 9).transpose(0, 2, 1).reshape(-1))
        parts.append(np.asarray(p[name + ".b"]).reshape(-1))
    return np.concatenate(parts).astype(np.float32)


def flat_to_params(net: Net, flat: np.ndarray) -> dict:
    out, o = {}, 0
    for name, (co, ci) in zip(LAYERS, net.shapes()):
        n = co * 9 * ci
        out[name + ".w"] = flat[o:o + n].reshape(co, 9, ci).transpose(0, 2, 1).reshape(co, ci, 3, 3)
        o += n
        out[name + ".b"] = flat[o:o + co]
        o += co
    return out
