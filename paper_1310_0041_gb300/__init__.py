"""Python binding of libgd.so, the GB300 gradient-domain multigrid solver.

Thin ctypes marshalling over the C ABI declared in ``include/gd.h``: the
functions here carry the same names and arguments; every step of the solve
runs in the library's CUDA kernels.  Arrays are torch CUDA tensors (device
pointers) or numpy arrays (host pointers, staged by the library); float32,
contiguous, shape (nz, ny, nx).

There is no CPU fallback: if ``libgd.so`` is missing or cannot be loaded,
every call raises.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgd.so")

GD_OK, GD_ERR_INVALID_ARG, GD_ERR_UNSUPPORTED, GD_ERR_OOM, GD_ERR_CUDA = 0, 1, 2, 3, 4
GD_ERR_NOT_CONVERGED, GD_ERR_DIVERGED, GD_ERR_TIMEOUT = 5, 6, 7
GD_BC_NEUMANN = 0
GD_DISC_CONSTANT, GD_DISC_HYBRID, GD_DISC_LINEAR = 0, 1, 2
GD_PREC_FP32, GD_PREC_MIXED = 0, 1
GD_SYSTEM_AD, GD_SYSTEM_SP = 0, 1
GD_FLAG_REPORT_OUTPUT_RESIDUAL = 1
GD_HISTORY = 64

# the symbols include/gd.h declares
EXPORTS = ("gd_stack_create", "gd_diffuse_z", "gd_screened_poisson_slices", "gd_vcycle",
           "gd_destroy", "gd_residual", "gd_smooth", "gd_profile_enable", "gd_profile_reset",
           "gd_profile_query", "gd_launch_count", "gd_status_string", "gd_last_error",
           "gd_version", "gd_smooth_noalloc", "gd_screened_poisson", "gd_npr_rhs",
           "gd_batch_create", "gd_batch_screened_poisson", "gd_batch_voxels", "gd_batch_offset",
           "gd_batch_levels", "gd_batch_launch_count", "gd_batch_last_error", "gd_batch_destroy",
           "gd_batch_traffic", "gd_batch_tune", "gd_ad_then_sp", "gd_selftest_wait",
           "gd_batch_last_traffic", "gd_level_count", "gd_level_info", "gd_level_fetch")
# the symbols include/gd_learn.h declares (the learned initial guess)
EXPORTS_LEARN = ("gd_nn_conv3x3", "gd_nn_conv3x3_wgrad", "gd_nn_bias_grad", "gd_nn_flip_weights",
                 "gd_nn_pool2", "gd_nn_pool2_backward", "gd_nn_up2_backward", "gd_nn_adam",
                 "gd_nn_selftest_wait",
                 "gd_learn_stack_tiles", "gd_learn_create", "gd_learn_destroy",
                 "gd_learn_param_count", "gd_learn_set_params", "gd_learn_get_params",
                 "gd_learn_get_grads", "gd_learn_forward", "gd_learn_train_step",
                 "gd_learn_predict_stack", "gd_learn_lowmodes", "gd_learn_launch_count",
                 "gd_learn_last_error")
GD_NOALLOC_MAX_VOXELS = 4 * 1024 * 1024


class GdWeights(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta_x", ctypes.c_double),
                ("beta_y", ctypes.c_double), ("beta_z", ctypes.c_double)]


class GdSolveCtl(ctypes.Structure):
    _fields_ = [("max_cycles", ctypes.c_int), ("rel_tol", ctypes.c_double),
                ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("coarsest_xy", ctypes.c_int),
                ("flags", ctypes.c_int)]


class GdReport(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("cycles", ctypes.c_int), ("levels", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("rel_residual_out", ctypes.c_double),
                ("rho_per_cycle", ctypes.c_double), ("rhs_norm", ctypes.c_double),
                ("history", ctypes.c_double * GD_HISTORY)]

    def to_dict(self) -> dict:
        n = min(self.cycles + 1, GD_HISTORY)
        return dict(status=self.status, cycles=self.cycles, levels=self.levels,
                    rel_residual=self.rel_residual, rel_residual_out=self.rel_residual_out,
                    rho_per_cycle=self.rho_per_cycle, rhs_norm=self.rhs_norm,
                    history=[self.history[i] for i in range(n)])


class GdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (status %d): %s" % (_status_name(status), status, msg))
        self.status = status


_lock = threading.Lock()
_lib = None


def _status_name(st: int) -> str:
    names = {0: "ok", 1: "invalid argument", 2: "unsupported", 3: "out of memory", 4: "CUDA error",
             5: "not converged", 6: "diverged", 7: "timeout"}
    return names.get(st, "unknown")


def lib():
    """The loaded libgd.so (raises if it is missing: build it with build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError("libgd.so not found at %s; build it with "
                                  "`python -m paper_1310_0041_gb300.buildlib`" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            sig = {
                "gd_stack_create": (I, [ctypes.POINTER(P), I, I, I, I, I, I, P]),
                "gd_diffuse_z": (I, [P, P, P, GdWeights, ctypes.POINTER(GdSolveCtl), P,
                                     ctypes.POINTER(GdReport)]),
                "gd_screened_poisson_slices": (I, [P, P, P, P, D, ctypes.POINTER(GdSolveCtl), P,
                                                   ctypes.POINTER(GdReport)]),
                "gd_vcycle": (I, [P, I, GdWeights, P, P, I, ctypes.POINTER(GdReport)]),
                "gd_destroy": (I, [P]),
                "gd_residual": (I, [P, I, GdWeights, P, P, P, ctypes.POINTER(D)]),
                "gd_smooth": (I, [P, GdWeights, P, P, I]),
                "gd_profile_enable": (I, [P, I]),
                "gd_profile_reset": (I, [P]),
                "gd_profile_query": (I, [P, I, ctypes.c_char_p, I, ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.POINTER(D), ctypes.POINTER(D)]),
                "gd_launch_count": (ctypes.c_longlong, [P]),
                "gd_status_string": (ctypes.c_char_p, [I]),
                "gd_last_error": (ctypes.c_char_p, [P]),
                "gd_version": (I, []),
                "gd_smooth_noalloc": (I, [I, I, I, GdWeights, P, P, I, P]),
                "gd_screened_poisson": (I, [P, GdWeights, P, P, ctypes.POINTER(GdSolveCtl), P,
                                            ctypes.POINTER(GdReport)]),
                "gd_npr_rhs": (I, [P, P, P, GdWeights, D, D]),
                "gd_ad_then_sp": (I, [P, P, P, GdWeights, D, ctypes.POINTER(GdSolveCtl),
                                      ctypes.POINTER(GdSolveCtl), P, ctypes.POINTER(GdReport),
                                      ctypes.POINTER(GdReport)]),
                "gd_batch_create": (I, [ctypes.POINTER(P), I, ctypes.POINTER(I), ctypes.POINTER(I),
                                        ctypes.POINTER(D), I, P]),
                "gd_batch_screened_poisson": (I, [P, P, P, P, ctypes.POINTER(GdSolveCtl), P,
                                                  ctypes.POINTER(GdReport), ctypes.POINTER(D)]),
                "gd_batch_voxels": (ctypes.c_longlong, [P]),
                "gd_batch_offset": (ctypes.c_longlong, [P, I]),
                "gd_batch_levels": (I, [P]),
                "gd_batch_traffic": (I, [P, I, I, ctypes.POINTER(D), ctypes.POINTER(D)]),
                "gd_batch_tune": (I, [P, ctypes.POINTER(I)]),
                "gd_batch_last_traffic": (D, [P]),
                "gd_selftest_wait": (I, [ctypes.c_uint]),
                "gd_batch_launch_count": (ctypes.c_longlong, [P]),
                "gd_batch_last_error": (ctypes.c_char_p, [P]),
                "gd_batch_destroy": (I, [P]),
                "gd_level_count": (I, [P]),
                "gd_level_info": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(D)]),
                "gd_level_fetch": (I, [P, I, I, P]),
                # learned initial guess (include/gd_learn.h)
                "gd_nn_conv3x3": (I, [P, I, I, P, I, I, I, I, P, P, I, I, P, P, P, P]),
                "gd_nn_conv3x3_wgrad": (I, [P, I, I, P, I, I, I, I, P, I, P, P]),
                "gd_nn_bias_grad": (I, [P, ctypes.c_longlong, I, P, P]),
                "gd_nn_flip_weights": (I, [P, I, I, P, P, P]),
                "gd_nn_pool2": (I, [P, I, I, I, I, P, P]),
                "gd_nn_pool2_backward": (I, [P, P, I, I, P, I, I, I, I, P, P]),
                "gd_nn_up2_backward": (I, [P, I, I, P, I, I, I, P, P]),
                "gd_nn_adam": (I, [P, P, P, P, ctypes.c_longlong, D, D, D, D, I, P]),
                "gd_nn_selftest_wait": (I, [ctypes.c_uint]),
                "gd_learn_stack_tiles": (I, [P, P, I, I, I, I, I, I, ctypes.c_longlong,
                                             ctypes.c_longlong, D, D, P, P, P]),
                "gd_learn_create": (I, [ctypes.POINTER(P), I, I, ctypes.POINTER(I), I, I, I,
                                        ctypes.c_ulonglong, P]),
                "gd_learn_destroy": (I, [P]),
                "gd_learn_param_count": (ctypes.c_longlong, [P]),
                "gd_learn_set_params": (I, [P, P]),
                "gd_learn_get_params": (I, [P, P]),
                "gd_learn_get_grads": (I, [P, P]),
                "gd_learn_forward": (I, [P, P, I, P]),
                "gd_learn_train_step": (I, [P, P, P, ctypes.c_longlong, ctypes.POINTER(I), I, D,
                                            ctypes.POINTER(D)]),
                "gd_learn_predict_stack": (I, [P, P, I, I, I, D, D, D, P]),
                "gd_learn_lowmodes": (I, [P, P, P, I, I, I, GdWeights, I]),
                "gd_learn_launch_count": (ctypes.c_longlong, [P]),
                "gd_learn_last_error": (ctypes.c_char_p, [P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def build(force: bool = False) -> str:
    """Compile libgd.so in-tree (nvcc, sm_103a)."""
    from . import buildlib
    return buildlib.build(force=force)


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _ptr(a, n: Optional[int] = None, name: str = "array"):
    """Pointer of a float32 contiguous torch tensor (device or host) or numpy array."""
    if a is None:
        return None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float32 or not a.is_contiguous():
                raise ValueError("%s must be a contiguous float32 tensor" % name)
            if n is not None and a.numel() != n:
                raise ValueError("%s has %d elements, expected %d" % (name, a.numel(), n))
            return ctypes.c_void_p(a.data_ptr())
    except ImportError:
        pass
    import numpy as np
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("%s must be a C-contiguous float32 array" % name)
        if n is not None and a.size != n:
            raise ValueError("%s has %d elements, expected %d" % (name, a.size, n))
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError("%s: expected a torch tensor or numpy array" % name)


def _weights(w) -> GdWeights:
    if isinstance(w, GdWeights):
        return w
    if isinstance(w, dict):
        return GdWeights(w.get("alpha", 0.0), w.get("beta_x", 1.0), w.get("beta_y", 1.0),
                         w.get("beta_z", 0.0))
    a, bx, by, bz = w
    return GdWeights(a, bx, by, bz)


def solve_ctl(max_cycles=20, rel_tol=1e-6, nu1=2, nu2=2, coarsest_xy=16, flags=0) -> GdSolveCtl:
    return GdSolveCtl(max_cycles, rel_tol, nu1, nu2, coarsest_xy, flags)


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


class Stack:
    """Handle returned by gd_stack_create (holds the opaque gd_stack*)."""

    def __init__(self, handle, nx, ny, nz):
        self.handle = handle
        self.nx, self.ny, self.nz = nx, ny, nz
        self.n = nx * ny * nz

    def __repr__(self):
        return "Stack(%dx%dx%d)" % (self.nx, self.ny, self.nz)

    @property
    def last_error(self) -> str:
        return gd_last_error(self)


def _check(st: int, stack: Optional[Stack], ok=(GD_OK,)):
    if st not in ok:
        msg = gd_last_error(stack) if stack is not None else ""
        raise GdError(st, msg)
    return st


# ---------------------------------------------------------------------------
# the C ABI, same names
# ---------------------------------------------------------------------------
def gd_stack_create(nx: int, ny: int, nz: int, bc: int = GD_BC_NEUMANN,
                    disc: int = GD_DISC_CONSTANT, prec: int = GD_PREC_FP32, stream=None) -> Stack:
    if stream is None:
        stream = _default_stream()
    h = ctypes.c_void_p()
    st = lib().gd_stack_create(ctypes.byref(h), nx, ny, nz, bc, disc, prec,
                               ctypes.c_void_p(stream) if stream else None)
    _check(st, None)
    return Stack(h, nx, ny, nz)


def gd_destroy(s: Stack) -> int:
    if s is None or s.handle is None:
        return GD_OK
    st = lib().gd_destroy(s.handle)
    s.handle = None
    return st


def gd_diffuse_z(s: Stack, I0, I1, w, ctl: Optional[GdSolveCtl] = None, x0=None,
                 raise_on_error: bool = True) -> dict:
    rep = GdReport()
    st = lib().gd_diffuse_z(s.handle, _ptr(I0, s.n, "I0"), _ptr(I1, s.n, "I1"), _weights(w),
                            ctypes.byref(ctl) if ctl is not None else None, _ptr(x0, s.n, "x0"),
                            ctypes.byref(rep))
    if raise_on_error:
        _check(st, s, ok=(GD_OK, GD_ERR_NOT_CONVERGED))
    return rep.to_dict()


def gd_screened_poisson_slices(s: Stack, I0, I1, I2, alpha: float,
                               ctl: Optional[GdSolveCtl] = None, x0=None,
                               raise_on_error: bool = True) -> dict:
    rep = GdReport()
    st = lib().gd_screened_poisson_slices(s.handle, _ptr(I0, s.n, "I0"), _ptr(I1, s.n, "I1"),
                                          _ptr(I2, s.n, "I2"), float(alpha),
                                          ctypes.byref(ctl) if ctl is not None else None,
                                          _ptr(x0, s.n, "x0"), ctypes.byref(rep))
    if raise_on_error:
        _check(st, s, ok=(GD_OK, GD_ERR_NOT_CONVERGED))
    return rep.to_dict()


def gd_screened_poisson(s: Stack, w, b, x, ctl: Optional[GdSolveCtl] = None, x0=None,
                        raise_on_error: bool = True) -> dict:
    """(alpha + bx Kx + by Ky + bz Kz) x = b; w = (alpha, bx, by, bz)."""
    rep = GdReport()
    st = lib().gd_screened_poisson(s.handle, _weights(w), _ptr(b, s.n, "b"), _ptr(x, s.n, "x"),
                                   ctypes.byref(ctl) if ctl is not None else None,
                                   _ptr(x0, s.n, "x0"), ctypes.byref(rep))
    if raise_on_error:
        _check(st, s, ok=(GD_OK, GD_ERR_NOT_CONVERGED))
    return rep.to_dict()


def gd_ad_then_sp(s: Stack, I0, I2, w_ad, alpha: float, ctl_ad: Optional[GdSolveCtl] = None,
                  ctl_sp: Optional[GdSolveCtl] = None, I1=None, raise_on_error: bool = True) -> tuple:
    """AD then SP in one call (I0 uploaded once); returns the two reports."""
    ra, rs = GdReport(), GdReport()
    st = lib().gd_ad_then_sp(s.handle, _ptr(I0, s.n, "I0"), _ptr(I2, s.n, "I2"), _weights(w_ad),
                             float(alpha), ctypes.byref(ctl_ad) if ctl_ad is not None else None,
                             ctypes.byref(ctl_sp) if ctl_sp is not None else None,
                             _ptr(I1, s.n, "I1"), ctypes.byref(ra), ctypes.byref(rs))
    if raise_on_error:
        _check(st, s, ok=(GD_OK, GD_ERR_NOT_CONVERGED))
    return ra.to_dict(), rs.to_dict()


def gd_npr_rhs(s: Stack, I0, b, w, lam: float, sigma: float) -> int:
    """b = alpha I0 - div(W V) of the NPR filter; w = (alpha, wx, wy, wz)."""
    st = lib().gd_npr_rhs(s.handle, _ptr(I0, s.n, "I0"), _ptr(b, s.n, "b"), _weights(w),
                          float(lam), float(sigma))
    _check(st, s)
    return st


def gd_vcycle(s: Stack, system: int, w, b, x, ncycles: int, raise_on_error: bool = True) -> dict:
    rep = GdReport()
    st = lib().gd_vcycle(s.handle, system, _weights(w), _ptr(b, s.n, "b"), _ptr(x, s.n, "x"),
                         ncycles, ctypes.byref(rep))
    if raise_on_error:
        _check(st, s)
    return rep.to_dict()


def gd_residual(s: Stack, system: int, w, I0, I1, x) -> float:
    out = ctypes.c_double(math.nan)
    st = lib().gd_residual(s.handle, system, _weights(w), _ptr(I0, s.n, "I0"),
                           _ptr(I1, s.n, "I1"), _ptr(x, s.n, "x"), ctypes.byref(out))
    _check(st, s)
    return out.value


def gd_smooth(s: Stack, w, b, x, nsweeps: int) -> int:
    return _check(lib().gd_smooth(s.handle, _weights(w), _ptr(b, s.n, "b"), _ptr(x, s.n, "x"),
                                  nsweeps), s)


def gd_smooth_noalloc(nx: int, ny: int, nz: int, w, b, x, nsweeps: int, stream=None) -> int:
    """Red-black sweeps like gd_smooth with no device allocation (device
    arrays only, at most GD_NOALLOC_MAX_VOXELS voxels); returns the status."""
    import torch
    for name, t in (("b", b), ("x", x)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda):
            raise ValueError("%s must be a CUDA tensor (no staging: nothing is allocated)" % name)
        if t.device.index != torch.cuda.current_device():
            raise ValueError("%s lives on %s, but cuda:%d is current" % (name, t.device,
                                                                      torch.cuda.current_device()))
    if stream is None:
        stream = _default_stream()
    n = nx * ny * nz
    return lib().gd_smooth_noalloc(nx, ny, nz, _weights(w), _ptr(b, n, "b"), _ptr(x, n, "x"),
                                   nsweeps, ctypes.c_void_p(stream) if stream else None)


def gd_level_count(s: Stack) -> int:
    return lib().gd_level_count(s.handle)


def gd_level_info(s: Stack, level: int) -> dict:
    info = (ctypes.c_int * 10)()
    w = (ctypes.c_double * 4)()
    _check(lib().gd_level_info(s.handle, level, info, w), s)
    return {"dims": tuple(info[0:3]), "s": tuple(info[3:6]), "l": tuple(info[6:9]),
            "bytes": info[9], "weights": tuple(w)}


def gd_level_fetch(s: Stack, level: int, which: int, dst) -> int:
    return _check(lib().gd_level_fetch(s.handle, level, which, _ptr(dst)), s)


def gd_profile_enable(s: Stack, on: bool) -> int:
    return _check(lib().gd_profile_enable(s.handle, 1 if on else 0), s)


def gd_profile_reset(s: Stack) -> int:
    return _check(lib().gd_profile_reset(s.handle), s)


def gd_profile_query(s: Stack, k: int):
    """(name, launches, ms, bytes) of kernel class k, or None past the last class."""
    name = ctypes.create_string_buffer(64)
    n, ms, by = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
    st = lib().gd_profile_query(s.handle, k, name, 64, ctypes.byref(n), ctypes.byref(ms),
                                ctypes.byref(by))
    if st != GD_OK:
        return None
    return name.value.decode(), n.value, ms.value, by.value


def gd_profile_all(s: Stack) -> list:
    out, k = [], 0
    while True:
        q = gd_profile_query(s, k)
        if q is None:
            return out
        out.append(q)
        k += 1


def gd_launch_count(s: Stack) -> int:
    return lib().gd_launch_count(s.handle)


def gd_status_string(st: int) -> str:
    return lib().gd_status_string(st).decode()


class Batch:
    """Handle returned by gd_batch_create (holds the opaque gd_batch*)."""

    def __init__(self, handle, nx, ny, alpha):
        self.handle = handle
        self.nx, self.ny, self.alpha = list(nx), list(ny), list(alpha)
        self.ns = len(self.nx)
        self.n = sum(a * b for a, b in zip(self.nx, self.ny))

    def __repr__(self):
        return "Batch(%d slices, %d cells)" % (self.ns, self.n)

    @property
    def last_error(self) -> str:
        return gd_batch_last_error(self)


def gd_batch_create(nx, ny, alpha, coarsest_xy: int = 0, stream=None) -> Batch:
    """Plans the batch of slices nx[s] x ny[s] with screening weights alpha[s]."""
    nx, ny, alpha = [int(v) for v in nx], [int(v) for v in ny], [float(v) for v in alpha]
    ns = len(nx)
    if len(ny) != ns or len(alpha) != ns:
        raise ValueError("nx, ny and alpha must have the same length")
    if stream is None:
        stream = _default_stream()
    h = ctypes.c_void_p()
    st = lib().gd_batch_create(ctypes.byref(h), ns, (ctypes.c_int * ns)(*nx), (ctypes.c_int * ns)(*ny),
                               (ctypes.c_double * ns)(*alpha), int(coarsest_xy),
                               ctypes.c_void_p(stream) if stream else None)
    if st != GD_OK:
        raise GdError(st, gd_batch_last_error(None))
    return Batch(h, nx, ny, alpha)


def gd_batch_screened_poisson(b: Batch, I0, I1, I2, ctl: Optional[GdSolveCtl] = None, x0=None,
                              raise_on_error: bool = True, slice_rel: bool = False) -> dict:
    """Packed arrays of b.n floats; returns the report (+ 'slice_rel' if asked)."""
    rep = GdReport()
    sr = (ctypes.c_double * b.ns)() if slice_rel else None
    st = lib().gd_batch_screened_poisson(b.handle, _ptr(I0, b.n, "I0"), _ptr(I1, b.n, "I1"),
                                         _ptr(I2, b.n, "I2"),
                                         ctypes.byref(ctl) if ctl is not None else None,
                                         _ptr(x0, b.n, "x0"), ctypes.byref(rep), sr)
    if raise_on_error and st not in (GD_OK, GD_ERR_NOT_CONVERGED):
        raise GdError(st, gd_batch_last_error(b))
    out = rep.to_dict()
    if slice_rel:
        out["slice_rel"] = list(sr)
    return out


def gd_batch_voxels(b: Batch) -> int:
    return lib().gd_batch_voxels(b.handle)


def gd_batch_offset(b: Batch, s: int) -> int:
    return lib().gd_batch_offset(b.handle, s)


def gd_batch_levels(b: Batch) -> int:
    return lib().gd_batch_levels(b.handle)


def gd_batch_traffic(b: Batch, nu1: int = 2, nu2: int = 2) -> tuple:
    """(bytes per V-cycle with its outer pass, bytes of the once-per-solve passes)."""
    pc, ps = ctypes.c_double(), ctypes.c_double()
    st = lib().gd_batch_traffic(b.handle, nu1, nu2, ctypes.byref(pc), ctypes.byref(ps))
    if st != GD_OK:
        raise GdError(st, gd_batch_last_error(b))
    return pc.value, ps.value


def gd_batch_last_traffic(b: Batch) -> float:
    """Algorithmic bytes of the last batched solve (the work actually done)."""
    return lib().gd_batch_last_traffic(b.handle)


def gd_batch_tune(b: Batch) -> int:
    """Times the candidate work-item heights and keeps the fastest; returns it."""
    c = ctypes.c_int()
    st = lib().gd_batch_tune(b.handle, ctypes.byref(c))
    if st != GD_OK:
        raise GdError(st, gd_batch_last_error(b))
    return c.value


def gd_batch_launch_count(b: Batch) -> int:
    return lib().gd_batch_launch_count(b.handle)


def gd_batch_last_error(b: Optional[Batch]) -> str:
    r = lib().gd_batch_last_error(b.handle if b is not None else None)
    return r.decode() if r else ""


def gd_batch_destroy(b: Batch) -> int:
    if b is None or b.handle is None:
        return GD_OK
    st = lib().gd_batch_destroy(b.handle)
    b.handle = None
    return st


def gd_selftest_wait(polls: int) -> int:
    """Bounded-wait self-test; returns the status (GD_ERR_TIMEOUT expected)."""
    return lib().gd_selftest_wait(int(polls))


def gd_last_error(s: Optional[Stack]) -> str:
    r = lib().gd_last_error(s.handle if s is not None else None)
    return r.decode() if r else ""


def gd_version() -> int:
    return lib().gd_version()
