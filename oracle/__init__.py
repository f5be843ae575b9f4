"""FP64 CPU oracle for the gradient-domain solver -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The solver library never does, and this package
imports nothing from it.

Two independent routes to the exact discrete solutions:

* ``closed_form`` -- the DCT-diagonal closed form of the 6-point Neumann
  system (the discrete counterpart of the frequency-space filters of Sec. 3.2);
* ``gd_oracle.c`` (this module's ``ad_solve`` / ``sp_solve``) -- plain FP64
  loops: right-hand sides, operator, Gauss-Seidel, conjugate gradients, the
  paper's V-cycle (Sec. 4.1) and a dense Cholesky solve.

Further modules: ``npr`` (the NPR gradient filter of Sec. 7), ``batch``
(screened Poisson on independent slices of different sizes), ``linear``
(the Linear discretisation of Sec. 4.2, trilinear elements) and ``learned``
(the convolutional network of a learned initial guess: forward, backward,
Adam).

System (paper Sec. 3.1 and Sec. 4, 6-point discretisation of Sec. 4.2, read
with homogeneous Neumann boundaries):

* anisotropic diffusion:  (bx Kx + by Ky + bz Kz) I1 = (bx Kx + by Ky) I0,
  with mean(I1) = mean(I0) fixing the constant null space;
* screened Poisson, per slice:  (alpha + Kx + Ky) I2 = alpha I1 + (Kx + Ky) I0.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import closed_form  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libgdoracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.c_double
_I = ctypes.c_int
_P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile gd_oracle.c into libgdoracle.so (gcc, FP64, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            sig = {
                "gdo_rhs_ad": (_I, [_I, _I, _I, _D, _D, _P, _P]),
                "gdo_rhs_sp": (_I, [_I, _I, _I, _D, _P, _P, _P]),
                "gdo_apply": (_I, [_I, _I, _I, _D, _D, _D, _D, _P, _P]),
                "gdo_rel_residual": (_D, [_I, _I, _I, _D, _D, _D, _D, _P, _P]),
                "gdo_gs_sweeps": (_I, [_I, _I, _I, _D, _D, _D, _D, _P, _P, _I, _I]),
                "gdo_cg": (_I, [_I, _I, _I, _D, _D, _D, _D, _P, _P, _D, _I, _P, _P]),
                "gdo_dense": (_I, [_I, _I, _I, _D, _D, _D, _D, _P, _P]),
                "gdo_restrict": (_I, [_I, _I, _I, _I, _I, _I, _P, _P]),
                "gdo_prolong_add": (_I, [_I, _I, _I, _I, _I, _I, _P, _P]),
                "gdo_mg": (_I, [_I, _I, _I, _D, _D, _D, _D, _P, _P, _I, _I, _I, _I, _D, _I, _P, _P, _P]),
                "gdo_threads": (_I, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dims(a):
    nz, ny, nx = a.shape
    return nx, ny, nz


def threads() -> int:
    return lib().gdo_threads()


# --------------------------------------------------------------------------
# right-hand sides and operator
# --------------------------------------------------------------------------
def rhs_ad(I0, bx=1.0, by=1.0) -> np.ndarray:
    """b = (bx Kx + by Ky) I0, i.e. minus the divergence of W G, Eq. (anisotropic_diffusion)."""
    I0 = _f64(I0)
    b = np.empty_like(I0)
    rc = lib().gdo_rhs_ad(*_dims(I0), bx, by, I0.ctypes.data, b.ctypes.data)
    assert rc == 0
    return b


def rhs_sp(I0, I1, alpha) -> np.ndarray:
    """b = alpha I1 + (Kx + Ky) I0, Eq. (screened_poisson)."""
    I0, I1 = _f64(I0), _f64(I1)
    b = np.empty_like(I0)
    rc = lib().gdo_rhs_sp(*_dims(I0), alpha, I0.ctypes.data, I1.ctypes.data, b.ctypes.data)
    assert rc == 0
    return b


def apply(x, alpha=0.0, bx=1.0, by=1.0, bz=1.0) -> np.ndarray:
    """A x with A = alpha I + bx Kx + by Ky + bz Kz (general form of Sec. 4)."""
    x = _f64(x)
    y = np.empty_like(x)
    rc = lib().gdo_apply(*_dims(x), alpha, bx, by, bz, x.ctypes.data, y.ctypes.data)
    assert rc == 0
    return y


def rel_residual(b, x, alpha=0.0, bx=1.0, by=1.0, bz=1.0) -> float:
    """||b - A x||_2 / ||b||_2 (Table 1 caption: residual over initial constraints)."""
    b, x = _f64(b), _f64(x)
    return lib().gdo_rel_residual(*_dims(x), alpha, bx, by, bz, b.ctypes.data, x.ctypes.data)


def gs_sweeps(b, x, alpha=0.0, bx=1.0, by=1.0, bz=1.0, order="redblack", nsweeps=1) -> np.ndarray:
    """Gauss-Seidel sweeps on the fine-level system; returns the new iterate.
    order: "lex" (x fastest) or "redblack" (red = (i+j+k) even first)."""
    b = _f64(b)
    x = _f64(x).copy()
    rc = lib().gdo_gs_sweeps(*_dims(x), alpha, bx, by, bz, b.ctypes.data, x.ctypes.data,
                             0 if order == "lex" else 1, nsweeps)
    assert rc == 0
    return x


def cg(b, x0, alpha=0.0, bx=1.0, by=1.0, bz=1.0, tol=1e-12, maxit=200000):
    b = _f64(b)
    x = _f64(x0).copy()
    it, rr = _I(0), _D(0.0)
    rc = lib().gdo_cg(*_dims(x), alpha, bx, by, bz, b.ctypes.data, x.ctypes.data, tol, maxit,
                      ctypes.byref(it), ctypes.byref(rr))
    return x, dict(status=rc, iters=it.value, rel_residual=rr.value)


def dense(b, alpha=0.0, bx=1.0, by=1.0, bz=1.0) -> np.ndarray:
    b = _f64(b)
    x = np.empty_like(b)
    rc = lib().gdo_dense(*_dims(b), alpha, bx, by, bz, b.ctypes.data, x.ctypes.data)
    if rc != 0:
        raise ValueError("gdo_dense failed: %d" % rc)
    return x


def restrict(r, fx=1, fy=1, fz=1) -> np.ndarray:
    """Down-sampling by summing the children (P^T of the replication prolongation)."""
    r = _f64(r)
    nz, ny, nx = r.shape
    out = np.empty(((nz + 1) // 2 if fz else nz, (ny + 1) // 2 if fy else ny,
                    (nx + 1) // 2 if fx else nx))
    rc = lib().gdo_restrict(nx, ny, nz, fx, fy, fz, r.ctypes.data, out.ctypes.data)
    assert rc == 0
    return out


def prolong_add(ec, x, fx=1, fy=1, fz=1) -> np.ndarray:
    """x + P ec with P replicating each coarse value into its children."""
    ec = _f64(ec)
    x = _f64(x).copy()
    nz, ny, nx = x.shape
    rc = lib().gdo_prolong_add(nx, ny, nz, fx, fy, fz, ec.ctypes.data, x.ctypes.data)
    assert rc == 0
    return x


def mg(b, x0, alpha=0.0, bx=1.0, by=1.0, bz=1.0, order="redblack", nu1=2, nu2=2, min_xy=16,
       tol=1e-10, max_cycles=200):
    b = _f64(b)
    x = _f64(x0).copy()
    cyc, rr = _I(0), _D(0.0)
    hist = np.zeros(max_cycles + 1)
    rc = lib().gdo_mg(*_dims(x), alpha, bx, by, bz, b.ctypes.data, x.ctypes.data,
                      0 if order == "lex" else 1, nu1, nu2, min_xy, tol, max_cycles,
                      ctypes.byref(cyc), ctypes.byref(rr), hist.ctypes.data)
    return x, dict(status=rc, cycles=cyc.value, rel_residual=rr.value, history=hist[:cyc.value + 1])


# --------------------------------------------------------------------------
# the two steps of the method, solved to a tolerance
# --------------------------------------------------------------------------
def ad_solve(I0, bx=1.0, by=1.0, bz=0.1, method="mg", tol=1e-10, x0=None, **kw):
    """I1 of the anisotropic diffusion step (Sec. 3.1) in FP64, with
    mean(I1) = mean(I0).  method: "mg" (paper V-cycle), "cg" or "dense"."""
    I0 = _f64(I0)
    b = rhs_ad(I0, bx, by)
    start = I0 if x0 is None else _f64(x0)
    if method == "dense":
        x, info = dense(b, 0.0, bx, by, bz), dict(status=0)
    elif method == "cg":
        x, info = cg(b, start, 0.0, bx, by, bz, tol=tol, **kw)
    else:
        x, info = mg(b, start, 0.0, bx, by, bz, tol=tol, **kw)
    x = x + (I0.mean() - x.mean())
    info["rel_residual_final"] = rel_residual(b, x, 0.0, bx, by, bz)
    return x, info


def sp_solve(I0, I1, alpha=0.01, method="mg", tol=1e-10, x0=None, **kw):
    """I2 of the screened-Poisson step (Sec. 3.1), slice by slice, in FP64."""
    I0, I1 = _f64(I0), _f64(I1)
    start = I1 if x0 is None else _f64(x0)
    out = np.empty_like(I0)
    infos = []
    for k in range(I0.shape[0]):
        b = rhs_sp(I0[k:k + 1], I1[k:k + 1], alpha)
        if method == "dense":
            x, info = dense(b, alpha, 1.0, 1.0, 0.0), dict(status=0)
        elif method == "cg":
            x, info = cg(b, start[k:k + 1], alpha, 1.0, 1.0, 0.0, tol=tol, **kw)
        else:
            x, info = mg(b, start[k:k + 1], alpha, 1.0, 1.0, 0.0, tol=tol, **kw)
        out[k] = x[0]
        infos.append(info)
    b = rhs_sp(I0, I1, alpha)
    return out, dict(slices=infos, rel_residual_final=rel_residual(b, out, alpha, 1.0, 1.0, 0.0))
