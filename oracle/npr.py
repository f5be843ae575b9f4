"""NPR gradient filter of the paper's discussion (Sec. 7, after Bhat et al.
2010, Sec. 6.2) -- TEST INFRASTRUCTURE ONLY.

The filter solves the global screened Poisson equation

    (alpha + wx Kx + wy Ky + wz Kz) I1 = alpha I0 - div(W V),
    V = lambda (1 - exp(-|grad I0|^2 / (2 sigma^2))) grad I0,

i.e. the general system of Sec. 4 with the target gradients V modulated by
the magnitude of the input gradient (small gradients suppressed, large ones
scaled by lambda).  The paper's video example uses alpha = 0.001,
W = Diag(1, 1, 0.1), lambda = 1.25, sigma = 5 (grey values in [0, 256)).

Discrete reading (the paper gives only the continuous form): gradients are
forward differences on voxel faces with homogeneous Neumann boundaries (a
face leaving the domain carries no gradient); |grad I0|^2 of the face
between voxel p and p + e_d is the squared norm of the forward-difference
vector at its lower voxel p (all three axes, unweighted); -div(W V) at p is
sum_d w_d (V_d(p - e_d -> p) - V_d(p -> p + e_d)), the adjoint of the forward
difference, so that V = grad I0 gives (wx Kx + wy Ky + wz Kz) I0.
"""
from __future__ import annotations

import numpy as np

from .closed_form import _dct3, _idct3, neumann_eigenvalues


def forward_differences(I0):
    """(gx, gy, gz): forward differences along x, y, z (axes 2, 1, 0), with
    zero on the last face of each axis (no face outside the domain)."""
    I0 = np.asarray(I0, dtype=np.float64)
    g = []
    for ax in (2, 1, 0):
        d = np.zeros_like(I0)
        sl_hi = [slice(None)] * 3
        sl_lo = [slice(None)] * 3
        sl_hi[ax] = slice(1, None)
        sl_lo[ax] = slice(None, -1)
        d[tuple(sl_lo)] = I0[tuple(sl_hi)] - I0[tuple(sl_lo)]
        g.append(d)
    return g


def npr_field(I0, lam=1.25, sigma=5.0):
    """The modulated gradients (Vx, Vy, Vz) on the faces p -> p + e_d, stored
    at the lower voxel p."""
    gx, gy, gz = forward_differences(I0)
    mag2 = gx * gx + gy * gy + gz * gz
    m = lam * (1.0 - np.exp(-mag2 / (2.0 * sigma * sigma)))
    return m * gx, m * gy, m * gz


def npr_rhs(I0, alpha=0.001, wx=1.0, wy=1.0, wz=0.1, lam=1.25, sigma=5.0):
    """b = alpha I0 - div(W V) for the NPR filter."""
    I0 = np.asarray(I0, dtype=np.float64)
    V = npr_field(I0, lam, sigma)
    b = alpha * I0
    for w, v, ax in zip((wx, wy, wz), V, (2, 1, 0)):
        # -div: + V on the face entering p, - V on the face leaving p
        inc = np.zeros_like(v)
        sl_hi = [slice(None)] * 3
        sl_lo = [slice(None)] * 3
        sl_hi[ax] = slice(1, None)
        sl_lo[ax] = slice(None, -1)
        inc[tuple(sl_hi)] = v[tuple(sl_lo)]
        b = b + w * (inc - v)
    return b


def screened(b, alpha, wx=1.0, wy=1.0, wz=1.0):
    """Exact x of (alpha + wx Kx + wy Ky + wz Kz) x = b (alpha > 0) in the DCT
    basis (the 6-point Neumann operator is diagonal there)."""
    b = np.asarray(b, dtype=np.float64)
    nz, ny, nx = b.shape
    lam = (wx * neumann_eigenvalues(nx)[None, None, :] + wy * neumann_eigenvalues(ny)[None, :, None]
           + wz * neumann_eigenvalues(nz)[:, None, None])
    return _idct3(_dct3(b) / (alpha + lam))


def npr_loops(I0, alpha, wx, wy, wz, lam, sigma):
    """The same right-hand side by explicit loops over voxels and faces (small
    inputs only): an independent restatement used to pin `npr_rhs`."""
    I0 = np.asarray(I0, dtype=np.float64)
    nz, ny, nx = I0.shape
    w = (wx, wy, wz)
    shape = (nx, ny, nz)

    def val(i, j, k):
        return I0[k, j, i]

    def grad(i, j, k):
        p = (i, j, k)
        out = []
        for d in range(3):
            q = list(p)
            q[d] += 1
            out.append(val(*q) - val(*p) if q[d] < shape[d] else 0.0)
        return out

    def face(i, j, k, d):  # V_d on the face p -> p + e_d
        g = grad(i, j, k)
        m = lam * (1.0 - np.exp(-(g[0] ** 2 + g[1] ** 2 + g[2] ** 2) / (2.0 * sigma ** 2)))
        return m * g[d]

    b = np.zeros_like(I0)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                s = alpha * val(i, j, k)
                p = [i, j, k]
                for d in range(3):
                    if p[d] > 0:
                        q = list(p)
                        q[d] -= 1
                        s += w[d] * face(*q, d)
                    s -= w[d] * face(i, j, k, d)
                b[k, j, i] = s
    return b
