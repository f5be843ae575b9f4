"""The "Linear" discretisation of Sec. 4.2 -- TEST INFRASTRUCTURE ONLY (same
rules as the rest of ``oracle``).

First-order B-spline (trilinear) finite elements: with the 1D stiffness
K_n = tridiag(-1, [1, 2, ..., 2, 1], -1) and the 1D mass
M_n = (1/6) tridiag(1, [2, 4, ..., 4, 2], 1) of hat functions on n nodes, the
operators of both steps are Kronecker sums (a 27-point stencil in 3D):

  AD:  (bx Kx(x)My(x)Mz + by Mx(x)Ky(x)Mz + bz Mx(x)My(x)Kz) I1
         = (bx Kx(x)My(x)Mz + by Mx(x)Ky(x)Mz) I0,   sum(I1) = sum(I0);
  SP, per slice:  (alpha Mx(x)My + Kx(x)My + Mx(x)Ky) I2
         = alpha Mx(x)My I1 + (Kx(x)My + Mx(x)Ky) I0.

Readings: an axis with a single node has no element, so it carries no term:
K_1 = [0], M_1 = [1] (a stack with nz = 1 is one slice).  AD keeps the plain
sum of I0 (the constant is the null space; any fixed mean is a reading).

Arrays are ``[nz][ny][nx]`` (x fastest); the Kronecker products are written
with z outermost, so ``kron(Mz, kron(My, Kx))`` acts on the flattened array.
Solves use scipy's sparse direct solver (SP) and conjugate gradients on the
mean-free part (AD).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def K1(n: int):
    """1D stiffness of hat functions on n nodes (Neumann ends)."""
    if n == 1:
        return sp.csr_matrix((1, 1))
    d = np.full(n, 2.0)
    d[0] = d[-1] = 1.0
    o = np.full(n - 1, -1.0)
    return sp.diags([o, d, o], [-1, 0, 1], format="csr")


def M1(n: int):
    """1D mass of hat functions on n nodes."""
    if n == 1:
        return sp.identity(1, format="csr")
    d = np.full(n, 4.0 / 6.0)
    d[0] = d[-1] = 2.0 / 6.0
    o = np.full(n - 1, 1.0 / 6.0)
    return sp.diags([o, d, o], [-1, 0, 1], format="csr")


def kron3(Az, Ay, Ax):
    return sp.kron(Az, sp.kron(Ay, Ax, format="csr"), format="csr")


def operator(shape, alpha=0.0, bx=1.0, by=1.0, bz=1.0, slices=False):
    """alpha M(x)M(x)M + bx Kx(x)My(x)Mz + by Mx(x)Ky(x)Mz + bz Mx(x)My(x)Kz;
    slices=True: independent slices (no z term, the z factor is I)."""
    nz, ny, nx = shape
    Kx, Ky, Kz, Mx, My = K1(nx), K1(ny), K1(nz), M1(nx), M1(ny)
    Mz = sp.identity(nz, format="csr") if slices else M1(nz)
    A = bx * kron3(Mz, My, Kx) + by * kron3(Mz, Ky, Mx)
    if not slices:
        A = A + bz * kron3(Kz, My, Mx)
    if alpha:
        A = A + alpha * kron3(Mz, My, Mx)
    return A.tocsr()


def rhs_ad(I0, bx=1.0, by=1.0):
    I0 = np.asarray(I0, dtype=np.float64)
    G = operator(I0.shape, 0.0, bx, by, 0.0)
    return (G @ I0.ravel()).reshape(I0.shape)


def rhs_sp(I0, I1, alpha):
    I0 = np.asarray(I0, dtype=np.float64)
    I1 = np.asarray(I1, dtype=np.float64)
    G = operator(I0.shape, 0.0, 1.0, 1.0, 0.0, slices=True)
    Mm = operator(I0.shape, 1.0, 0.0, 0.0, 0.0, slices=True)
    return (G @ I0.ravel() + alpha * (Mm @ I1.ravel())).reshape(I0.shape)


def ad(I0, bx=1.0, by=1.0, bz=0.1, tol=1e-13):
    """Exact (to CG tolerance) I1 of the Linear AD system with sum(I1) = sum(I0)."""
    I0 = np.asarray(I0, dtype=np.float64)
    A = operator(I0.shape, 0.0, bx, by, bz)
    b = rhs_ad(I0, bx, by).ravel()
    n = b.size
    # A is singular with null space 1 and b is consistent (1^T b = 0): CG
    # from 0 stays mean-free
    x, info = spla.cg(A, b, rtol=tol, atol=0.0, maxiter=20000)
    assert info == 0, info
    x = x - x.mean() + I0.mean()
    return x.reshape(I0.shape)


def sp_solve(I0, I1, alpha=0.01):
    """Exact I2 of the Linear SP system (sparse direct solve)."""
    I0 = np.asarray(I0, dtype=np.float64)
    A = operator(I0.shape, alpha, 1.0, 1.0, 0.0, slices=True)
    b = rhs_sp(I0, I1, alpha).ravel()
    return spla.spsolve(A.tocsc(), b).reshape(I0.shape)


def rel_residual(A, b, x) -> float:
    b = np.asarray(b, dtype=np.float64).ravel()
    r = b - A @ np.asarray(x, dtype=np.float64).ravel()
    return float(np.linalg.norm(r) / np.linalg.norm(b))


# ---------------------------------------------------------------------------
# the same exact solutions by fast diagonalisation (Lynch, Rice & Thomas,
# 1964): per axis the generalised eigenpairs K v = lam M v with V^T M V = I
# (scipy.linalg.eigh), so that V^T A V is diagonal for the Kronecker sums
# above; usable at sizes where the sparse solves are slow.
# ---------------------------------------------------------------------------
def _axis_eig(n: int):
    import scipy.linalg as sla
    lam, V = sla.eigh(K1(n).toarray(), M1(n).toarray())
    return lam, V


def _apply_axes(a, Vz, Vy, Vx, transpose: bool):
    """(Vz (x) Vy (x) Vx)^T a (transpose) or (Vz (x) Vy (x) Vx) a, a [nz][ny][nx]."""
    T = (lambda V: V.T) if transpose else (lambda V: V)
    a = np.tensordot(T(Vz), a, axes=(1, 0))                   # z
    a = np.tensordot(T(Vy), a, axes=(1, 1)).transpose(1, 0, 2)  # y
    a = np.tensordot(a, T(Vx), axes=(2, 1))                   # x
    return a


def ad_fdm(I0, bx=1.0, by=1.0, bz=0.1):
    """I1 of the Linear AD system with sum(I1) = sum(I0), by fast diagonalisation."""
    I0 = np.asarray(I0, dtype=np.float64)
    nz, ny, nx = I0.shape
    (lz, Vz), (ly, Vy), (lx, Vx) = _axis_eig(nz), _axis_eig(ny), _axis_eig(nx)
    b = _apply_axes(rhs_ad(I0, bx, by), Vz, Vy, Vx, True)
    D = bx * lx[None, None, :] + by * ly[None, :, None] + bz * lz[:, None, None]
    zero = np.abs(D) <= 1e-12 * max(1.0, np.abs(D).max())
    b = np.where(zero, 0.0, b / np.where(zero, 1.0, D))   # pseudo-inverse: null space dropped
    x = _apply_axes(b, Vz, Vy, Vx, False)
    return x - x.mean() + I0.mean()


def sp_fdm(I0, I1, alpha=0.01):
    """I2 of the Linear SP system (independent slices), by fast diagonalisation."""
    I0 = np.asarray(I0, dtype=np.float64)
    nz, ny, nx = I0.shape
    (ly, Vy), (lx, Vx) = _axis_eig(ny), _axis_eig(nx)
    Iz = np.eye(nz)
    b = _apply_axes(rhs_sp(I0, I1, alpha), Iz, Vy, Vx, True)
    b = b / (alpha + lx[None, None, :] + ly[None, :, None])
    return _apply_axes(b, Iz, Vy, Vx, False)
