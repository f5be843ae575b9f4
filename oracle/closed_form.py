"""Exact discrete solutions in the DCT basis -- TEST INFRASTRUCTURE ONLY.

Sec. 3.2 of the paper reads both steps as filters in frequency space: with
Fourier eigenvalues k^2, l^2, m^2 of the second derivatives,

  AD:  I1^_klm = (bx k^2 + by l^2) / (bx k^2 + by l^2 + bz m^2) * I0^_klm
  SP:  I2^_klm = (alpha I1^_klm + (k^2 + l^2) I0^_klm) / (alpha + k^2 + l^2)

(the printed AD denominator has "bz^2 m^2" in one line and "bz m^2" in the
others; the reading used is bz m^2, the one the Euler-Lagrange equation
gives).

For the 6-point Neumann discretisation the same statement is exact on the
grid: the 1D matrix K_n = tridiag(-1, [1,2,...,2,1], -1) is diagonalised by
the orthonormal DCT-II, with eigenvalues lambda_k = 4 sin^2(pi k / (2 n)),
so replacing k^2 by lambda_k (per axis) gives the exact discrete solution.
The all-zero mode of AD is undetermined by the equation; it is kept equal to
that of I0 (mean preservation).  Modes with bx lambda_k + by lambda_l = 0 and
bz lambda_m > 0 (slice means varying along z) are set to zero by AD.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft


def neumann_eigenvalues(n: int) -> np.ndarray:
    """Eigenvalues of K_n in DCT-II order: 4 sin^2(pi k / 2n), k = 0..n-1."""
    k = np.arange(n, dtype=np.float64)
    return 4.0 * np.sin(np.pi * k / (2.0 * n)) ** 2


def _dct3(a):
    return sfft.dctn(np.asarray(a, dtype=np.float64), type=2, norm="ortho", workers=-1)


def _idct3(a):
    return sfft.idctn(a, type=2, norm="ortho", workers=-1)


def ad_filter(shape, bx=1.0, by=1.0, bz=0.1) -> np.ndarray:
    """Per-mode multiplier of the AD step, shape (nz, ny, nx)."""
    nz, ny, nx = shape
    lx = neumann_eigenvalues(nx)[None, None, :]
    ly = neumann_eigenvalues(ny)[None, :, None]
    lz = neumann_eigenvalues(nz)[:, None, None]
    num = bx * lx + by * ly
    den = num + bz * lz
    f = np.divide(num, den, out=np.zeros(np.broadcast_shapes(num.shape, den.shape)), where=den > 0)
    f[0, 0, 0] = 1.0
    return f


def ad(I0, bx=1.0, by=1.0, bz=0.1) -> np.ndarray:
    """Exact I1 of (bx Kx + by Ky + bz Kz) I1 = (bx Kx + by Ky) I0, mean(I1) = mean(I0)."""
    I0 = np.asarray(I0, dtype=np.float64)
    return _idct3(_dct3(I0) * ad_filter(I0.shape, bx, by, bz))


def sp(I0, I1, alpha=0.01) -> np.ndarray:
    """Exact I2 of (alpha + Kx + Ky) I2 = alpha I1 + (Kx + Ky) I0, slice by slice.
    Uses a 2D DCT per slice (the z axis is not transformed)."""
    I0 = np.asarray(I0, dtype=np.float64)
    I1 = np.asarray(I1, dtype=np.float64)
    nz, ny, nx = I0.shape
    lxy = neumann_eigenvalues(nx)[None, None, :] + neumann_eigenvalues(ny)[None, :, None]
    H0 = sfft.dctn(I0, type=2, norm="ortho", axes=(1, 2), workers=-1)
    H1 = sfft.dctn(I1, type=2, norm="ortho", axes=(1, 2), workers=-1)
    H2 = (alpha * H1 + lxy * H0) / (alpha + lxy)
    return sfft.idctn(H2, type=2, norm="ortho", axes=(1, 2), workers=-1)


def combined_filter(shape, alpha=0.01, bx=1.0, by=1.0, bz=0.1) -> np.ndarray:
    """Discrete F^ of Sec. 3.2 (AD followed by SP with I1 from AD), (nz, ny, nx).
    Uses the unweighted in-slice term for SP (W = pi = Diag(1,1,0))."""
    nz, ny, nx = shape
    lx = neumann_eigenvalues(nx)[None, None, :]
    ly = neumann_eigenvalues(ny)[None, :, None]
    return (alpha * ad_filter(shape, bx, by, bz) + (lx + ly)) / (alpha + lx + ly)
