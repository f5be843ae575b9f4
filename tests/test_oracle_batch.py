"""Pins of the batched screened Poisson oracle (``oracle.batch``), CPU only.

The batch oracle answers slice by slice through the DCT closed form.  These
tests pin it to things other than itself: a dense solve of the operator
written out from its definition (Sec. 3.1, Eq. screened_poisson, with the
6-point Neumann stencil of Sec. 4.2) on tiny ragged slices with their own
alphas, and the special cases the equation fixes.
"""
import numpy as np
import pytest

import gdsynth
import oracle.batch as ob


def dense_operator(nx: int, ny: int, alpha: float) -> np.ndarray:
    """alpha I + Kx + Ky as a dense (nx ny)^2 matrix, from the stencil: each
    cell couples with -1 to each existing x and y neighbour and has the
    number of existing neighbours (plus alpha) on the diagonal."""
    n = nx * ny
    A = np.zeros((n, n))
    for j in range(ny):
        for i in range(nx):
            p = j * nx + i
            A[p, p] += alpha
            for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < nx and 0 <= jj < ny:
                    A[p, p] += 1.0
                    A[p, jj * nx + ii] -= 1.0
    return A


SIZES = [(1, 1), (1, 5), (4, 3), (7, 5), (9, 2), (6, 6), (3, 8)]


def test_batch_oracle_matches_dense_solves():
    nx = [a for a, _ in SIZES]
    ny = [b for _, b in SIZES]
    I0s, I1s = gdsynth.batch_slices(nx, ny, seed=11)
    al = gdsynth.batch_alphas(len(SIZES), seed=11)
    xs = ob.sp_batch(I0s, I1s, al)
    for (a, b), i0, i1, alpha, x in zip(SIZES, I0s, I1s, al, xs):
        A = dense_operator(a, b, alpha)
        K = dense_operator(a, b, 0.0)
        rhs = alpha * i1.astype(np.float64).ravel() + K @ i0.astype(np.float64).ravel()
        ref = np.linalg.solve(A, rhs).reshape(b, a)
        assert x.shape == (b, a)
        assert np.max(np.abs(x - ref)) < 1e-9, (a, b)
        # the oracle's loop-based right-hand side and operator agree with the dense ones
        assert np.allclose(ob.rhs_slice(i0, i1, alpha).ravel(), rhs, atol=1e-10)
        assert np.allclose(ob.apply_slice(ref, alpha).ravel(), A @ ref.ravel(), atol=1e-9)


def test_batch_oracle_special_cases():
    nx, ny = [13, 40, 1], [9, 3, 17]
    I0s, I1s = gdsynth.batch_slices(nx, ny, seed=5)
    # I1 == I0: the right-hand side is A I0, so I2 == I0
    for i0, alpha in zip(I0s, (0.001, 0.05, 0.1)):
        assert np.max(np.abs(ob.sp_slice(i0, i0, alpha) - i0)) < 1e-8
    # a dominant screening weight pins I2 to I1: |I2 - I1| <= |K (I0 - I1)|_inf / alpha
    for i0, i1 in zip(I0s, I1s):
        x = ob.sp_slice(i0, i1, 1e7)
        assert np.max(np.abs(x - i1)) < 1e-3
    # a single cell has no neighbours: I2 == I1
    x = ob.sp_slice(np.array([[7.0]]), np.array([[3.0]]), 0.01)
    assert abs(x[0, 0] - 3.0) < 1e-12


def test_batch_oracle_residual_flags_planted_mistakes():
    # a wrong sign in the gradient term, or a dropped screening term, is seen
    # by the loop-based residual the GPU parity tests rely on
    nx, ny = [33], [21]
    I0s, I1s = gdsynth.batch_slices(nx, ny, seed=2)
    i0, i1, alpha = I0s[0], I1s[0], 0.02
    x = ob.sp_slice(i0, i1, alpha)
    assert ob.rel_residual_slice(i0, i1, alpha, x) < 1e-12
    K = dense_operator(33, 21, 0.0)
    wrong_sign = np.linalg.solve(dense_operator(33, 21, alpha),
                                 alpha * i1.ravel() - K @ i0.ravel()).reshape(21, 33)
    assert ob.rel_residual_slice(i0, i1, alpha, wrong_sign) > 1e-2
    no_screen = np.linalg.solve(dense_operator(33, 21, alpha), K @ i0.ravel()).reshape(21, 33)
    assert ob.rel_residual_slice(i0, i1, alpha, no_screen) > 1e-3
