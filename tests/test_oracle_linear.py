"""Pins of the Linear-discretisation oracle (``oracle/linear.py``), CPU only.

The oracle assembles the operators from 1D stiffness and mass matrices by
Kronecker products.  These tests pin it to the finite-element definition it
stands for (trilinear hat functions on a unit grid, Sec. 4.2 "Linear"): the
1D matrices and the full 3D operator are integrated directly with Gauss
quadrature on tiny grids, and the solutions are checked against dense solves
and the special cases the equations fix.
"""
import itertools

import numpy as np
import pytest

import gdsynth
import oracle.linear as ol

G2 = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))  # 2-point Gauss on [0, 1]


def hat(i, x):
    return max(0.0, 1.0 - abs(x - i))


def dhat(i, x, e):
    # derivative of hat i inside element [e, e+1]
    if i == e:
        return -1.0
    if i == e + 1:
        return 1.0
    return 0.0


def test_1d_matrices_are_the_hat_function_integrals():
    for n in (2, 3, 6):
        K = np.zeros((n, n))
        M = np.zeros((n, n))
        for e in range(n - 1):
            for g in G2:
                x = e + g
                for i in range(n):
                    for j in range(n):
                        K[i, j] += 0.5 * dhat(i, x, e) * dhat(j, x, e)
                        M[i, j] += 0.5 * hat(i, x) * hat(j, x)
        assert np.allclose(K, ol.K1(n).toarray(), atol=1e-14)
        assert np.allclose(M, ol.M1(n).toarray(), atol=1e-14)


def test_3d_operator_is_the_trilinear_integral():
    # grad(phi_I) . W grad(phi_J) + alpha phi_I phi_J over the box, with
    # 2x2x2 Gauss points per element and trilinear hat products
    shape = (2, 3, 4)  # nz, ny, nx nodes
    nz, ny, nx = shape
    bx, by, bz, alpha = 1.3, 0.7, 2.1, 0.4
    nodes = list(itertools.product(range(nz), range(ny), range(nx)))
    N = len(nodes)
    A = np.zeros((N, N))
    for ez, ey, ex in itertools.product(range(nz - 1), range(ny - 1), range(nx - 1)):
        for gz, gy, gx in itertools.product(G2, G2, G2):
            z, y, x = ez + gz, ey + gy, ex + gx
            w = 0.125
            val = np.array([hat(k, z) * hat(j, y) * hat(i, x) for k, j, i in nodes])
            gxv = np.array([hat(k, z) * hat(j, y) * dhat(i, x, ex) for k, j, i in nodes])
            gyv = np.array([hat(k, z) * dhat(j, y, ey) * hat(i, x) for k, j, i in nodes])
            gzv = np.array([dhat(k, z, ez) * hat(j, y) * hat(i, x) for k, j, i in nodes])
            A += w * (bx * np.outer(gxv, gxv) + by * np.outer(gyv, gyv) + bz * np.outer(gzv, gzv)
                      + alpha * np.outer(val, val))
    assert np.allclose(A, ol.operator(shape, alpha, bx, by, bz).toarray(), atol=1e-13)


def test_solutions_solve_the_systems():
    I0 = gdsynth.em_stack(11, 9, 5, seed=3).astype(np.float64)
    for bz in (10.0, 0.1):
        I1 = ol.ad(I0, 1.0, 1.0, bz)
        A = ol.operator(I0.shape, 0.0, 1.0, 1.0, bz)
        assert ol.rel_residual(A, ol.rhs_ad(I0), I1) < 1e-11
        assert abs(I1.sum() - I0.sum()) < 1e-8 * abs(I0.sum())
        # dense least-squares solve of the singular system, mean matched
        Ad = A.toarray()
        xd = np.linalg.lstsq(Ad, ol.rhs_ad(I0).ravel(), rcond=None)[0]
        xd = xd - xd.mean() + I0.mean()
        assert np.abs(xd.reshape(I0.shape) - I1).max() < 1e-7
    I2 = ol.sp_solve(I0, I1, 0.02)
    A2 = ol.operator(I0.shape, 0.02, 1.0, 1.0, 0.0, slices=True)
    xd = np.linalg.solve(A2.toarray(), ol.rhs_sp(I0, I1, 0.02).ravel())
    assert np.abs(xd.reshape(I0.shape) - I2).max() < 1e-9


def test_special_cases():
    I0 = gdsynth.em_stack(10, 7, 4, seed=8).astype(np.float64)
    # SP with I1 = I0 reproduces I0
    assert np.abs(ol.sp_solve(I0, I0, 0.05) - I0).max() < 1e-9
    # a z-constant stack is a fixed point of AD (Kz annihilates it)
    zc = np.repeat(I0[:1], 4, axis=0)
    assert np.abs(ol.ad(zc, 1.0, 1.0, 10.0) - zc).max() < 1e-7
    # a wrong mass (the identity: the Constant operator) is detected by the residual
    I1 = ol.ad(I0, 1.0, 1.0, 10.0)
    from oracle import closed_form as cf
    wrong = cf.ad(I0, 1.0, 1.0, 10.0)
    A = ol.operator(I0.shape, 0.0, 1.0, 1.0, 10.0)
    assert ol.rel_residual(A, ol.rhs_ad(I0), wrong) > 1e-3
    assert ol.rel_residual(A, ol.rhs_ad(I0), I1) < 1e-11


@pytest.mark.parametrize("shape,bz", [((5, 7, 9), 10.0), ((1, 6, 11), 1.0), ((4, 1, 8), 0.1), ((3, 10, 4), 2.0)])
def test_fast_diagonalisation_equals_the_sparse_solves(shape, bz):
    """ad_fdm / sp_fdm (per-axis generalised eigenpairs) against the sparse
    CG and direct solves of the assembled Kronecker systems, ragged shapes
    and one-node axes included."""
    rng = np.random.default_rng(sum(shape))
    I0 = rng.uniform(0, 255, size=shape)
    I1 = rng.uniform(0, 255, size=shape)
    a = ol.ad_fdm(I0, 1.0, 1.3, bz)
    b = ol.ad(I0, 1.0, 1.3, bz)
    assert np.abs(a - b).max() <= 1e-8 * np.abs(b).max()
    assert abs(a.sum() - I0.sum()) <= 1e-8 * abs(I0.sum())
    c = ol.sp_fdm(I0, I1, 0.05)
    d = ol.sp_solve(I0, I1, 0.05)
    assert np.abs(c - d).max() <= 1e-8 * np.abs(d).max()
