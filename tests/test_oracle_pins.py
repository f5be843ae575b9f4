"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here uses the CUDA path.  Each pin is chosen so that a plausible slip
in the oracle (a dropped term, a wrong sign, a swapped axis, a wrong boundary
row, a wrong transfer) fails at least one test:

* hand-worked fixtures from the frequency-space formulas of Sec. 3.2
  (tests/golden/);
* the DCT closed form (exact for the 6-point Neumann operator) against a dense
  solve of the Kronecker-assembled matrix built here from 1D matrices;
* the oracle's C solvers (dense, CG, V-cycle) against both;
* invariants the paper states or implies: self-reproduction, z-constant
  stacks, mean preservation, the limits of Sec. 3.2, and the aliasing example
  of Fig. 2.
"""
import numpy as np
import pytest

import gdsynth
import oracle
from oracle import closed_form as cf
from golden_io import load


# ----------------------------------------------------------------------------
# independent constructions used as references
# ----------------------------------------------------------------------------
def K1(n):
    """1D Neumann Laplacian as a matrix, from its quadratic form sum (u_{i+1}-u_i)^2."""
    K = np.zeros((n, n))
    for i in range(n - 1):
        e = np.zeros(n)
        e[i], e[i + 1] = -1.0, 1.0
        K += np.outer(e, e)
    return K


def kron_A(shape, alpha, bx, by, bz):
    """alpha I + bx Kx + by Ky + bz Kz on x-fastest vectors (z slowest)."""
    nz, ny, nx = shape
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    A = bx * np.kron(Iz, np.kron(Iy, K1(nx)))
    A += by * np.kron(Iz, np.kron(K1(ny), Ix))
    A += bz * np.kron(K1(nz), np.kron(Iy, Ix))
    A += alpha * np.eye(nx * ny * nz)
    return A


def kron_ad(I0, bx, by, bz):
    shape = I0.shape
    A = kron_A(shape, 0.0, bx, by, bz)
    b = kron_A(shape, 0.0, bx, by, 0.0) @ I0.ravel()
    x = np.linalg.lstsq(A, b, rcond=None)[0]
    x += I0.mean() - x.mean()
    return x.reshape(shape)


def kron_sp(I0, I1, alpha):
    out = np.empty(I0.shape)
    for k in range(I0.shape[0]):
        s = (1,) + I0.shape[1:]
        A = kron_A(s, alpha, 1.0, 1.0, 0.0)
        b = alpha * I1[k].ravel() + kron_A(s, 0.0, 1.0, 1.0, 0.0) @ I0[k].ravel()
        out[k] = np.linalg.solve(A, b).reshape(I0.shape[1:])
    return out


def rng_stack(shape, seed):
    return np.random.default_rng(seed).uniform(0, 255, size=shape)


# ----------------------------------------------------------------------------
# hand-worked fixtures
# ----------------------------------------------------------------------------
def test_golden_ad_2x1x2():
    g = load("ad_2x1x2.txt")
    shape = (int(g["nz"]), int(g["ny"]), int(g["nx"]))
    I0 = np.array(g["I0"]).reshape(shape)
    want = np.array(g["I1"]).reshape(shape)
    for method in ("dense", "cg", "mg"):
        got, _ = oracle.ad_solve(I0, g["bx"], g["by"], g["bz"], method=method, tol=1e-14)
        np.testing.assert_allclose(got, want, atol=1e-11, err_msg=method)
    np.testing.assert_allclose(cf.ad(I0, g["bx"], g["by"], g["bz"]), want, atol=1e-11)


def test_golden_sp_2x2():
    g = load("sp_2x2.txt")
    shape = (int(g["nz"]), int(g["ny"]), int(g["nx"]))
    I0 = np.array(g["I0"]).reshape(shape)
    I1 = np.array(g["I1"]).reshape(shape)
    want = np.array(g["I2"]).reshape(shape)
    for method in ("dense", "cg", "mg"):
        got, _ = oracle.sp_solve(I0, I1, g["alpha"], method=method, tol=1e-14)
        np.testing.assert_allclose(got, want, atol=1e-11, err_msg=method)
    np.testing.assert_allclose(cf.sp(I0, I1, g["alpha"]), want, atol=1e-11)


def test_golden_aliasing_1d():
    g = load("aliasing_1d.txt")
    s = np.array(g["signal"]).reshape(1, 1, -1)
    c = oracle.apply(s, 0.0, 1.0, 0.0, 0.0)
    np.testing.assert_array_equal(c.ravel(), g["constraints"])
    cc = oracle.restrict(c, 1, 0, 0)
    np.testing.assert_array_equal(cc.ravel(), g["coarse"])
    y = oracle.dense(cc, 0.0, 1.0, 0.0, 0.0)
    y -= y.mean()
    np.testing.assert_allclose(y.ravel(), g["coarse_solution"], atol=1e-13)
    up = oracle.prolong_add(y, np.zeros_like(s), 1, 0, 0)
    np.testing.assert_allclose(up.ravel(), g["upsampled"], atol=1e-13)
    # the coarse solution has the drop but no rise
    assert np.all(np.diff(y.ravel()) <= 1e-13)


# ----------------------------------------------------------------------------
# closed form vs dense Kronecker solve (no oracle C code involved)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(8, 8, 8), (5, 9, 7), (3, 4, 6)])
@pytest.mark.parametrize("w", [(1.0, 1.0, 10.0), (1.0, 1.0, 0.1), (1.0, 2.5, 0.7)])
def test_closed_form_ad_vs_kron(shape, w):
    I0 = rng_stack(shape, 1)
    np.testing.assert_allclose(cf.ad(I0, *w), kron_ad(I0, *w), atol=1e-9)


@pytest.mark.parametrize("shape", [(3, 8, 8), (2, 9, 7)])
@pytest.mark.parametrize("alpha", [0.01, 0.5])
def test_closed_form_sp_vs_kron(shape, alpha):
    I0, I1 = rng_stack(shape, 2), rng_stack(shape, 3)
    np.testing.assert_allclose(cf.sp(I0, I1, alpha), kron_sp(I0, I1, alpha), atol=1e-9)


def test_neumann_eigenvalues_match_matrix():
    for n in (1, 2, 5, 16):
        np.testing.assert_allclose(np.sort(cf.neumann_eigenvalues(n)), np.linalg.eigvalsh(K1(n)), atol=1e-12)


# ----------------------------------------------------------------------------
# the oracle's C code against the independent references
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(5, 9, 7), (1, 6, 4), (4, 1, 3)])
def test_oracle_apply_vs_kron(shape):
    x = rng_stack(shape, 4)
    for w in [(0.0, 1.0, 2.0, 3.0), (0.3, 1.0, 1.0, 0.0), (0.0, 1.0, 1.0, 10.0)]:
        A = kron_A(shape, *w)
        np.testing.assert_allclose(oracle.apply(x, *w).ravel(), A @ x.ravel(), rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("shape", [(5, 9, 7), (8, 8, 8)])
def test_oracle_rhs_vs_kron(shape):
    I0, I1 = rng_stack(shape, 5), rng_stack(shape, 6)
    bxy = kron_A(shape, 0.0, 1.3, 0.6, 0.0) @ I0.ravel()
    np.testing.assert_allclose(oracle.rhs_ad(I0, 1.3, 0.6).ravel(), bxy, rtol=1e-12, atol=1e-9)
    bsp = 0.05 * I1.ravel() + kron_A(shape, 0.0, 1.0, 1.0, 0.0) @ I0.ravel()
    np.testing.assert_allclose(oracle.rhs_sp(I0, I1, 0.05).ravel(), bsp, rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("w", [(1.0, 1.0, 10.0), (1.0, 1.0, 0.1), (2.0, 0.5, 1.0)])
def test_oracle_dense_and_cg_8cubed(w):
    I0 = rng_stack((8, 8, 8), 7)
    ref = kron_ad(I0, *w)
    d, _ = oracle.ad_solve(I0, *w, method="dense")
    np.testing.assert_allclose(d, ref, atol=1e-8)
    c, info = oracle.ad_solve(I0, *w, method="cg", tol=1e-13)
    np.testing.assert_allclose(c, ref, atol=1e-8)


@pytest.mark.parametrize("bz", [10.0, 0.1])
def test_oracle_mg_cg_config1_vs_closed_form(bz):
    """64x64x16 synthetic stack (the oracle-size workload), both z weights."""
    I0 = gdsynth.em_stack(64, 64, 16, seed=11).astype(np.float64)
    ref = cf.ad(I0, 1.0, 1.0, bz)
    x, info = oracle.ad_solve(I0, 1.0, 1.0, bz, method="mg", tol=1e-11, max_cycles=400)
    assert info["status"] == 0
    np.testing.assert_allclose(x, ref, atol=1e-6)
    y, _ = oracle.ad_solve(I0, 1.0, 1.0, bz, method="cg", tol=1e-12)
    np.testing.assert_allclose(y, ref, atol=1e-7)
    # the closed form satisfies the oracle's own residual definition
    b = oracle.rhs_ad(I0, 1.0, 1.0)
    assert oracle.rel_residual(b, ref, 0.0, 1.0, 1.0, bz) < 1e-12
    # V-cycle residuals decrease every cycle
    h = info["history"]
    assert np.all(np.diff(h) < 0)


def test_oracle_sp_config1_vs_closed_form():
    I0 = gdsynth.em_stack(64, 64, 16, seed=12).astype(np.float64)
    I1 = cf.ad(I0, 1.0, 1.0, 10.0)
    ref = cf.sp(I0, I1, 0.01)
    x, info = oracle.sp_solve(I0, I1, 0.01, method="mg", tol=1e-12)
    np.testing.assert_allclose(x, ref, atol=1e-7)
    b = oracle.rhs_sp(I0, I1, 0.01)
    assert oracle.rel_residual(b, ref, 0.01, 1.0, 1.0, 0.0) < 1e-12


# ----------------------------------------------------------------------------
# invariants (Sec. 3.2 observations and consequences of the equations)
# ----------------------------------------------------------------------------
def test_self_reproduction_sp():
    """If I1 already has the target gradients (I1 = I0), SP returns I0."""
    I0 = gdsynth.em_stack(48, 40, 3, seed=13).astype(np.float64)
    for method in ("mg", "cg"):
        x, _ = oracle.sp_solve(I0, I0, 0.01, method=method, tol=1e-13)
        np.testing.assert_allclose(x, I0, atol=1e-8)
    np.testing.assert_allclose(cf.sp(I0, I0, 0.01), I0, atol=1e-9)


def test_z_constant_stack_passes_ad():
    sl = gdsynth.em_stack(40, 36, 1, seed=14).astype(np.float64)
    I0 = np.repeat(sl, 9, axis=0)
    for method in ("mg", "cg"):
        x, _ = oracle.ad_solve(I0, 1.0, 1.0, 10.0, method=method, tol=1e-13)
        np.testing.assert_allclose(x, I0, atol=1e-7)
    np.testing.assert_allclose(cf.ad(I0, 1.0, 1.0, 10.0), I0, atol=1e-9)


def test_means():
    I0 = gdsynth.em_stack(40, 36, 7, seed=15).astype(np.float64)
    I1, _ = oracle.ad_solve(I0, 1.0, 1.0, 10.0, method="cg", tol=1e-13)
    assert abs(I1.mean() - I0.mean()) < 1e-10
    # AD removes every slice-mean variation along z: all slice means equal the global mean
    np.testing.assert_allclose(I1.mean(axis=(1, 2)), I0.mean(), atol=1e-7)
    # SP keeps each slice mean of I1 (sum the rows: alpha sum I2 = alpha sum I1)
    I2, _ = oracle.sp_solve(I0, I1, 0.01, method="cg", tol=1e-13)
    np.testing.assert_allclose(I2.mean(axis=(1, 2)), I1.mean(axis=(1, 2)), atol=1e-7)


def test_limits_of_sec_3_2():
    I0 = gdsynth.em_stack(32, 32, 6, seed=16).astype(np.float64)
    # bz -> 0: no diffusion, the signal is unchanged -- except the modes with
    # no in-slice frequency (k = l = 0, m > 0), whose multiplier is 0 for any
    # bz > 0: each slice mean is replaced by the global mean
    x, _ = oracle.ad_solve(I0, 1.0, 1.0, 1e-9, method="cg", tol=1e-14)
    want = I0 - I0.mean(axis=(1, 2), keepdims=True) + I0.mean()
    np.testing.assert_allclose(x, want, atol=1e-4)
    # alpha -> 0: I2 takes I0's gradients and I1's slice means
    I1 = cf.ad(I0, 1.0, 1.0, 10.0)
    y = cf.sp(I0, I1, 1e-10)
    shift = (I1.mean(axis=(1, 2)) - I0.mean(axis=(1, 2)))[:, None, None]
    np.testing.assert_allclose(y, I0 + shift, atol=1e-5)
    z, _ = oracle.sp_solve(I0, I1, 1e-10, method="cg", tol=1e-15, maxit=20000)
    np.testing.assert_allclose(z, I0 + shift, atol=1e-3)
    # large in-slice frequencies pass the combined filter, low in-slice / high z are damped
    F = cf.combined_filter((16, 64, 64), 0.01, 1.0, 1.0, 10.0)
    assert F[15, 63, 63] > 0.99
    assert F[15, 0, 0] < 1e-6


def test_rb_sweep_invariant():
    """After one red-black sweep the black equations hold exactly; an exact
    solution is a fixed point of the sweep."""
    shape = (6, 11, 9)
    I0 = rng_stack(shape, 17)
    w = (0.02, 1.0, 1.5, 4.0)
    b = oracle.rhs_sp(I0, I0, 0.02)
    x0 = rng_stack(shape, 18)
    x1 = oracle.gs_sweeps(b, x0, *w, order="redblack", nsweeps=1)
    r = b - oracle.apply(x1, *w)
    k, j, i = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    black = (i + j + k) % 2 == 1
    assert np.abs(r[black]).max() < 1e-9 * np.abs(b).max()
    assert np.abs(r[~black]).max() > 1e-3
    xs = np.linalg.solve(kron_A(shape, *w), b.ravel()).reshape(shape)
    np.testing.assert_allclose(oracle.gs_sweeps(b, xs, *w, nsweeps=3), xs, atol=1e-9)
    # lexicographic: the last voxel's equation holds after the sweep
    xl = oracle.gs_sweeps(b, x0, *w, order="lex", nsweeps=1)
    rl = b - oracle.apply(xl, *w)
    assert abs(rl[-1, -1, -1]) < 1e-9 * np.abs(b).max()


def test_restrict_prolong_are_transposes():
    rng = np.random.default_rng(19)
    for shape in [(5, 7, 9), (4, 6, 8), (1, 3, 2)]:
        for f in [(1, 1, 1), (1, 1, 0), (0, 0, 1)]:
            r = rng.standard_normal(shape)
            rc = oracle.restrict(r, *f)
            e = rng.standard_normal(rc.shape)
            Pe = oracle.prolong_add(e, np.zeros(shape), *f)
            assert abs(np.sum(rc * e) - np.sum(r * Pe)) < 1e-10
            # P 1 = 1: replication keeps constants
            np.testing.assert_array_equal(oracle.prolong_add(np.ones(rc.shape), np.zeros(shape), *f), 1.0)
