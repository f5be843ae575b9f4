"""Pins of the NPR oracle (paper Sec. 7): the filtered right-hand side and the
exact solve of the general screened Poisson system of Sec. 4."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import npr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "npr_1d_3.txt")


def load_golden():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            rows[k] = np.array([float(t) for t in v])
    return rows


def test_hand_worked_line():
    g = load_golden()
    I0 = g["I0"].reshape(1, 1, 3)
    sigma = math.sqrt(4.5 / math.log(2.0))
    b = npr.npr_rhs(I0, alpha=0.5, wx=1.0, wy=1.0, wz=1.0, lam=3.0, sigma=sigma)
    np.testing.assert_allclose(b.ravel(), g["b"], atol=1e-12)
    x = npr.screened(b, 0.5, 1.0, 1.0, 1.0)
    np.testing.assert_allclose(x.ravel(), g["x"], atol=1e-12)


@pytest.mark.parametrize("shape", [(3, 4, 5), (2, 7, 3), (1, 5, 6)])
def test_vectorised_equals_face_loops(shape):
    rng = np.random.default_rng(sum(shape))
    I0 = rng.integers(0, 256, shape).astype(np.float64)
    a = npr.npr_rhs(I0, 0.001, 1.0, 0.7, 0.1, 1.25, 5.0)
    b = npr.npr_loops(I0, 0.001, 1.0, 0.7, 0.1, 1.25, 5.0)
    np.testing.assert_allclose(a, b, atol=1e-10)


def test_sharp_limit_is_the_scaled_operator():
    """sigma -> 0: every nonzero gradient is scaled by lambda, so
    b = alpha I0 + lambda (wx Kx + wy Ky + wz Kz) I0 (the C oracle's operator)."""
    rng = np.random.default_rng(3)
    I0 = rng.integers(0, 256, (4, 6, 7)).astype(np.float64)
    b = npr.npr_rhs(I0, 0.01, 1.0, 0.5, 0.1, 1.25, 1e-6)
    want = 0.01 * I0 + 1.25 * oracle.apply(I0, 0.0, 1.0, 0.5, 0.1)
    np.testing.assert_allclose(b, want, atol=1e-9)


def test_zero_amplitude_and_flat_limits():
    rng = np.random.default_rng(4)
    I0 = rng.integers(0, 256, (3, 5, 6)).astype(np.float64)
    np.testing.assert_allclose(npr.npr_rhs(I0, 0.01, 1, 1, 0.1, 0.0, 5.0), 0.01 * I0, atol=1e-12)
    # sigma far above every gradient: the modulation ~ lambda |g|^2 / 2 sigma^2 -> 0
    np.testing.assert_allclose(npr.npr_rhs(I0, 0.01, 1, 1, 0.1, 1.25, 1e7), 0.01 * I0, atol=1e-6)


def test_divergence_sums_to_zero():
    """sum b = alpha sum I0 (Neumann: the divergence of any face field sums to 0),
    hence the solution keeps the mean of I0."""
    rng = np.random.default_rng(5)
    I0 = rng.integers(0, 256, (5, 9, 8)).astype(np.float64)
    b = npr.npr_rhs(I0, 0.001, 1, 1, 0.1, 1.25, 5.0)
    assert abs(b.sum() - 0.001 * I0.sum()) <= 1e-9 * abs(I0.sum())
    x = npr.screened(b, 0.001, 1, 1, 0.1)
    assert abs(x.mean() - I0.mean()) <= 1e-8 * I0.mean()


def test_screened_closed_form_vs_conjugate_gradients():
    rng = np.random.default_rng(6)
    b = rng.normal(0, 10, (5, 6, 7))
    x = npr.screened(b, 0.05, 1.0, 0.8, 0.3)
    y, _ = oracle.cg(b, np.zeros_like(b), 0.05, 1.0, 0.8, 0.3, tol=1e-13)
    np.testing.assert_allclose(x, y, atol=1e-8)
