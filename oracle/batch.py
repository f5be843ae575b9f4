"""Screened Poisson on a batch of independent slices of different sizes --
TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle``).

Slice s, of nx_s x ny_s cells with its own screening weight alpha_s, solves
the per-slice system of Sec. 3.1 (Eq. screened_poisson) with the 6-point
Neumann stencil of Sec. 4.2:

    (alpha_s + Kx + Ky) I2_s = alpha_s I1_s + (Kx + Ky) I0_s.

The slices share nothing, so the batch answer is the per-slice answer: each
slice goes through the oracle's exact routes for one 2D slice (the DCT closed
form, and the plain FP64 loops for the right-hand side, the operator and the
residual).  Nothing here depends on how the batch is laid out in memory.
"""
from __future__ import annotations

import numpy as np

from . import closed_form
from . import rhs_sp, apply, rel_residual


def _as_stack(a) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64)
    return a.reshape((1,) + a.shape)


def sp_slice(I0, I1, alpha: float) -> np.ndarray:
    """Exact I2 of one ``[ny][nx]`` slice (DCT closed form)."""
    return closed_form.sp(_as_stack(I0), _as_stack(I1), alpha)[0]


def sp_batch(I0s, I1s, alphas) -> list:
    """Exact I2 of every slice of the batch."""
    return [sp_slice(a, b, al) for a, b, al in zip(I0s, I1s, alphas)]


def rhs_slice(I0, I1, alpha: float) -> np.ndarray:
    """alpha I1 + (Kx + Ky) I0 of one slice (plain FP64 loops)."""
    return rhs_sp(_as_stack(I0), _as_stack(I1), alpha)[0]


def apply_slice(x, alpha: float) -> np.ndarray:
    """(alpha + Kx + Ky) x of one slice (plain FP64 loops)."""
    return apply(_as_stack(x), alpha, 1.0, 1.0, 0.0)[0]


def rel_residual_slice(I0, I1, alpha: float, x) -> float:
    """||b - A x|| / ||b|| of one slice, b = alpha I1 + (Kx + Ky) I0."""
    b = rhs_sp(_as_stack(I0), _as_stack(I1), alpha)
    return rel_residual(b, _as_stack(x), alpha, 1.0, 1.0, 0.0)
