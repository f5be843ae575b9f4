"""NPR gradient filter (Sec. 7) and the general screened Poisson solve on the
GPU against the FP64 oracle (oracle/npr.py): the filtered right-hand side
element by element, and the solution against the exact DCT solve."""
import math

import numpy as np
import pytest

import gdsynth
from oracle import npr
import paper_1310_0041_gb300 as gd

pytestmark = pytest.mark.gpu

W_VIDEO = (0.001, 1.0, 1.0, 0.1)  # alpha, W = Diag(1, 1, 0.1) of the paper's video example


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no GPU")
    gd.build()
    return t


def frames(nx, ny, nz, seed):
    # moving Voronoi cells along z (= time): a video-like synthetic stack
    return gdsynth.em_stack(nx, ny, nz, seed=seed, ncells=max(8, nx * ny // 524)).astype(np.float64)


@pytest.mark.parametrize("shape,lam,sigma", [((8, 24, 40), 1.25, 5.0), ((5, 17, 33), 1.25, 5.0),
                                             ((6, 20, 36), 3.0, 0.5), ((1, 30, 28), 1.25, 5.0)])
def test_npr_rhs_matches_oracle(torch, shape, lam, sigma):
    nz, ny, nx = shape
    I0 = frames(nx, ny, nz, seed=41 + nz)
    s = gd.gd_stack_create(nx, ny, nz)
    try:
        x = torch.from_numpy(I0.astype(np.float32)).cuda()
        b = torch.empty_like(x)
        gd.gd_npr_rhs(s, x, b, W_VIDEO, lam, sigma)
        got = b.cpu().numpy().astype(np.float64)
    finally:
        gd.gd_destroy(s)
    want = npr.npr_rhs(I0, *W_VIDEO, lam=lam, sigma=sigma)
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max() + 1e-4


def test_npr_rhs_host_arrays(torch):
    nz, ny, nx = 4, 12, 20
    I0 = frames(nx, ny, nz, seed=50).astype(np.float32)
    s = gd.gd_stack_create(nx, ny, nz)
    try:
        b = np.zeros_like(I0)
        gd.gd_npr_rhs(s, I0, b, W_VIDEO, 1.25, 5.0)
    finally:
        gd.gd_destroy(s)
    want = npr.npr_rhs(I0.astype(np.float64), *W_VIDEO, lam=1.25, sigma=5.0)
    assert np.abs(b - want).max() <= 1e-5 * np.abs(want).max() + 1e-4


@pytest.mark.parametrize("shape", [(16, 64, 64), (12, 40, 72), (24, 96, 128)])
def test_npr_filter_solution(torch, shape):
    """b from the GPU kernel, x from gd_screened_poisson: max |x - exact| <= 1e-3
    (0..255 scale), the exact x being the FP64 DCT solve of the oracle's b.
    alpha = 0.001 magnifies smooth error ~1000x, hence the tight tolerance."""
    nz, ny, nx = shape
    I0 = frames(nx, ny, nz, seed=60 + nz)
    s = gd.gd_stack_create(nx, ny, nz)
    try:
        xi = torch.from_numpy(I0.astype(np.float32)).cuda()
        b = torch.empty_like(xi)
        out = torch.empty_like(xi)
        gd.gd_npr_rhs(s, xi, b, W_VIDEO, 1.25, 5.0)
        rep = gd.gd_screened_poisson(s, W_VIDEO, b, out, gd.solve_ctl(40, 1e-9), x0=xi)
        got = out.cpu().numpy().astype(np.float64)
    finally:
        gd.gd_destroy(s)
    assert rep["status"] == gd.GD_OK and rep["rel_residual"] <= 1e-9, rep
    want = npr.screened(npr.npr_rhs(I0, *W_VIDEO, lam=1.25, sigma=5.0), W_VIDEO[0], *W_VIDEO[1:])
    assert np.abs(got - want).max() <= 1e-3


@pytest.mark.parametrize("w", [(0.05, 1.0, 0.7, 0.0), (0.01, 1.0, 1.0, 3.0), (2.0, 0.5, 1.5, 0.2)])
def test_general_solve_explicit_rhs(torch, w):
    nz, ny, nx = 10, 36, 52
    rng = np.random.default_rng(70)
    b = rng.normal(0.0, 20.0, (nz, ny, nx))
    s = gd.gd_stack_create(nx, ny, nz)
    try:
        bt = torch.from_numpy(b.astype(np.float32)).cuda()
        out = torch.empty_like(bt)
        rep = gd.gd_screened_poisson(s, w, bt, out, gd.solve_ctl(40, 1e-9))
        got = out.cpu().numpy().astype(np.float64)
    finally:
        gd.gd_destroy(s)
    assert rep["status"] == gd.GD_OK
    want = npr.screened(b.astype(np.float32).astype(np.float64), w[0], *w[1:])
    assert np.abs(got - want).max() <= 1e-3 * max(1.0, np.abs(want).max() / 255.0)
