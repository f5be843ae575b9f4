"""The Hybrid discretisation (Sec. 4.2): same 6-point fine system as the
Constant one, first-order B-spline transfers and Galerkin 27-point coarse
operators.  Its converged answers must be the exact discrete solutions (the
DCT closed form of the oracle), and its V-cycle must converge."""
import numpy as np
import pytest

import gdsynth
from oracle import closed_form as cf
import paper_1310_0041_gb300 as gd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no GPU")
    gd.build()
    return t


def run(torch, shape, disc, bz=10.0, alpha=0.01, tol_ad=1e-8, tol_sp=1e-9):
    nz, ny, nx = shape
    I0h = gdsynth.em_stack(nx, ny, nz, seed=17 + nz).astype(np.float32)
    I0 = torch.from_numpy(I0h).cuda()
    I1, I2 = torch.empty_like(I0), torch.empty_like(I0)
    s = gd.gd_stack_create(nx, ny, nz, disc=disc)
    try:
        r1 = gd.gd_diffuse_z(s, I0, I1, (0.0, 1.0, 1.0, bz), gd.solve_ctl(60, tol_ad))
        r2 = gd.gd_screened_poisson_slices(s, I0, I1, I2, alpha, gd.solve_ctl(60, tol_sp))
    finally:
        gd.gd_destroy(s)
    return I0h.astype(np.float64), I1.cpu().numpy().astype(np.float64), I2.cpu().numpy().astype(np.float64), r1, r2


@pytest.mark.parametrize("shape,bz", [((16, 64, 64), 10.0), ((11, 29, 37), 10.0), ((8, 96, 72), 0.1),
                                      ((1, 70, 52), 10.0), ((24, 40, 36), 1.0),
                                      # tile seams in x and y with ragged last tiles, odd nz
                                      ((9, 70, 150), 10.0)])
def test_hybrid_matches_exact_solutions(torch, shape, bz):
    I0, I1, I2, r1, r2 = run(torch, shape, gd.GD_DISC_HYBRID, bz=bz)
    assert r1["status"] == gd.GD_OK and r2["status"] == gd.GD_OK, (r1, r2)
    want1 = cf.ad(I0, 1.0, 1.0, bz)
    assert np.abs(I1 - want1).max() <= 1e-3
    want2 = cf.sp(I0, I1, 0.01)
    assert np.abs(I2 - want2).max() <= 1e-3


def test_hybrid_converges_faster_than_constant(torch):
    shape = (32, 128, 128)
    _, _, _, h1, h2 = run(torch, shape, gd.GD_DISC_HYBRID, tol_ad=1e-7, tol_sp=1e-7)
    _, _, _, c1, c2 = run(torch, shape, gd.GD_DISC_CONSTANT, tol_ad=1e-7, tol_sp=1e-7)
    assert h1["status"] == gd.GD_OK and h2["status"] == gd.GD_OK
    # the Galerkin hierarchy with B-spline transfers needs no more cycles
    assert h1["cycles"] <= c1["cycles"] and h2["cycles"] <= c2["cycles"], (h1, c1, h2, c2)
    assert h1["rho_per_cycle"] < 0.2 and h2["rho_per_cycle"] < 0.2, (h1, h2)


def test_hybrid_mixed_precision_is_unsupported(torch):
    with pytest.raises(gd.GdError) as ei:
        gd.gd_stack_create(32, 32, 4, disc=gd.GD_DISC_HYBRID, prec=gd.GD_PREC_MIXED)
    assert ei.value.status == gd.GD_ERR_UNSUPPORTED
