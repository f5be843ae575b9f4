"""The Linear discretisation (Sec. 4.2, trilinear finite elements) on the GPU
against its FP64 oracle (oracle/linear.py): both steps, element by element,
on cubes, ragged and single-slice stacks."""
import numpy as np
import pytest

import gdsynth
import oracle.linear as ol
import paper_1310_0041_gb300 as gd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no GPU")
    gd.build()
    return t


@pytest.mark.parametrize("shape,bz", [((12, 40, 48), 10.0), ((7, 29, 37), 10.0), ((6, 33, 20), 0.1),
                                      ((1, 45, 52), 10.0), ((16, 64, 64), 1.0),
                                      # three 64-column tiles with a ragged third (and three
                                      # 32-row tiles, ragged), an odd plane count: the fused
                                      # sweep's recompute rings across tile seams
                                      ((9, 70, 150), 10.0)])
def test_linear_matches_oracle(torch, shape, bz):
    nz, ny, nx = shape
    I0h = gdsynth.em_stack(nx, ny, nz, seed=23 + nz).astype(np.float32)
    I0 = torch.from_numpy(I0h).cuda()
    I1, I2 = torch.empty_like(I0), torch.empty_like(I0)
    s = gd.gd_stack_create(nx, ny, nz, disc=gd.GD_DISC_LINEAR)
    try:
        r1 = gd.gd_diffuse_z(s, I0, I1, (0.0, 1.0, 1.0, bz), gd.solve_ctl(60, 1e-9))
        r2 = gd.gd_screened_poisson_slices(s, I0, I1, I2, 0.01, gd.solve_ctl(60, 1e-9))
    finally:
        gd.gd_destroy(s)
    assert r1["status"] == gd.GD_OK and r2["status"] == gd.GD_OK, (r1, r2)
    for r in (r1, r2):  # (a single slice is its own AD answer and SP then starts converged)
        assert r["cycles"] == 0 or r["rho_per_cycle"] < 0.3, (r1, r2)
    I0d = I0h.astype(np.float64)
    got1 = I1.cpu().numpy().astype(np.float64)
    want1 = ol.ad(I0d, 1.0, 1.0, bz)
    assert np.abs(got1 - want1).max() <= 1e-3
    assert abs(got1.mean() - I0d.mean()) <= 1e-4
    got2 = I2.cpu().numpy().astype(np.float64)
    want2 = ol.sp_solve(I0d, got1, 0.01)
    assert np.abs(got2 - want2).max() <= 1e-3


def test_linear_differs_from_constant(torch):
    # a different fine system: the answers differ by much more than the tolerance
    nz, ny, nx = 8, 32, 32
    I0h = gdsynth.em_stack(nx, ny, nz, seed=5).astype(np.float32)
    outs = []
    for disc in (gd.GD_DISC_CONSTANT, gd.GD_DISC_LINEAR):
        I0 = torch.from_numpy(I0h).cuda()
        I1 = torch.empty_like(I0)
        s = gd.gd_stack_create(nx, ny, nz, disc=disc)
        try:
            gd.gd_diffuse_z(s, I0, I1, (0.0, 1.0, 1.0, 10.0), gd.solve_ctl(60, 1e-9))
        finally:
            gd.gd_destroy(s)
        outs.append(I1.cpu().numpy())
    assert np.abs(outs[0] - outs[1]).max() > 0.1


def test_linear_kernel_level_calls_are_unsupported(torch):
    s = gd.gd_stack_create(16, 16, 4, disc=gd.GD_DISC_LINEAR)
    try:
        z = torch.zeros(16 * 16 * 4, device="cuda")
        x = torch.zeros_like(z)
        with pytest.raises(gd.GdError) as ei:
            gd.gd_smooth(s, (0.0, 1.0, 1.0, 1.0), z, x, 1)
        assert ei.value.status == gd.GD_ERR_UNSUPPORTED
    finally:
        gd.gd_destroy(s)


def test_linear_at_256x256x32(torch):
    """Both steps on a 256 x 256 x 32 stack (2.1 M unknowns of the 27-point
    system) against the oracle's fast-diagonalisation solves."""
    nz, ny, nx = 32, 256, 256
    I0h = gdsynth.em_stack(nx, ny, nz, seed=41).astype(np.float32)
    I0 = torch.from_numpy(I0h).cuda()
    I1, I2 = torch.empty_like(I0), torch.empty_like(I0)
    s = gd.gd_stack_create(nx, ny, nz, disc=gd.GD_DISC_LINEAR)
    try:
        r1 = gd.gd_diffuse_z(s, I0, I1, (0.0, 1.0, 1.0, 10.0), gd.solve_ctl(60, 1e-9))
        r2 = gd.gd_screened_poisson_slices(s, I0, I1, I2, 0.01, gd.solve_ctl(60, 1e-9))
    finally:
        gd.gd_destroy(s)
    assert r1["status"] == gd.GD_OK and r2["status"] == gd.GD_OK, (r1, r2)
    I0d = I0h.astype(np.float64)
    got1 = I1.cpu().numpy().astype(np.float64)
    assert np.abs(got1 - ol.ad_fdm(I0d, 1.0, 1.0, 10.0)).max() <= 1e-3
    got2 = I2.cpu().numpy().astype(np.float64)
    assert np.abs(got2 - ol.sp_fdm(I0d, got1, 0.01)).max() <= 1e-3
