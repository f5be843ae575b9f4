"""Mixed precision (bfloat16 storage of the multigrid levels, float32
arithmetic, float-pair outer refinement): the solves reach the same
tolerances and the same answers as the float32 mode, against the exact
discrete solutions (DCT closed form, FP64)."""
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


def solve_pair(torch, I0, bz, alpha, prec, tol_ad, tol_sp, max_cycles=30):
    nz, ny, nx = I0.shape
    s = gd.gd_stack_create(nx, ny, nz, prec=prec)
    try:
        x = torch.from_numpy(np.ascontiguousarray(I0, np.float32)).cuda()
        y = torch.empty_like(x)
        z = torch.empty_like(x)
        r1 = gd.gd_diffuse_z(s, x, y, (0.0, 1.0, 1.0, bz), gd.solve_ctl(max_cycles, tol_ad))
        r2 = gd.gd_screened_poisson_slices(s, x, y, z, alpha, gd.solve_ctl(max_cycles, tol_sp))
        return y.cpu().numpy().astype(np.float64), z.cpu().numpy().astype(np.float64), r1, r2
    finally:
        gd.gd_destroy(s)


@pytest.mark.parametrize("shape,bz", [((16, 64, 64), 10.0), ((16, 64, 64), 0.1), ((24, 96, 128), 10.0),
                                      ((32, 256, 256), 10.0)])
def test_mixed_matches_exact(torch, shape, bz):
    nz, ny, nx = shape
    I0 = gdsynth.em_stack(nx, ny, nz, seed=31, ncells=max(8, nx * ny // 524)).astype(np.float64)
    y, z, r1, r2 = solve_pair(torch, I0, bz, 0.01, gd.GD_PREC_MIXED, 1e-6, 1e-7)
    assert r1["status"] == gd.GD_OK and r1["rel_residual"] <= 1e-6, r1
    assert r2["status"] == gd.GD_OK and r2["rel_residual"] <= 1e-7, r2
    ref1 = cf.ad(I0, 1.0, 1.0, bz)
    ref2 = cf.sp(I0, y, 0.01)
    assert np.abs(y - ref1).max() <= 1e-3
    assert np.abs(z - ref2).max() <= 1e-3
    # the mean of the AD result is the mean of the input
    assert abs(y.mean() - I0.mean()) <= 1e-4


def test_mixed_costs_at_most_one_more_cycle(torch):
    I0 = gdsynth.em_stack(128, 96, 24, seed=32, ncells=24).astype(np.float64)
    _, _, f1, f2 = solve_pair(torch, I0, 10.0, 0.01, gd.GD_PREC_FP32, 1e-6, 1e-7)
    _, _, m1, m2 = solve_pair(torch, I0, 10.0, 0.01, gd.GD_PREC_MIXED, 1e-6, 1e-7)
    assert m1["cycles"] <= f1["cycles"] + 1, (f1["history"][:8], m1["history"][:8])
    assert m2["cycles"] <= f2["cycles"] + 1, (f2["history"][:8], m2["history"][:8])


def test_mixed_ragged_sizes_fall_back_to_float32(torch):
    """x extents that are not multiples of 8 keep float32 storage; the solve
    is still correct."""
    I0 = gdsynth.em_stack(68, 40, 9, seed=33, ncells=6).astype(np.float64)
    y, z, r1, r2 = solve_pair(torch, I0, 10.0, 0.01, gd.GD_PREC_MIXED, 1e-7, 1e-8)
    assert r1["status"] == gd.GD_OK and r2["status"] == gd.GD_OK
    assert np.abs(y - cf.ad(I0, 1.0, 1.0, 10.0)).max() <= 1e-3


def test_per_level_error_of_the_mixed_mode():
    """One V-cycle on a 512 x 512 x 64 crop of the 4096 x 4096 x 256 stack
    (solved as its own problem): the first coarse level's correction (modulo
    the AD operator's constants) differs from the float32-storage hierarchy's
    by at most 5 % RMS of its size and every level's by at most 30 % --
    bfloat16 keeps 8 significant bits, a coarse correction is a sum of
    nearly cancelling smoothing and coarser-grid terms, and each level
    inherits the finer ones' rounding; measured 3 % growing to 19 %; the two
    modes' fine residuals still agree to 0.1 % cycle by cycle -- and the coarsest
    level's float32 fast-diagonalisation solve is within 1e-5 of an FP64
    dense solve of the same system."""
    import torch
    import bench
    import gdsynth
    gdsynth.build_cuda()
    I0 = gdsynth.em_stack_cuda(4096, 4096, 256, seed=3, window=(1024, 2048, 96, 512, 512, 64)).float()
    rep = bench.mixed_level_errors(gd, torch, I0, (0.0, 1.0, 1.0, 10.0))
    print(rep)
    assert len(rep["levels"]) >= 3
    assert any(r["storage"] == "bf16" for r in rep["levels"])
    assert rep["levels"][0]["rel_rms_diff"] <= 5e-2, rep["levels"][0]
    for r in rep["levels"]:  # (float32 levels below bfloat16 ones inherit their rounding)
        assert r["rel_rms_diff"] <= 0.3 and r["rel_max_diff"] <= 0.3, r
    c = rep["coarsest"]
    assert c["rel_max_err_vs_fp64"] <= 1e-5 and c["rel_residual_fp32_solve"] <= 1e-5, c
