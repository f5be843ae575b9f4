"""The 4096 x 4096 x 256 workload (4.3 G voxels, 17.2 GB per float32 array),
where the mixed-precision mode is specified: AD (beta_z = 10) to 1e-6 then
SP (alpha = 0.01) to 1e-7, in the float32 and the mixed mode.

The host cannot hold FP64 copies of the whole stack for the closed form, so
the full-size check is (a) each solve's own residual, accumulated in FP64
over the whole stack, at its tolerance, (b) the two modes' answers within
1e-3 of each other everywhere (each is within ~5e-4 of the exact one at these
tolerances), and (c) a 1024 x 1024 x 64 crop of the same stack, solved as its
own problem in the mixed mode, within 1e-3 of the DCT closed form."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NX, NY, NZ = 4096, 4096, 256
W_AD = (0.0, 1.0, 1.0, 10.0)


def test_config3_float32_and_mixed():
    import torch
    import gdsynth
    import paper_1310_0041_gb300 as gd
    from oracle import closed_form as cf
    gd.build()
    gdsynth.build_cuda()
    I0 = gdsynth.em_stack_cuda(NX, NY, NZ, seed=3).float()
    res = {}
    outs = {}
    for prec in (gd.GD_PREC_FP32, gd.GD_PREC_MIXED):
        I1 = torch.empty_like(I0)
        I2 = torch.empty_like(I0)
        s = gd.gd_stack_create(NX, NY, NZ, prec=prec)
        try:
            r1 = gd.gd_diffuse_z(s, I0, I1, W_AD, gd.solve_ctl(30, 1e-6))
            r2 = gd.gd_screened_poisson_slices(s, I0, I1, I2, 0.01, gd.solve_ctl(30, 1e-7))
        finally:
            gd.gd_destroy(s)
        torch.cuda.synchronize()
        res[prec] = (r1, r2)
        outs[prec] = (I1, I2)
        assert r1["status"] == gd.GD_OK and r1["rel_residual"] <= 1e-6, r1
        assert r2["status"] == gd.GD_OK and r2["rel_residual"] <= 1e-7, r2
    (a1, a2), (b1, b2) = outs[gd.GD_PREC_FP32], outs[gd.GD_PREC_MIXED]
    assert (a1 - b1).abs().max().item() <= 1e-3
    assert (a2 - b2).abs().max().item() <= 1e-3
    del a1, a2, b1, b2, outs, I0
    torch.cuda.empty_cache()
    # a crop solved as its own problem, against the closed form
    win = (1536, 1024, 96, 1024, 1024, 64)
    C0 = gdsynth.em_stack_cuda(NX, NY, NZ, seed=3, window=win).float()
    C1, C2 = torch.empty_like(C0), torch.empty_like(C0)
    s = gd.gd_stack_create(win[3], win[4], win[5], prec=gd.GD_PREC_MIXED)
    try:
        gd.gd_diffuse_z(s, C0, C1, W_AD, gd.solve_ctl(30, 1e-6))
        gd.gd_screened_poisson_slices(s, C0, C1, C2, 0.01, gd.solve_ctl(30, 1e-7))
    finally:
        gd.gd_destroy(s)
    c0 = C0.cpu().numpy().astype(np.float64)
    g1 = C1.cpu().numpy().astype(np.float64)
    assert np.abs(g1 - cf.ad(c0, 1.0, 1.0, 10.0)).max() <= 1e-3
    g2 = C2.cpu().numpy().astype(np.float64)
    assert np.abs(g2 - cf.sp(c0, g1, 0.01)).max() <= 1e-3
