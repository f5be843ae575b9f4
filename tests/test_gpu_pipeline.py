"""gd_ad_then_sp: the two steps in one call give the same I1 and I2 as the
two separate calls, from device and from host arrays."""
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


def test_ad_then_sp_matches_separate_calls(torch):
    nz, ny, nx = 12, 72, 80
    I0h = gdsynth.em_stack(nx, ny, nz, seed=41).astype(np.float32)
    w = (0.0, 1.0, 1.0, 10.0)
    ca, cs = gd.solve_ctl(40, 1e-8), gd.solve_ctl(40, 1e-9)
    s = gd.gd_stack_create(nx, ny, nz)
    try:
        I0 = torch.from_numpy(I0h).cuda()
        I1, I2 = torch.empty_like(I0), torch.empty_like(I0)
        r1 = gd.gd_diffuse_z(s, I0, I1, w, ca)
        r2 = gd.gd_screened_poisson_slices(s, I0, I1, I2, 0.01, cs)
        # device arrays, I1 returned
        J1, J2 = torch.empty_like(I0), torch.empty_like(I0)
        q1, q2 = gd.gd_ad_then_sp(s, I0, J2, w, 0.01, ca, cs, I1=J1)
        # host arrays, I1 kept inside
        H2 = np.zeros_like(I0h)
        h1, h2 = gd.gd_ad_then_sp(s, I0h, H2, w, 0.01, ca, cs)
    finally:
        gd.gd_destroy(s)
    assert q1["cycles"] == r1["cycles"] and q2["cycles"] == r2["cycles"]
    assert torch.equal(J1, I1) and torch.equal(J2, I2)
    np.testing.assert_array_equal(H2, I2.cpu().numpy())
    want2 = cf.sp(I0h.astype(np.float64), I1.cpu().numpy().astype(np.float64), 0.01)
    assert np.abs(H2 - want2).max() <= 1e-3


def test_ad_then_sp_validation(torch):
    s = gd.gd_stack_create(16, 16, 4)
    try:
        a = torch.zeros(16 * 16 * 4, device="cuda")
        for args in ((a, a, (0.0, 1.0, 1.0, 1.0), 0.01), (a, torch.empty_like(a), (0.0, 1.0, 1.0, 1.0), 0.0)):
            with pytest.raises(gd.GdError) as ei:
                gd.gd_ad_then_sp(s, *args)
            assert ei.value.status == gd.GD_ERR_INVALID_ARG
    finally:
        gd.gd_destroy(s)
