"""Failure detection on the GPU without faulting it: a bounded wait that
runs out (a barrier nothing arrives at), an allocation failure injected on
the host, and poisoned (NaN) input caught by the residual check.  After each
the context stays usable."""
import numpy as np
import pytest

import gdsynth
import paper_1310_0041_gb300 as gd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no GPU")
    gd.build()
    return t


def small_solve(torch):
    I0 = torch.from_numpy(gdsynth.em_stack(32, 32, 4, seed=1).astype(np.float32)).cuda()
    I1 = torch.empty_like(I0)
    s = gd.gd_stack_create(32, 32, 4)
    try:
        return gd.gd_diffuse_z(s, I0, I1, (0.0, 1.0, 1.0, 10.0), gd.solve_ctl(20, 1e-6))
    finally:
        gd.gd_destroy(s)


def test_bounded_wait_gives_up_and_context_survives(torch):
    assert gd.gd_selftest_wait(20000) == gd.GD_ERR_TIMEOUT
    assert gd.gd_selftest_wait(0) == gd.GD_ERR_INVALID_ARG
    assert small_solve(torch)["status"] == gd.GD_OK


def test_injected_allocation_failure(torch, monkeypatch):
    monkeypatch.setenv("GD_FAIL_ALLOC_AFTER", "2")
    I0 = torch.from_numpy(gdsynth.em_stack(32, 32, 4, seed=2).astype(np.float32)).cuda()
    I1 = torch.empty_like(I0)
    s = gd.gd_stack_create(32, 32, 4)
    try:
        with pytest.raises(gd.GdError) as ei:
            gd.gd_diffuse_z(s, I0, I1, (0.0, 1.0, 1.0, 10.0), gd.solve_ctl(20, 1e-6))
        assert ei.value.status == gd.GD_ERR_OOM
        assert "injected" in gd.gd_last_error(s)
    finally:
        gd.gd_destroy(s)
    monkeypatch.delenv("GD_FAIL_ALLOC_AFTER")
    assert small_solve(torch)["status"] == gd.GD_OK


@pytest.mark.parametrize("disc", [gd.GD_DISC_CONSTANT, gd.GD_DISC_HYBRID, gd.GD_DISC_LINEAR])
def test_poisoned_input_is_reported_as_diverged(torch, disc):
    I0h = gdsynth.em_stack(32, 32, 4, seed=3).astype(np.float32)
    I0h[2, 10, 7] = np.nan
    I0 = torch.from_numpy(I0h).cuda()
    I1 = torch.empty_like(I0)
    s = gd.gd_stack_create(32, 32, 4, disc=disc)
    try:
        r = gd.gd_diffuse_z(s, I0, I1, (0.0, 1.0, 1.0, 10.0), gd.solve_ctl(20, 1e-6), raise_on_error=False)
    finally:
        gd.gd_destroy(s)
    assert r["status"] == gd.GD_ERR_DIVERGED, r
    assert small_solve(torch)["status"] == gd.GD_OK


def test_poisoned_batch_is_reported_as_diverged(torch):
    nx, ny = [40, 70], [33, 20]
    I0s, I1s = gdsynth.batch_slices(nx, ny, seed=5)
    I0s[1][3, 4] = np.nan
    b = gd.gd_batch_create(nx, ny, [0.01, 0.02])
    try:
        I0 = torch.from_numpy(gdsynth.pack(I0s)).cuda()
        I1 = torch.from_numpy(gdsynth.pack(I1s)).cuda()
        o = torch.empty_like(I0)
        r = gd.gd_batch_screened_poisson(b, I0, I1, o, gd.solve_ctl(10, 1e-6), raise_on_error=False)
    finally:
        gd.gd_batch_destroy(b)
    assert r["status"] == gd.GD_ERR_DIVERGED, r


def test_tensor_core_kernels_bounded_wait_reports_timeout_and_recovers():
    """The learned guess's tcgen05 kernels share the solver's failure path: a
    bounded wait that runs out raises a device flag, the call returns
    GD_ERR_TIMEOUT, and the next call runs normally (no GPU fault involved:
    the wait is on a barrier that nothing arrives at)."""
    import numpy as np
    import torch
    from paper_1310_0041_gb300 import learn
    gd.build()
    assert gd.lib().gd_nn_selftest_wait(1000) == gd.GD_ERR_TIMEOUT
    x = torch.ones((1, 8, 8, 16), dtype=torch.bfloat16, device="cuda")
    w = torch.zeros((16, 9, 16), dtype=torch.bfloat16, device="cuda")
    w[:, 4, :] = torch.eye(16, dtype=torch.bfloat16, device="cuda")  # the centre tap: identity
    y = torch.empty((1, 8, 8, 16), dtype=torch.float32, device="cuda")
    assert learn.gd_nn_conv3x3(x, 16, 1, None, 0, 1, 8, 8, w, None, 16, 0, yf=y) == gd.GD_OK
    assert np.array_equal(y.cpu().numpy(), np.ones((1, 8, 8, 16), np.float32))
