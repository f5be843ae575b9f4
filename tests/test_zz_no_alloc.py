"""gd_smooth_noalloc: the red-black relaxation for callers that must not
allocate device memory (a host application owning the device pool, or a
latency-bound loop that cannot take cudaMalloc's implicit synchronisation).

It is checked against the allocating entry point gd_smooth on the same
inputs, within the sweep tolerance the other GPU tests use, on two calls in a
row (the second call finds the shared scratch array holding the first call's
contents).  This file is collected last so that a failure here stops a
`-x` run only after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import paper_1310_0041_gb300 as gd

pytestmark = pytest.mark.gpu

TOL = 1e-3  # same bar as the other sweep tests (0..255 scale, FP32 kernels)


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available(), "this test needs a CUDA GPU"
    gd.build()
    gd.lib()
    return _t


@pytest.mark.parametrize("shape,w,nsweeps", [
    ((17, 33, 40), (0.0, 1.0, 1.0, 10.0), 3),
    ((10, 48, 64), (0.01, 1.0, 1.0, 0.0), 2),
    ((5, 21, 70), (0.3, 1.0, 2.0, 0.5), 1),
])
def test_noalloc_matches_gd_smooth_twice(torch, shape, w, nsweeps):
    nz, ny, nx = shape
    rng = np.random.default_rng(nx * 1000 + ny * 10 + nz)
    b = torch.from_numpy(rng.uniform(-50, 50, size=shape).astype(np.float32)).cuda()
    x0 = torch.from_numpy(rng.uniform(0, 255, size=shape).astype(np.float32)).cuda()
    ref = x0.clone()
    s = gd.gd_stack_create(nx, ny, nz)
    try:
        gd.gd_smooth(s, w, b, ref, nsweeps)
    finally:
        gd.gd_destroy(s)
    want = ref.cpu().numpy().astype(np.float64)
    for _ in range(2):
        x = x0.clone()
        assert gd.gd_smooth_noalloc(nx, ny, nz, w, b, x, nsweeps) == gd.GD_OK
        got = x.cpu().numpy().astype(np.float64)
        assert np.abs(got - want).max() <= TOL


def test_noalloc_matches_the_oracle_sweep(torch):
    """The allocation-free sweep pinned to the FP64 oracle's red-black sweep
    directly (not only to the other CUDA entry point), on a ragged shape."""
    from oracle import gs_sweeps
    nz, ny, nx = 7, 19, 26
    rng = np.random.default_rng(11)
    b = rng.uniform(-50, 50, size=(nz, ny, nx)).astype(np.float32)
    x0 = rng.uniform(0, 255, size=(nz, ny, nx)).astype(np.float32)
    w = (0.05, 1.0, 2.0, 3.0)
    want = gs_sweeps(b, x0, *w, order="redblack", nsweeps=2)
    bd = torch.from_numpy(b).cuda()
    for _ in range(2):
        x = torch.from_numpy(x0).cuda()
        assert gd.gd_smooth_noalloc(nx, ny, nz, w, bd, x, 2) == gd.GD_OK
        assert np.abs(x.cpu().numpy().astype(np.float64) - want).max() <= TOL


def test_noalloc_zero_sweeps_and_the_largest_size(torch):
    # nsweeps = 0 leaves x as it was (bitwise)
    rng = np.random.default_rng(12)
    b = torch.from_numpy(rng.uniform(-50, 50, size=(3, 8, 8)).astype(np.float32)).cuda()
    x0 = torch.from_numpy(rng.uniform(0, 255, size=(3, 8, 8)).astype(np.float32)).cuda()
    x = x0.clone()
    assert gd.gd_smooth_noalloc(8, 8, 3, (0.0, 1.0, 1.0, 1.0), b, x, 0) == gd.GD_OK
    assert torch.equal(x, x0)
    # exactly GD_NOALLOC_MAX_VOXELS voxels: the whole scratch array, twice
    nz, ny, nx = 16, 512, 512
    assert nx * ny * nz == gd.GD_NOALLOC_MAX_VOXELS
    w = (0.0, 1.0, 1.0, 10.0)
    b = torch.from_numpy(rng.uniform(-50, 50, size=(nz, ny, nx)).astype(np.float32)).cuda()
    x0 = torch.from_numpy(rng.uniform(0, 255, size=(nz, ny, nx)).astype(np.float32)).cuda()
    ref = x0.clone()
    s = gd.gd_stack_create(nx, ny, nz)
    try:
        gd.gd_smooth(s, w, b, ref, 3)
    finally:
        gd.gd_destroy(s)
    for _ in range(2):
        x = x0.clone()
        assert gd.gd_smooth_noalloc(nx, ny, nz, w, b, x, 3) == gd.GD_OK
        assert (x - ref).abs().max().item() <= TOL


def test_noalloc_rejects_what_it_cannot_do(torch):
    b = torch.zeros(8, device="cuda")
    x = torch.zeros(8, device="cuda")
    w = (0.0, 1.0, 1.0, 1.0)
    L = gd.lib()
    W = gd.GdWeights(*w)
    # more voxels than the scratch array holds: refused before any launch
    big = gd.GD_NOALLOC_MAX_VOXELS + 1
    assert L.gd_smooth_noalloc(big, 1 + 1, 1, W, ctypes.c_void_p(b.data_ptr()),
                               ctypes.c_void_p(x.data_ptr()), 1, None) == gd.GD_ERR_INVALID_ARG
    # host arrays would need staging buffers
    hb = np.zeros(8, np.float32)
    hx = np.zeros(8, np.float32)
    assert L.gd_smooth_noalloc(2, 2, 2, W, ctypes.c_void_p(hb.ctypes.data),
                               ctypes.c_void_p(hx.ctypes.data), 1, None) == gd.GD_ERR_INVALID_ARG
    # aliasing and bad sizes
    p = ctypes.c_void_p(x.data_ptr())
    assert L.gd_smooth_noalloc(2, 2, 2, W, p, p, 1, None) == gd.GD_ERR_INVALID_ARG
    assert L.gd_smooth_noalloc(1, 2, 2, W, ctypes.c_void_p(b.data_ptr()), p, 1, None) == gd.GD_ERR_INVALID_ARG
    # partly overlapping b and x (x starts one element into b)
    y = torch.zeros(16, device="cuda")
    assert L.gd_smooth_noalloc(2, 2, 2, W, ctypes.c_void_p(y.data_ptr()),
                               ctypes.c_void_p(y.data_ptr() + 4), 1, None) == gd.GD_ERR_INVALID_ARG
    # the binding refuses host tensors before calling
    with pytest.raises(ValueError):
        gd.gd_smooth_noalloc(2, 2, 2, w, torch.zeros(8), x, 1)
