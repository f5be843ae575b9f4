"""The C-ABI library: it loads, exports every symbol include/gd.h declares,
and rejects bad arguments before touching the GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

import paper_1310_0041_gb300 as gd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header="gd.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_ ]+\*?\s*\b(gd_[a-z0-9_]+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    gd.build()
    return gd.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("gd_stack_create", "gd_diffuse_z", "gd_screened_poisson_slices", "gd_vcycle", "gd_destroy"):
        assert f in names
    assert set(names) == set(gd.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions() + declared_functions("gd_learn.h"):
        assert hasattr(lib, name), name


def test_learn_header_declares_the_network_calls():
    assert set(declared_functions("gd_learn.h")) == set(gd.EXPORTS_LEARN)


def test_status_strings_and_version(lib):
    assert gd.gd_version() == 1
    assert gd.gd_status_string(gd.GD_OK) == "ok"
    assert gd.gd_status_string(gd.GD_ERR_NOT_CONVERGED) == "not converged"


def test_create_validation_without_gpu(lib):
    h = ctypes.c_void_p()
    f = lib.gd_stack_create
    assert f(None, 8, 8, 8, 0, 0, 0, None) == gd.GD_ERR_INVALID_ARG
    assert f(ctypes.byref(h), 1, 8, 8, 0, 0, 0, None) == gd.GD_ERR_INVALID_ARG
    assert f(ctypes.byref(h), 8, 8, 0, 0, 0, 0, None) == gd.GD_ERR_INVALID_ARG
    assert f(ctypes.byref(h), 8, 8, 8, 1, 0, 0, None) == gd.GD_ERR_UNSUPPORTED
    # the Hybrid and Linear discretisations run in float32 only
    for disc in (gd.GD_DISC_HYBRID, gd.GD_DISC_LINEAR):
        assert f(ctypes.byref(h), 8, 8, 8, 0, disc, gd.GD_PREC_MIXED, None) == gd.GD_ERR_UNSUPPORTED
    assert f(ctypes.byref(h), 8, 8, 8, 0, 3, 0, None) == gd.GD_ERR_INVALID_ARG
    assert f(ctypes.byref(h), 8, 8, 8, 0, 0, 7, None) == gd.GD_ERR_INVALID_ARG
    assert f(ctypes.byref(h), 8, 8, 8, 0, 0, 0, None) == gd.GD_OK
    s = gd.Stack(h, 8, 8, 8)
    # argument checks that return before any CUDA call
    rep = gd.GdReport()
    W = gd.GdWeights
    assert lib.gd_diffuse_z(h, None, None, W(0, 1, 1, 10), None, None, ctypes.byref(rep)) == gd.GD_ERR_INVALID_ARG
    assert rep.status == gd.GD_ERR_INVALID_ARG
    p = ctypes.c_void_p(0x1000)
    assert lib.gd_diffuse_z(h, p, p, W(0, 1, 1, 10), None, None, None) == gd.GD_ERR_INVALID_ARG  # aliasing
    q = ctypes.c_void_p(0x2000)
    assert lib.gd_diffuse_z(h, p, q, W(0, 1, 1, 0.0), None, None, None) == gd.GD_ERR_INVALID_ARG  # bz = 0
    assert lib.gd_diffuse_z(h, p, q, W(0, -1, 1, 1), None, None, None) == gd.GD_ERR_INVALID_ARG
    assert lib.gd_diffuse_z(h, p, q, W(0, float("nan"), 1, 1), None, None, None) == gd.GD_ERR_INVALID_ARG
    r = ctypes.c_void_p(0x3000)
    assert lib.gd_screened_poisson_slices(h, p, q, r, 0.0, None, None, None) == gd.GD_ERR_INVALID_ARG
    assert lib.gd_screened_poisson_slices(h, p, q, p, 0.01, None, None, None) == gd.GD_ERR_INVALID_ARG
    assert lib.gd_vcycle(h, 5, W(0.1, 1, 1, 0), p, q, 1, None) == gd.GD_ERR_INVALID_ARG
    assert lib.gd_vcycle(h, gd.GD_SYSTEM_SP, W(0.1, 1, 1, 1), p, q, 1, None) == gd.GD_ERR_INVALID_ARG
    assert lib.gd_vcycle(h, gd.GD_SYSTEM_AD, W(0.0, 1, 1, 0), p, q, 1, None) == gd.GD_ERR_INVALID_ARG
    assert lib.gd_smooth(h, W(0, 1, 1, 1), p, p, 1) == gd.GD_ERR_INVALID_ARG
    assert gd.gd_destroy(s) == gd.GD_OK
    assert lib.gd_destroy(None) == gd.GD_OK


def test_binding_marshalling_rejects_wrong_dtype(lib):
    import numpy as np
    with pytest.raises(ValueError):
        gd._ptr(np.zeros(8, np.float64), 8, "x")
    with pytest.raises(ValueError):
        gd._ptr(np.zeros(7, np.float32), 8, "x")
    assert gd._ptr(None) is None


def test_general_solve_and_npr_validation_without_gpu(lib):
    """Argument checks of gd_screened_poisson / gd_npr_rhs return before any
    CUDA call."""
    h = ctypes.c_void_p()
    assert lib.gd_stack_create(ctypes.byref(h), 8, 8, 8, 0, 0, 0, None) == gd.GD_OK
    s = gd.Stack(h, 8, 8, 8)
    try:
        buf = (ctypes.c_float * 512)()
        buf2 = (ctypes.c_float * 512)()
        rep = gd.GdReport()
        p, q = ctypes.cast(buf, ctypes.c_void_p), ctypes.cast(buf2, ctypes.c_void_p)
        # alpha must be > 0
        assert lib.gd_screened_poisson(s.handle, gd.GdWeights(0.0, 1, 1, 1), p, q, None, None,
                                       ctypes.byref(rep)) == gd.GD_ERR_INVALID_ARG
        # x aliasing b
        assert lib.gd_screened_poisson(s.handle, gd.GdWeights(0.1, 1, 1, 1), p, p, None, None,
                                       ctypes.byref(rep)) == gd.GD_ERR_INVALID_ARG
        # sigma must be > 0, b must not alias I0
        assert lib.gd_npr_rhs(s.handle, p, q, gd.GdWeights(0.001, 1, 1, 0.1), 1.25, 0.0) == gd.GD_ERR_INVALID_ARG
        assert lib.gd_npr_rhs(s.handle, p, p, gd.GdWeights(0.001, 1, 1, 0.1), 1.25, 5.0) == gd.GD_ERR_INVALID_ARG
    finally:
        gd.gd_destroy(s)


def test_batch_validation_without_gpu(lib):
    # argument checks return before any CUDA call
    for nx, ny, al in (([10], [10], [0.0]), ([10], [10], [-1.0]), ([0], [5], [0.01]),
                       ([5], [1 << 21], [0.01]), ([4, 4], [4, 4], [0.01, float("nan")])):
        with pytest.raises(gd.GdError) as ei:
            gd.gd_batch_create(nx, ny, al)
        assert ei.value.status == gd.GD_ERR_INVALID_ARG
        assert gd.gd_batch_last_error(None)
    with pytest.raises(gd.GdError) as ei:
        gd.gd_batch_create([10], [10], [0.01], coarsest_xy=1)
    assert ei.value.status == gd.GD_ERR_INVALID_ARG
    # a slice whose coarsest level exceeds the batched direct solve (planned on
    # the host before any allocation)
    with pytest.raises(gd.GdError) as ei:
        gd.gd_batch_create([64, 20], [64, 100000], [0.01, 0.01])
    assert ei.value.status == gd.GD_ERR_UNSUPPORTED
    assert "coarsest level" in gd.gd_batch_last_error(None)
    # NULL handles
    assert lib.gd_batch_voxels(None) == -1
    assert lib.gd_batch_offset(None, 0) == -1
    assert lib.gd_batch_destroy(None) == gd.GD_ERR_INVALID_ARG
    assert lib.gd_batch_screened_poisson(None, None, None, None, None, None, None, None) == \
        gd.GD_ERR_INVALID_ARG


def test_pipeline_and_selftest_validation_without_gpu(lib):
    # argument checks of the newer entry points return before any CUDA call
    h = ctypes.c_void_p()
    assert lib.gd_stack_create(ctypes.byref(h), 8, 8, 2, 0, 0, 0, None) == gd.GD_OK
    s = gd.Stack(h, 8, 8, 2)
    try:
        import numpy as np
        a = np.zeros(8 * 8 * 2, np.float32)
        b = np.zeros_like(a)
        with pytest.raises(gd.GdError) as ei:
            gd.gd_ad_then_sp(s, a, a, (0.0, 1.0, 1.0, 1.0), 0.01)
        assert ei.value.status == gd.GD_ERR_INVALID_ARG
        with pytest.raises(gd.GdError) as ei:
            gd.gd_ad_then_sp(s, a, b, (0.0, 1.0, 1.0, 1.0), 0.0)
        assert ei.value.status == gd.GD_ERR_INVALID_ARG
        with pytest.raises(gd.GdError) as ei:
            gd.gd_ad_then_sp(s, a, b, (0.0, 1.0, 1.0, 1.0), 0.01, I1=a)
        assert ei.value.status == gd.GD_ERR_INVALID_ARG
    finally:
        gd.gd_destroy(s)
    assert gd.gd_selftest_wait(0) == gd.GD_ERR_INVALID_ARG
    assert gd.gd_selftest_wait(1 << 25) == gd.GD_ERR_INVALID_ARG
    pc, ps = ctypes.c_double(), ctypes.c_double()
    assert lib.gd_batch_traffic(None, 2, 2, ctypes.byref(pc), ctypes.byref(ps)) == gd.GD_ERR_INVALID_ARG
    assert lib.gd_batch_last_traffic(None) == -1.0
    assert lib.gd_batch_tune(None, None) == gd.GD_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        gd.gd_batch_create([4, 4], [4], [0.01, 0.01])
