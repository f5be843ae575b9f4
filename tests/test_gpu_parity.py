"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

References are the oracle's (tests-only) routes: the DCT closed form, which
is the exact discrete solution of the 6-point Neumann systems, and the C
oracle's red-black sweep.  Bars (stated with each test):
  * solves: max |GPU - exact| <= 1e-3 on the 0..255 intensity scale, and the
    solver's relative residual ||b - A x|| / ||b|| <= the requested tolerance;
  * one or two relaxation sweeps: FP32 kernel vs FP64 oracle on the same
    float32 inputs, max |diff| <= 1e-3 (FP32 rounding of values up to 255 is
    ~1.5e-5 per operation).
"""
import numpy as np
import pytest

import gdsynth
import oracle
from oracle import closed_form as cf
import paper_1310_0041_gb300 as gd

pytestmark = pytest.mark.gpu

TOL_INTENSITY = 1e-3


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available(), "these tests need a CUDA GPU"
    gd.build()
    gd.lib()
    return _t


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def stack_u8(nx, ny, nz, seed, **kw):
    return gdsynth.em_stack(nx, ny, nz, seed=seed, **kw).astype(np.float32)


def ad_gpu(torch, I0, bz, tol=1e-6, max_cycles=30, bx=1.0, by=1.0, x0=None, flags=0, host=False):
    nz, ny, nx = I0.shape
    s = gd.gd_stack_create(nx, ny, nz)
    try:
        if host:
            i0 = np.ascontiguousarray(I0, np.float32)
            out = np.zeros_like(i0)
        else:
            i0 = dev(torch, I0)
            out = torch.zeros_like(i0)
        rep = gd.gd_diffuse_z(s, i0, out, (0.0, bx, by, bz),
                              gd.solve_ctl(max_cycles, tol, flags=flags), x0=x0)
        res = out if host else out.cpu().numpy()
    finally:
        gd.gd_destroy(s)
    return res.astype(np.float64), rep


def sp_gpu(torch, I0, I1, alpha, tol=1e-6, max_cycles=30, flags=0):
    nz, ny, nx = I0.shape
    s = gd.gd_stack_create(nx, ny, nz)
    try:
        i0, i1 = dev(torch, I0), dev(torch, I1)
        out = torch.zeros_like(i0)
        rep = gd.gd_screened_poisson_slices(s, i0, i1, out, alpha, gd.solve_ctl(max_cycles, tol, flags=flags))
        res = out.cpu().numpy()
    finally:
        gd.gd_destroy(s)
    return res.astype(np.float64), rep


# ---------------------------------------------------------------------------
# kernel-level: one and two red-black sweeps vs the oracle's red-black sweep
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(5, 37, 70), (40, 19, 9), (1, 16, 64), (3, 2, 2), (9, 130, 67),
                                   (5, 37, 68), (40, 19, 12), (9, 130, 132), (70, 33, 200)])
@pytest.mark.parametrize("w", [(0.0, 1.0, 1.0, 10.0), (0.01, 1.0, 1.0, 0.0), (0.3, 1.0, 2.0, 0.5)])
@pytest.mark.parametrize("nsweeps", [1, 2])
def test_rb_sweep_matches_oracle(torch, shape, w, nsweeps):
    rng = np.random.default_rng(hash((shape, w, nsweeps)) % 2**32)
    b = rng.uniform(-50, 50, size=shape).astype(np.float32)
    x = rng.uniform(0, 255, size=shape).astype(np.float32)
    want = oracle.gs_sweeps(b, x, *w, order="redblack", nsweeps=nsweeps)
    nz, ny, nx = shape
    s = gd.gd_stack_create(nx, ny, nz)
    try:
        xd = dev(torch, x)
        gd.gd_smooth(s, w, dev(torch, b), xd, nsweeps)
        got = xd.cpu().numpy().astype(np.float64)
    finally:
        gd.gd_destroy(s)
    assert np.abs(got - want).max() <= TOL_INTENSITY


def test_rb_sweep_host_pointers(torch):
    """Host (numpy) arrays go through the library's staging copies."""
    shape = (6, 21, 33)
    rng = np.random.default_rng(3)
    b = rng.uniform(-50, 50, size=shape).astype(np.float32)
    x = rng.uniform(0, 255, size=shape).astype(np.float32)
    w = (0.0, 1.0, 1.0, 10.0)
    want = oracle.gs_sweeps(b, x, *w, nsweeps=3)
    s = gd.gd_stack_create(33, 21, 6)
    try:
        gd.gd_smooth(s, w, b, x, 3)
    finally:
        gd.gd_destroy(s)
    assert np.abs(x - want).max() <= TOL_INTENSITY


# ---------------------------------------------------------------------------
# solves: oracle-size stack (64x64x16), both z weights, to 1e-8
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("bz", [10.0, 0.1])
def test_ad_64x64x16(torch, bz):
    """Oracle-size stack solved to 1e-8 (the float-pair iterate with a
    double-float residual goes well below what a float32 array represents)."""
    I0 = stack_u8(64, 64, 16, seed=1)
    got, rep = ad_gpu(torch, I0, bz, tol=1e-8, flags=gd.GD_FLAG_REPORT_OUTPUT_RESIDUAL)
    assert rep["status"] == gd.GD_OK, rep
    assert rep["rel_residual"] <= 1e-8
    want = cf.ad(I0, 1.0, 1.0, bz)
    assert np.abs(got - want).max() <= TOL_INTENSITY
    assert abs(got.mean() - I0.astype(np.float64).mean()) < 1e-4
    # the library's residual of the float32 output agrees with the oracle's
    b = oracle.rhs_ad(I0, 1.0, 1.0)
    ro = oracle.rel_residual(b, got, 0.0, 1.0, 1.0, bz)
    assert abs(rep["rel_residual_out"] - ro) <= 0.05 * ro + 1e-9
    assert ro < 2e-6  # the float32 representation floor (~1.2e-6 for bz = 10)


def test_sp_64x64x16(torch):
    I0 = stack_u8(64, 64, 16, seed=2)
    I1 = cf.ad(I0, 1.0, 1.0, 10.0).astype(np.float32)
    got, rep = sp_gpu(torch, I0, I1, 0.01, tol=1e-8)
    assert rep["status"] == gd.GD_OK, rep
    assert rep["rel_residual"] <= 1e-8
    want = cf.sp(I0, I1, 0.01)
    assert np.abs(got - want).max() <= TOL_INTENSITY
    # slice means of I1 are kept (Sec. 3.1 consequence)
    np.testing.assert_allclose(got.mean(axis=(1, 2)), I1.astype(np.float64).mean(axis=(1, 2)), atol=1e-3)


def test_pipeline_64x64x16(torch):
    """AD then SP on the GPU against the closed form of both steps."""
    I0 = stack_u8(64, 64, 16, seed=3)
    I1, r1 = ad_gpu(torch, I0, 10.0, tol=1e-8)
    I2, r2 = sp_gpu(torch, I0, I1.astype(np.float32), 0.01, tol=1e-8)
    want = cf.sp(I0, cf.ad(I0, 1.0, 1.0, 10.0), 0.01)
    assert np.abs(I2 - want).max() <= TOL_INTENSITY


# ---------------------------------------------------------------------------
# solves: the 256x256x32 crop of the 1024x1024x128 stack, solved as its own
# problem, to 1e-6 (several tiles, several z chunks, ragged-free and ragged)
# ---------------------------------------------------------------------------
def crop_256():
    return gdsynth.em_stack(1024, 1024, 128, seed=7, ncells=2000,
                            window=(384, 512, 48, 256, 256, 32)).astype(np.float32)


def test_ad_sp_crop_256x256x32(torch):
    """AD to 1e-6 and SP to 1e-7: with alpha = 0.01 the slice-smooth error of
    SP is ~100x its residual, so 1e-6 alone does not give max|d| <= 1e-3."""
    I0 = crop_256()
    I1, r1 = ad_gpu(torch, I0, 10.0, tol=1e-6)
    assert r1["status"] == gd.GD_OK and r1["rel_residual"] <= 1e-6, r1
    assert np.abs(I1 - cf.ad(I0, 1.0, 1.0, 10.0)).max() <= TOL_INTENSITY
    assert r1["rho_per_cycle"] < 0.2
    I2, r2 = sp_gpu(torch, I0, I1.astype(np.float32), 0.01, tol=1e-7)
    assert r2["status"] == gd.GD_OK and r2["rel_residual"] <= 1e-7, r2
    assert np.abs(I2 - cf.sp(I0, I1, 0.01)).max() <= TOL_INTENSITY


@pytest.mark.parametrize("shape", [(13, 75, 100), (7, 61, 47), (3, 33, 40), (1, 50, 30), (2, 2, 2),
                                   (1, 2, 2), (33, 17, 65)])
def test_ragged_sizes(torch, shape):
    nz, ny, nx = shape
    I0 = stack_u8(nx, ny, nz, seed=11)
    for bz in (10.0, 0.1):
        got, rep = ad_gpu(torch, I0, bz, tol=1e-7)
        assert rep["status"] == gd.GD_OK, (bz, rep)
        assert np.abs(got - cf.ad(I0, 1.0, 1.0, bz)).max() <= TOL_INTENSITY
    I1 = cf.ad(I0, 1.0, 1.0, 10.0).astype(np.float32)
    for alpha in (0.001, 0.1):
        got, rep = sp_gpu(torch, I0, I1, alpha, tol=1e-7)
        assert rep["status"] == gd.GD_OK, (alpha, rep)
        assert np.abs(got - cf.sp(I0, I1, alpha)).max() <= TOL_INTENSITY


# ---------------------------------------------------------------------------
# degenerate inputs and options
# ---------------------------------------------------------------------------
def test_z_constant_stack_is_a_fixed_point(torch):
    sl = stack_u8(80, 48, 1, seed=12)
    I0 = np.repeat(sl, 9, axis=0)
    # started from I0: b - A I0 = -bz Kz I0 = 0, converged before any cycle
    got, rep = ad_gpu(torch, I0, 10.0, tol=1e-6, x0=dev(torch, I0))
    assert rep["status"] == gd.GD_OK
    assert rep["cycles"] == 0
    np.testing.assert_array_equal(got, I0)
    # from the default zero start the cycles reach the same fixed point
    got, rep = ad_gpu(torch, I0, 10.0, tol=1e-7)
    assert rep["status"] == gd.GD_OK and rep["cycles"] > 0
    np.testing.assert_allclose(got, I0, atol=1e-3)


def test_slice_constant_stack(torch):
    """b = 0 (each slice constant): the solution is the global mean."""
    I0 = np.broadcast_to(np.arange(6, dtype=np.float32)[:, None, None] * 10.0, (6, 20, 24)).copy()
    got, rep = ad_gpu(torch, I0, 10.0, tol=1e-6)
    np.testing.assert_allclose(got, I0.mean(), atol=1e-3)


def test_self_reproduction(torch):
    I0 = stack_u8(96, 64, 4, seed=13)
    got, rep = sp_gpu(torch, I0, I0, 0.01, tol=1e-6)
    assert rep["cycles"] == 0
    np.testing.assert_array_equal(got, I0)


def test_initial_guess_and_host_arrays(torch):
    I0 = stack_u8(64, 48, 8, seed=14)
    want = cf.ad(I0, 1.0, 1.0, 10.0)
    # a caller's initial guess with the wrong mean: the mean is still fixed
    x0 = dev(torch, I0 + 7.0)
    got, rep = ad_gpu(torch, I0, 10.0, tol=1e-7, x0=x0)
    assert np.abs(got - want).max() <= TOL_INTENSITY
    # x0 aliasing the output buffer
    nz, ny, nx = I0.shape
    s = gd.gd_stack_create(nx, ny, nz)
    try:
        i0 = dev(torch, I0)
        out = dev(torch, want)  # exact solution as the start: no cycle needed
        rep = gd.gd_diffuse_z(s, i0, out, (0, 1, 1, 10.0), gd.solve_ctl(10, 1e-6), x0=out)
        assert rep["cycles"] <= 1
        assert np.abs(out.cpu().numpy() - want).max() <= TOL_INTENSITY
    finally:
        gd.gd_destroy(s)
    # host arrays in and out
    got, rep = ad_gpu(torch, I0, 10.0, tol=1e-7, host=True)
    assert np.abs(got - want).max() <= TOL_INTENSITY


def test_max_cycles_and_status(torch):
    I0 = stack_u8(64, 64, 8, seed=15)
    got, rep = ad_gpu(torch, I0, 10.0, tol=1e-12, max_cycles=2)
    assert rep["status"] == gd.GD_ERR_NOT_CONVERGED
    assert rep["cycles"] == 2
    assert rep["history"][2] < rep["history"][0]


def test_deterministic(torch):
    I0 = stack_u8(128, 96, 12, seed=16)
    a, _ = ad_gpu(torch, I0, 10.0, tol=1e-7)
    b, _ = ad_gpu(torch, I0, 10.0, tol=1e-7)
    np.testing.assert_array_equal(a, b)


def test_vcycle_primitive(torch):
    """gd_vcycle: plain FP32 V-cycles on an explicit right-hand side."""
    I0 = stack_u8(128, 128, 16, seed=17)
    b = oracle.rhs_ad(I0, 1.0, 1.0).astype(np.float32)
    s = gd.gd_stack_create(128, 128, 16)
    try:
        x = dev(torch, I0)
        rep = gd.gd_vcycle(s, gd.GD_SYSTEM_AD, (0, 1, 1, 10.0), dev(torch, b), x, 8)
        assert rep["rho_per_cycle"] < 0.2, rep
        xs = x.cpu().numpy().astype(np.float64)
        want = cf.ad(I0, 1.0, 1.0, 10.0)
        xs += want.mean() - xs.mean()
        assert np.abs(xs - want).max() < 0.01
        # residual definition agrees with the oracle
        ro = oracle.rel_residual(b, x.cpu().numpy(), 0.0, 1.0, 1.0, 10.0)
        assert abs(rep["rel_residual"] - ro) <= 0.02 * ro
        # SP system with odd sweep parity handled
        bsp = oracle.rhs_sp(I0, I0 * 0.5, 0.05).astype(np.float32)
        y = dev(torch, I0)
        rep = gd.gd_vcycle(s, gd.GD_SYSTEM_SP, (0.05, 1, 1, 0.0), dev(torch, bsp), y, 3)
        assert rep["rel_residual"] < 1e-3
    finally:
        gd.gd_destroy(s)


def test_residual_entry_point(torch):
    I0 = stack_u8(64, 40, 6, seed=18)
    x = (cf.ad(I0, 1.0, 1.0, 10.0) + np.random.default_rng(0).normal(0, 0.1, I0.shape)).astype(np.float32)
    s = gd.gd_stack_create(64, 40, 6)
    try:
        rel = gd.gd_residual(s, gd.GD_SYSTEM_AD, (0, 1, 1, 10.0), dev(torch, I0), None, dev(torch, x))
    finally:
        gd.gd_destroy(s)
    ro = oracle.rel_residual(oracle.rhs_ad(I0, 1.0, 1.0), x, 0.0, 1.0, 1.0, 10.0)
    assert abs(rel - ro) <= 1e-4 * ro


@pytest.mark.parametrize("shape", [(24, 96, 128), (13, 75, 100), (40, 50, 36)])
def test_tma_pipeline_matches_plain_kernels(torch, shape, monkeypatch):
    """The TMA z-march path (fused restriction / prolongation, pipelined outer
    pass) and the plain kernels (GD_DISABLE_TMA) run the same V-cycles: the
    residual histories and the results agree to rounding."""
    nz, ny, nx = shape
    I0 = stack_u8(nx, ny, nz, seed=19)
    out = {}
    for mode in ("tma", "plain"):
        if mode == "plain":
            monkeypatch.setenv("GD_DISABLE_TMA", "1")
        else:
            monkeypatch.delenv("GD_DISABLE_TMA", raising=False)
        a, ra = ad_gpu(torch, I0, 10.0, tol=1e-9, max_cycles=6)
        I1 = cf.ad(I0, 1.0, 1.0, 10.0).astype(np.float32)
        b, rb = sp_gpu(torch, I0, I1, 0.01, tol=1e-9, max_cycles=4)
        out[mode] = (a, ra, b, rb)
    a1, r1, b1, s1 = out["tma"]
    a2, r2, b2, s2 = out["plain"]
    # the TMA path's early outer passes keep only the high word of the iterate
    # (plain FP32 while the residual is above 1e-4); the plain kernels always
    # keep both words, so below 1e-4 the histories differ by rounding and are
    # compared by their rates: every cycle there still gains a factor 4
    for h1, h2 in ((r1["history"], r2["history"]), (s1["history"], s2["history"])):
        assert len(h1) == len(h2)
        for k, (u, v) in enumerate(zip(h1, h2)):
            if max(u, v) > 1e-4:
                assert abs(u - v) <= 0.02 * max(u, v), (h1, h2)
            else:
                assert u <= 0.25 * h1[k - 1] and v <= 0.25 * h2[k - 1], (h1, h2)
    assert np.abs(a1 - a2).max() < 1e-3
    assert np.abs(b1 - b2).max() < 1e-3


@pytest.mark.parametrize("shape,prof", [((24, 96, 128), False), ((13, 75, 100), True), ((5, 37, 68), False)])
def test_graph_replay_matches_direct_launches(torch, shape, prof, monkeypatch):
    """A solve replays its V-cycle from a captured CUDA graph; with
    GD_DISABLE_GRAPHS every kernel is launched directly.  Both run the same
    kernels on the same buffers, so results and histories are bitwise equal,
    and the per-class profile sees the same launches."""
    nz, ny, nx = shape
    I0 = stack_u8(nx, ny, nz, seed=23)
    out = {}
    for mode in ("graph", "direct"):
        if mode == "direct":
            monkeypatch.setenv("GD_DISABLE_GRAPHS", "1")
        else:
            monkeypatch.delenv("GD_DISABLE_GRAPHS", raising=False)
        s = gd.gd_stack_create(nx, ny, nz)
        try:
            gd.gd_profile_enable(s, 1 if prof else 0)
            x0 = dev(torch, I0)
            y = torch.empty_like(x0)
            z = torch.empty_like(x0)
            r1 = gd.gd_diffuse_z(s, x0, y, (0.0, 1.0, 1.0, 10.0), gd.solve_ctl(12, 1e-9))
            r2 = gd.gd_screened_poisson_slices(s, x0, y, z, 0.01, gd.solve_ctl(12, 1e-9))
            # a second solve on the same stack reuses the captured graphs
            r3 = gd.gd_diffuse_z(s, x0, y, (0.0, 1.0, 1.0, 10.0), gd.solve_ctl(12, 1e-9))
            torch.cuda.synchronize()
            prof_rows = gd.gd_profile_all(s) if prof else None
        finally:
            gd.gd_destroy(s)
        out[mode] = (y.cpu().numpy(), z.cpu().numpy(), r1, r2, r3, prof_rows)
    g, d = out["graph"], out["direct"]
    assert np.array_equal(g[0], d[0]) and np.array_equal(g[1], d[1])
    for i in (2, 3, 4):
        assert g[i]["status"] == gd.GD_OK
        assert g[i]["cycles"] == d[i]["cycles"]
        assert list(g[i]["history"]) == list(d[i]["history"])
    if prof:
        lg = {row[0]: row[1] for row in g[5]}
        ld = {row[0]: row[1] for row in d[5]}
        assert lg == ld
        assert all(row[2] > 0 for row in g[5] if row[1] > 0)


def test_plan_cache_eviction_keeps_results(torch):
    """A stack keeps a few hierarchies (one per weight set); cycling through
    more weight sets than it keeps evicts and rebuilds them.  Every solve on
    the shared stack equals the same solve on a fresh stack, bit for bit."""
    nx, ny, nz = 70, 33, 20
    I0 = stack_u8(nx, ny, nz, seed=29)
    x0 = dev(torch, I0)
    betas = [10.0, 3.0, 1.0, 0.5, 20.0, 10.0, 3.0]
    s = gd.gd_stack_create(nx, ny, nz)
    shared = []
    try:
        for bz in betas:
            y = torch.empty_like(x0)
            r = gd.gd_diffuse_z(s, x0, y, (0.0, 1.0, 1.0, bz), gd.solve_ctl(20, 1e-8))
            assert r["status"] == gd.GD_OK
            z = torch.empty_like(x0)
            r2 = gd.gd_screened_poisson_slices(s, x0, y, z, 0.01, gd.solve_ctl(20, 1e-8))
            assert r2["status"] == gd.GD_OK
            shared.append((y.cpu().numpy(), z.cpu().numpy()))
    finally:
        gd.gd_destroy(s)
    for bz, (y_s, z_s) in zip(betas, shared):
        f = gd.gd_stack_create(nx, ny, nz)
        try:
            y = torch.empty_like(x0)
            gd.gd_diffuse_z(f, x0, y, (0.0, 1.0, 1.0, bz), gd.solve_ctl(20, 1e-8))
            z = torch.empty_like(x0)
            gd.gd_screened_poisson_slices(f, x0, y, z, 0.01, gd.solve_ctl(20, 1e-8))
        finally:
            gd.gd_destroy(f)
        assert np.array_equal(y.cpu().numpy(), y_s)
        assert np.array_equal(z.cpu().numpy(), z_s)


def test_pinned_and_pageable_host_arrays_give_the_device_result(torch):
    """gd_ad_then_sp from pinned host buffers (moved by the wide copy kernel
    on their mapped addresses), from pageable ones (cudaMemcpyAsync) and from
    device buffers: the same kernels run on the same values, so the outputs
    (I2, and I1 read back) are bit-identical; ragged extents exercise the
    copy's tail, and the result matches the exact solutions."""
    I0 = stack_u8(37, 29, 6, seed=31).astype(np.float32)
    nz, ny, nx = I0.shape
    w = (0.0, 1.0, 1.0, 10.0)
    ctl_ad, ctl_sp = gd.solve_ctl(30, 1e-7), gd.solve_ctl(30, 1e-9)
    s = gd.gd_stack_create(nx, ny, nz)
    try:
        i0d = torch.from_numpy(I0).cuda()
        i1d, i2d = torch.empty_like(i0d), torch.empty_like(i0d)
        gd.gd_ad_then_sp(s, i0d, i2d, w, 0.05, ctl_ad, ctl_sp, I1=i1d)
        want1, want2 = i1d.cpu().numpy(), i2d.cpu().numpy()
        pin0 = torch.from_numpy(I0).pin_memory()
        pin1 = torch.empty(I0.shape, dtype=torch.float32).pin_memory()
        pin2 = torch.empty(I0.shape, dtype=torch.float32).pin_memory()
        gd.gd_ad_then_sp(s, pin0, pin2, w, 0.05, ctl_ad, ctl_sp, I1=pin1)
        page1, page2 = np.empty_like(I0), np.empty_like(I0)
        gd.gd_ad_then_sp(s, I0.copy(), page2, w, 0.05, ctl_ad, ctl_sp, I1=page1)
    finally:
        gd.gd_destroy(s)
    np.testing.assert_array_equal(pin1.numpy(), want1)
    np.testing.assert_array_equal(pin2.numpy(), want2)
    np.testing.assert_array_equal(page1, want1)
    np.testing.assert_array_equal(page2, want2)
    i0 = I0.astype(np.float64)
    ref1 = cf.ad(i0, 1.0, 1.0, 10.0)
    assert np.abs(want1 - ref1).max() <= TOL_INTENSITY
    assert np.abs(want2 - cf.sp(i0, want1.astype(np.float64), 0.05)).max() <= TOL_INTENSITY
