"""Batched screened Poisson on slices of different sizes (``gd_batch_*``) on
the GPU against the FP64 oracle (``oracle/batch.py``): every slice of ragged
small batches element by element, and the full-size batch of 512 slices
(sides log-uniform in [256, 4096], alpha ~ U(0.001, 0.1)) on sampled slices
plus the per-slice residuals of all of them."""
import numpy as np
import pytest

import gdsynth
import oracle.batch as ob
import paper_1310_0041_gb300 as gd

pytestmark = pytest.mark.gpu

# one tile, several tiles with ragged tails, single cells and columns,
# slices that never coarsen (< 32 cells) next to ones that do, rectangles
RAGGED = [(1, 1), (1, 7), (5, 3), (17, 23), (64, 32), (65, 33), (100, 37), (130, 257), (31, 200),
          (256, 256), (300, 129), (20, 300), (33, 64), (64, 1), (2, 2), (129, 130)]
TOL_ABS = 1e-3  # max |I2 - I2*| on the 0..255 scale


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no GPU")
    gd.build()
    return t


def solve(torch, nx, ny, al, I0s, I1s, ctl, x0s=None, host=False):
    b = gd.gd_batch_create(nx, ny, al)
    try:
        assert gd.gd_batch_voxels(b) == sum(a * c for a, c in zip(nx, ny))
        I0, I1 = gdsynth.pack(I0s), gdsynth.pack(I1s)
        x0 = gdsynth.pack(x0s) if x0s is not None else None
        if host:
            out = np.zeros_like(I0)
            rep = gd.gd_batch_screened_poisson(b, I0, I1, out, ctl, x0=x0, slice_rel=True)
        else:
            d = [torch.from_numpy(a).cuda() if a is not None else None for a in (I0, I1, x0)]
            o = torch.empty_like(d[0])
            rep = gd.gd_batch_screened_poisson(b, d[0], d[1], o, ctl, x0=d[2], slice_rel=True)
            out = o.cpu().numpy()
        rep["levels_api"] = gd.gd_batch_levels(b)
        rep["offsets"] = [gd.gd_batch_offset(b, s) for s in range(len(nx))]
    finally:
        gd.gd_batch_destroy(b)
    return gdsynth.unpack(out, nx, ny), rep


def ragged_case(seed):
    nx = [a for a, _ in RAGGED]
    ny = [c for _, c in RAGGED]
    al = gdsynth.batch_alphas(len(RAGGED), seed=seed)
    I0s, I1s = gdsynth.batch_slices(nx, ny, seed=seed)
    return nx, ny, al, I0s, I1s


def check_slices(outs, I0s, I1s, al, idx=None):
    for s in (idx if idx is not None else range(len(outs))):
        want = ob.sp_slice(I0s[s], I1s[s], al[s])
        got = outs[s].astype(np.float64)
        assert np.abs(got - want).max() <= TOL_ABS, (s, outs[s].shape, np.abs(got - want).max())
        # the float32 output as stored: its rounding alone gives ~1e-6
        assert ob.rel_residual_slice(I0s[s], I1s[s], al[s], got) <= 5e-6, s


def test_batch_ragged_parity(torch):
    nx, ny, al, I0s, I1s = ragged_case(21)
    outs, rep = solve(torch, nx, ny, al, I0s, I1s, gd.solve_ctl(40, 1e-7))
    assert rep["status"] == gd.GD_OK, rep
    assert rep["rel_residual"] <= 1e-7
    assert max(rep["slice_rel"]) <= 1e-7
    assert rep["cycles"] <= 12 and rep["rho_per_cycle"] < 0.3, rep
    assert rep["levels"] == rep["levels_api"] >= 4
    assert rep["offsets"] == list(np.cumsum([0] + [a * c for a, c in zip(nx, ny)])[:-1])
    check_slices(outs, I0s, I1s, al)


def test_batch_host_arrays_match_device(torch):
    nx, ny, al, I0s, I1s = ragged_case(22)
    ctl = gd.solve_ctl(40, 1e-7)
    dev, r1 = solve(torch, nx, ny, al, I0s, I1s, ctl)
    hst, r2 = solve(torch, nx, ny, al, I0s, I1s, ctl, host=True)
    assert r1["cycles"] == r2["cycles"]
    for a, c in zip(dev, hst):
        np.testing.assert_array_equal(a, c)


def test_batch_exact_initial_guess(torch):
    nx, ny, al, I0s, I1s = ragged_case(23)
    x0s = [s.astype(np.float32) for s in ob.sp_batch(I0s, I1s, al)]
    outs, rep = solve(torch, nx, ny, al, I0s, I1s, gd.solve_ctl(40, 1e-6), x0s=x0s)
    assert rep["status"] == gd.GD_OK
    assert rep["cycles"] <= 1, rep
    check_slices(outs, I0s, I1s, al)


def test_batch_equal_slices_match_stack_solver(torch):
    # a batch of equal slices with one alpha is the stack solver's screened
    # Poisson step: both must reach the oracle's answer
    nz, ny, nx = 6, 72, 96
    I0 = gdsynth.em_stack(nx, ny, nz, seed=9).astype(np.float32)
    I1 = np.clip(I0 * 0.9 + 11.0, 0, 255).astype(np.float32)
    al = [0.02] * nz
    outs, rep = solve(torch, [nx] * nz, [ny] * nz, al, list(I0), list(I1), gd.solve_ctl(40, 1e-7))
    assert rep["status"] == gd.GD_OK
    check_slices(outs, list(I0), list(I1), al)


def test_batch_solve_control_validation(torch):
    b = gd.gd_batch_create([40, 9], [30, 70], [0.01, 0.05])
    try:
        z = torch.zeros(gd.gd_batch_voxels(b), device="cuda")
        o = torch.empty_like(z)
        for ctl in (gd.solve_ctl(10, 1e-6, 2, 1), gd.solve_ctl(10, 1e-6, 2, 2, 8),
                    gd.solve_ctl(-1, 1e-6), gd.solve_ctl(0, 0.0)):
            with pytest.raises(gd.GdError) as ei:
                gd.gd_batch_screened_poisson(b, z, z, o, ctl)
            assert ei.value.status == gd.GD_ERR_INVALID_ARG
        # zero input: b = 0, the answer is 0 at once
        rep = gd.gd_batch_screened_poisson(b, z, z, o, gd.solve_ctl(10, 1e-6))
        assert rep["status"] == gd.GD_OK and rep["cycles"] == 0
        assert float(o.abs().max()) == 0.0
    finally:
        gd.gd_batch_destroy(b)


@pytest.mark.slow
def test_batch_full_size_512_slices(torch):
    n = 512
    sides = gdsynth.batch_sides(n, 256, 4096, seed=4)
    al = gdsynth.batch_alphas(n, seed=4)
    I0s, I1s = gdsynth.batch_slices(sides, sides, seed=4)
    outs, rep = solve(torch, sides, sides, al, I0s, I1s, gd.solve_ctl(40, 1e-7))
    assert rep["status"] == gd.GD_OK, rep
    assert max(rep["slice_rel"]) <= 1e-7
    order = np.argsort(sides)
    sample = [int(order[0]), int(order[n // 2]), int(order[-1]), int(np.argmin(al))]
    check_slices(outs, I0s, I1s, al, idx=sample)


def test_batch_tuning_keeps_results_bitwise(torch):
    # the work decomposition (rows per item) changes no cell's arithmetic:
    # a red value depends only on old black values wherever it is computed
    nx, ny, al, I0s, I1s = ragged_case(24)
    ctl = gd.solve_ctl(40, 1e-7)
    b = gd.gd_batch_create(nx, ny, al)
    try:
        I0 = torch.from_numpy(gdsynth.pack(I0s)).cuda()
        I1 = torch.from_numpy(gdsynth.pack(I1s)).cuda()
        o1, o2 = torch.empty_like(I0), torch.empty_like(I0)
        r1 = gd.gd_batch_screened_poisson(b, I0, I1, o1, ctl)
        chunk = gd.gd_batch_tune(b)
        assert chunk in (32, 64, 128, 256)
        r2 = gd.gd_batch_screened_poisson(b, I0, I1, o2, ctl)
    finally:
        gd.gd_batch_destroy(b)
    assert r1["cycles"] == r2["cycles"]
    assert torch.equal(o1, o2)
