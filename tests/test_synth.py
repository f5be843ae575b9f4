"""The seeded input generator: determinism, windows, and the recipe's statistics."""
import numpy as np
import pytest

import gdsynth


def test_deterministic_and_windowed():
    a = gdsynth.em_stack(96, 80, 6, seed=3)
    b = gdsynth.em_stack(96, 80, 6, seed=3)
    assert a.dtype == np.uint8 and a.shape == (6, 80, 96)
    np.testing.assert_array_equal(a, b)
    w = gdsynth.em_stack(96, 80, 6, seed=3, window=(17, 5, 2, 40, 33, 3))
    np.testing.assert_array_equal(w, a[2:5, 5:38, 17:57])
    assert not np.array_equal(a, gdsynth.em_stack(96, 80, 6, seed=4))


def test_statistics():
    s = gdsynth.em_stack(256, 256, 8, seed=5).astype(np.float64)
    # interiors ~160 scaled by gain 0.8..1.2 and offset: the median sits well above the membranes
    assert 120 < np.median(s) < 200
    # membranes (dark, 2 px wide) are a sizeable minority of pixels
    frac_dark = (s < 100).mean()
    assert 0.05 < frac_dark < 0.35
    # slices differ photometrically (gain/offset/ramp are drawn per slice)
    means = s.mean(axis=(1, 2))
    assert means.std() > 2.0
    # structure is continuous along z: adjacent slices correlate far more than distant ones
    def corr(a, b):
        a, b = a - a.mean(), b - b.mean()
        return float((a * b).sum() / np.sqrt((a * a).sum() * (b * b).sum()))
    assert corr(s[0], s[1]) > 0.5


def test_noise_off_and_photo_seed():
    a = gdsynth.em_stack(64, 64, 2, seed=9, noise_sigma=0.0)
    b = gdsynth.em_stack(64, 64, 2, seed=9, noise_sigma=0.0)
    np.testing.assert_array_equal(a, b)
    i0, i1 = gdsynth.sp_pair(64, 21)
    assert i0.shape == (64, 64) and i1.shape == (64, 64)
    assert not np.array_equal(i0, i1)


def test_batch_inputs():
    sides = gdsynth.batch_sides(512, 256, 4096, seed=1)
    assert len(sides) == 512 and min(sides) >= 256 and max(sides) <= 4096
    # log-uniform: the median is near the geometric mean 1024 of the bounds
    assert 700 < sorted(sides)[256] < 1500
    al = gdsynth.batch_alphas(512, seed=1)
    assert min(al) >= 0.001 and max(al) < 0.1
    nx, ny = [5, 1, 70], [3, 9, 2]
    I0s, I1s = gdsynth.batch_slices(nx, ny, seed=4)
    assert [a.shape for a in I0s] == [(3, 5), (9, 1), (2, 70)]
    assert all(a.dtype == np.float32 and b.dtype == np.float32 for a, b in zip(I0s, I1s))
    flat = gdsynth.pack(I0s)
    assert flat.size == 15 + 9 + 140
    back = gdsynth.unpack(flat, nx, ny)
    assert all(np.array_equal(a, b) for a, b in zip(I0s, back))
    # seeded
    J0s, _ = gdsynth.batch_slices(nx, ny, seed=4)
    assert all(np.array_equal(a, b) for a, b in zip(I0s, J0s))


@pytest.mark.gpu
@pytest.mark.parametrize("shape,window", [
    ((300, 200, 20), (37, 11, 3, 200, 150, 12)),
    ((256, 256, 80), (0, 0, 0, 256, 256, 80)),   # more than one 64-slice chunk
])
def test_gpu_generator_draws_the_same_bytes(shape, window):
    """The GPU version of the generator reproduces the CPU generator's bytes
    (a differing byte would need a value within ~1e-13 of a rounding
    boundary: at most a handful are allowed, none expected)."""
    import torch
    assert torch.cuda.is_available()
    nx, ny, nz = shape
    want = gdsynth.em_stack(nx, ny, nz, seed=9, window=window)
    got = gdsynth.em_stack_cuda(nx, ny, nz, seed=9, window=window).cpu().numpy()
    assert got.shape == want.shape
    assert int((got != want).sum()) <= 2
