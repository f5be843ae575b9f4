"""The seeded input generator: determinism, windows, and the recipe's statistics."""
import numpy as np

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
