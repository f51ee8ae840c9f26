"""Pins of the SSIM oracle (oracle/metrics.ssim, the index Sec. 5.1 cites):
identity, closed forms for constant images and for a constant shift,
symmetry, and brute-force window sums on a tiny image."""
import itertools
import math

import numpy as np
import pytest

from oracle import metrics as m

C1, C2 = (0.01 * 255) ** 2, (0.03 * 255) ** 2


def test_window_is_normalised_gaussian():
    w = m.ssim_window()
    assert w.shape == (11, 11) and abs(w.sum() - 1) < 1e-15
    assert np.allclose(w, w.T) and np.allclose(w, w[::-1, ::-1])
    assert w.argmax() == 5 * 11 + 5
    # ratio of neighbours is the Gaussian's: exp(-(2c + 1) / (2 sigma^2)) along an axis
    assert math.isclose(w[5, 6] / w[5, 5], math.exp(-1 / (2 * 1.5 ** 2)), rel_tol=1e-12)


def test_identical_images_give_one():
    x = np.random.default_rng(0).integers(0, 256, size=(40, 37)).astype(np.float64)
    assert np.allclose(m.ssim_map(x, x), 1.0, atol=1e-12)


@pytest.mark.parametrize("a,b", [(0, 0), (10, 200), (255, 0), (128, 129)])
def test_constant_images_closed_form(a, b):
    x = np.full((15, 20), float(a))
    y = np.full((15, 20), float(b))
    want = (2 * a * b + C1) / (a * a + b * b + C1)
    assert np.allclose(m.ssim_map(x, y), want, rtol=1e-12)
    assert m.ssim_map(x, y).shape == (5, 10)


def test_constant_shift_leaves_only_the_luminance_term():
    x = np.random.default_rng(1).integers(0, 200, size=(30, 30)).astype(np.float64)
    y = x + 17.0
    w = m.ssim_window()
    got = m.ssim_map(x, y)
    for i, j in [(0, 0), (7, 12), (19, 19)]:
        mu = float(np.sum(w * x[i:i + 11, j:j + 11]))
        want = (2 * mu * (mu + 17) + C1) / (mu * mu + (mu + 17) ** 2 + C1)
        assert math.isclose(got[i, j], want, rel_tol=1e-12)


def test_symmetric():
    rng = np.random.default_rng(2)
    x = rng.integers(0, 256, size=(25, 31)).astype(np.float64)
    y = rng.normal(128, 40, size=(25, 31))
    assert math.isclose(m.ssim(x, y), m.ssim(y, x), rel_tol=1e-13)


def test_brute_force_windows():
    rng = np.random.default_rng(3)
    x = rng.integers(0, 256, size=(13, 14)).astype(np.float64)
    y = rng.integers(0, 256, size=(13, 14)).astype(np.float64)
    w = m.ssim_window()
    got = m.ssim_map(x, y)
    assert got.shape == (3, 4)
    for i, j in itertools.product(range(3), range(4)):
        sx = sy = sxx = syy = sxy = 0.0
        for k, l in itertools.product(range(11), range(11)):
            a, b = x[i + k, j + l], y[i + k, j + l]
            sx += w[k, l] * a
            sy += w[k, l] * b
            sxx += w[k, l] * a * a
            syy += w[k, l] * b * b
            sxy += w[k, l] * a * b
        vx, vy, cxy = sxx - sx * sx, syy - sy * sy, sxy - sx * sy
        want = (2 * sx * sy + C1) * (2 * cxy + C2) / ((sx * sx + sy * sy + C1) * (vx + vy + C2))
        assert math.isclose(got[i, j], want, rel_tol=1e-10)
