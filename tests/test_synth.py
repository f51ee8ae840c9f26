"""The seeded input generator: reproducible, and shaped like the stated model."""
import numpy as np

from paper_2207_11638_gb300 import synth


def test_ar1_image_statistics_and_seed():
    a = synth.ar1_image(256, 256, 0.95, seed=1)
    b = synth.ar1_image(256, 256, 0.95, seed=1)
    c = synth.ar1_image(256, 256, 0.95, seed=2)
    assert a.dtype == np.uint8 and a.shape == (256, 256)
    np.testing.assert_array_equal(a, b)
    assert np.any(a != c)
    x = a.astype(np.float64)
    # theoretical 128 / 40 with correlation 0.95 along both axes (wide tolerance: one field)
    assert abs(x.std() - 40.0) < 8.0
    for ax in (0, 1):
        lo = np.take(x, range(0, 255), axis=ax).ravel()
        hi = np.take(x, range(1, 256), axis=ax).ravel()
        assert abs(np.corrcoef(lo, hi)[0, 1] - 0.95) < 0.02


def test_unit_variance_field():
    rng = np.random.Generator(np.random.PCG64(9))
    z = synth.ar1_field(400, 400, 0.9, rng)
    assert abs(z.var() - 1.0) < 0.15
    assert abs(z[:, 0].var() - 1.0) < 0.25      # stationary from the first sample


def test_residual_batch_shape_and_range():
    luma, chroma = synth.residual_frames_420(2, 36, 40, seed=5, threads=2)
    assert luma.shape == (2, 36, 40) and chroma.shape == (4, 18, 20)
    assert luma.dtype == np.int16 and luma.min() >= -255 and luma.max() <= 255
    again, _ = synth.residual_frames_420(2, 36, 40, seed=5, threads=1)
    np.testing.assert_array_equal(luma, again)


def test_uneven_sizes_and_regions():
    h, w, rho = synth.uneven_sizes(500, seed=3)
    assert h.min() >= 64 and w.max() <= 2048 and np.all(h % 32 == 0) and np.all(w % 32 == 0)
    assert rho.min() >= 0.85 and rho.max() <= 0.97
    r = synth.residual_regions_32(300, seed=4, side=128)
    assert r.shape == (300, 32, 32) and r.dtype == np.int16
