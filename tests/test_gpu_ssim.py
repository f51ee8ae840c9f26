"""GPU SSIM (cdct_ssim) against the float64 oracle (oracle/metrics.ssim).

Both sides compute in float64 from the same integer / float32 inputs, so
the mean SSIM agrees to rounding order: 1e-10 absolute."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import metrics as m
from paper_2207_11638_gb300 import binding as b
from paper_2207_11638_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-10


def test_ssim_of_still_image_reconstructions_matches_oracle():
    img = synth.ar1_image(512, 512, 0.95, seed=1)
    dev = torch.from_numpy(img).cuda()
    for n, variant, r in ((8, "hat", 6), (8, "tilde", 1), (16, "hat", 64), (32, "tilde", 256)):
        rec, _, _ = b.Plan(n, variant).fwd_zonal_inv(dev, r, psnr=False)
        got = float(b.ssim(dev, rec).cpu()[0])
        want = m.ssim(img.astype(np.float64), rec.cpu().numpy()[0].astype(np.float64))
        print(f"N={n} {variant} r={r}: SSIM {got:.6f} (oracle {want:.6f})")
        assert abs(got - want) <= TOL
        assert 0 < got < 1


@pytest.mark.parametrize("shape", [(11, 11), (12, 45), (77, 40), (100, 130)])
def test_ssim_ragged_batches_match_oracle(shape):
    rng = np.random.default_rng(sum(shape))
    ref = rng.integers(0, 256, size=(3,) + shape).astype(np.uint8)
    rec = np.clip(ref + rng.normal(0, 12, size=ref.shape), -20, 280).astype(np.float32)
    got = b.ssim(torch.from_numpy(ref).cuda(), torch.from_numpy(rec).cuda()).cpu().numpy()
    want = [m.ssim(ref[i].astype(np.float64), rec[i].astype(np.float64)) for i in range(3)]
    np.testing.assert_allclose(got, want, rtol=0, atol=TOL)


def test_ssim_identical_and_int16_residuals():
    rng = np.random.default_rng(5)
    res = rng.integers(-255, 256, size=(2, 40, 64)).astype(np.int16)
    dev = torch.from_numpy(res).cuda()
    same = b.ssim(dev, dev.float()).cpu().numpy()
    np.testing.assert_allclose(same, 1.0, atol=1e-12)
    rec = (res * 0.5).astype(np.float32)
    got = b.ssim(dev, torch.from_numpy(rec).cuda()).cpu().numpy()
    want = [m.ssim(res[i].astype(np.float64), rec[i].astype(np.float64)) for i in range(2)]
    np.testing.assert_allclose(got, want, rtol=0, atol=TOL)
