"""The benchmark's own workload at full size, in the launch configuration it
times, against the oracle on sampled outputs.

64 frames of 1920x1080 4:2:0 int16 residuals (the video-frame workload,
398 MB resident), the bench's step object (workload.FrameStep: one fused
launch per plane set and pass, the persistent pipelined kernel) and every
pass N in {8, 16, 32} x {T~, T^} at r = N^2/4.  Blocks are independent, so
the oracle run on a 64 x 64 crop whose corner is a multiple of 32 gives the
same reconstruction as on the whole frame; crops are taken inside the frame
and at its ragged bottom-right corner (1080 and 540 are not multiples of 32).
Reconstructions must equal the float32 rounding of the oracle's exact value;
PSNRs of sampled whole planes must be within 1e-4 dB.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import pipeline as pl
from paper_2207_11638_gb300 import workload as wl

pytestmark = pytest.mark.gpu
PSNR_TOL_DB = 1e-4


@pytest.fixture(scope="module")
def frames(tmp_path_factory):
    from paper_2207_11638_gb300 import autotune
    luma_h, chroma_h = wl.host_batch()
    luma = torch.from_numpy(luma_h).cuda()
    step = wl.FrameStep(luma, torch.from_numpy(chroma_h).cuda())
    cache = str(tmp_path_factory.mktemp("tune") / "autotune.json")
    for (n, _), plan in step.plans.items():       # the bench's schedules: tuned on the luma planes
        autotune.tune(plan, luma, wl.zonal_r(n), path=cache)
    return luma_h, chroma_h, step


def crops(h, w, rng, k=3):
    """(y0, x0) corners: k random interior ones on the 32-grid and the ragged bottom-right one."""
    out = [(int(rng.integers(0, (h - 64) // 32)) * 32, int(rng.integers(0, (w - 64) // 32)) * 32) for _ in range(k)]
    out.append(((h - 1) // 32 * 32 - 32, (w - 1) // 32 * 32 - 32))
    return out


@pytest.mark.parametrize("n,variant", wl.PASSES)
def test_full_batch_sampled_against_oracle(frames, n, variant):
    luma_h, chroma_h, step = frames
    rng = np.random.default_rng(n * 13 + len(variant))
    r = wl.zonal_r(n)
    step.launch_pass((n, variant))
    torch.cuda.synchronize()
    for planes, recon, psnr in ((luma_h, step.recon_y, step.psnr_y[(n, variant)]),
                                (chroma_h, step.recon_c, step.psnr_c[(n, variant)])):
        h, w = planes.shape[1:]
        picks = rng.choice(planes.shape[0], size=2, replace=False)
        rec_dev = recon[torch.as_tensor(picks, device=recon.device)].cpu().numpy()
        for j, f in enumerate(picks):
            for y0, x0 in crops(h, w, rng):
                crop = planes[f, y0:y0 + 64, x0:x0 + 64]
                ref = pl.fzi_integer(crop[None], n, variant, r)["recon"][0]
                got = rec_dev[j, y0:y0 + 64, x0:x0 + 64]
                np.testing.assert_array_equal(got, ref.astype(np.float32))
        # whole-plane PSNR of the first pick
        f = int(picks[0])
        z = pl.fzi_integer(planes[f][None], n, variant, r)["z"]
        want = pl.psnr_from_sse(pl.sse_integer(planes[f], z[0], n), n, h * w)
        got = float(psnr[f].cpu())
        assert math.isfinite(want) and abs(got - want) <= PSNR_TOL_DB, (got, want)
