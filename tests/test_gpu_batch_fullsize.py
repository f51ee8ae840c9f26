"""Descriptor-table launches at the scale of the uneven benchmark, against the
oracle on sampled whole images.

512 images from the benchmark's own generator (u8 AR(1) images, sides
log-uniform in [64, 2048], multiples of 32), laid out in one device arena as
the benchmark lays them out, one batch per pass N in {8, 16, 32} x {T~, T^}
at r = N^2 / 4 (the benchmark's launch configuration, default schedule).
Per pass, whole images are compared with the oracle: the smallest and the
largest, one narrow enough to be packed several block rows per work unit,
one between half a unit and a unit wide, and one wider than a unit (several
segments per block row).  Reconstructions must equal the float32 rounding of
the oracle's exact value; PSNRs agree within 1e-4 dB, and every PSNR of the
batch is finite.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench
from oracle import pipeline as pl
from paper_2207_11638_gb300 import binding as b
from paper_2207_11638_gb300 import workload as wl

pytestmark = pytest.mark.gpu
PSNR_TOL_DB = 1e-4
S = {8: 128, 16: 32, 32: 8}      # blocks per work unit


@pytest.fixture(scope="module")
def batch_images():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    host = bench.uneven_host_images(512)
    offs, total = [], 0
    for im in host:
        offs.append(total)
        total += (im.size + 255) // 256 * 256
    arena_in = torch.empty(total, dtype=torch.uint8, device="cuda")
    arena_out = torch.empty(total, dtype=torch.float32, device="cuda")
    imgs, recs = [], []
    for im, o in zip(host, offs):
        t = arena_in[o:o + im.size].view(im.shape)
        t.copy_(torch.from_numpy(im))
        imgs.append(t)
        recs.append(arena_out[o:o + im.size].view(im.shape))
    return host, imgs, recs


def picks(host, n):
    nbx = [-(-im.shape[1] // n) for im in host]
    sizes = [im.size for im in host]
    out = {int(np.argmin(sizes)), int(np.argmax(sizes))}
    for cond in (lambda k: k <= S[n] // 2, lambda k: S[n] // 2 < k < S[n], lambda k: k > S[n]):
        hit = next((i for i, k in enumerate(nbx) if cond(k)), None)
        if hit is not None:
            out.add(hit)
    return sorted(out)


@pytest.mark.parametrize("n,variant", wl.PASSES)
def test_uneven_batch_sampled_against_oracle(batch_images, n, variant):
    host, imgs, recs = batch_images
    r = wl.zonal_r(n)
    batch = b.Batch(b.Plan(n, variant), imgs, recs)
    ps = batch.run(r)
    torch.cuda.synchronize()
    b.check_device()
    ps = ps.cpu().numpy()
    assert np.all(np.isfinite(ps)) and ps.min() > 0
    for i in picks(host, n):
        im = host[i]
        ref = pl.fzi_integer(im, n, variant, r)
        np.testing.assert_array_equal(recs[i].cpu().numpy(), ref["recon"].astype(np.float32))
        want = pl.psnr_from_sse(pl.sse_integer(im, ref["z"], n), n, im.size)
        assert math.isfinite(want) and abs(ps[i] - want) <= PSNR_TOL_DB, (i, ps[i], want)
