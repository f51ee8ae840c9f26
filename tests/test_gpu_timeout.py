"""Failure detection on the GPU: the library's bounded waits give up, the
time-out is reported once, and the context stays usable.

No GPU fault is provoked.  The test hook cdct_set_fault_injection makes the
fused pipelined kernel arm its staging barriers without issuing any bulk
copy (mode bit 0), or the training GEMM skip its tensor-core MMAs and their
commit (bit 1), with a wait limit of about a millisecond: nothing is ever in
flight, every wait simply runs out, the kernel records the error word and
returns.  cdct_check_device must then report CDCT_ETIMEOUT exactly once, and
the next ordinary call on the same context must match the CPU oracle.
"""
import numpy as np
import pytest

from oracle import cnn
from oracle import pipeline as pl
from paper_2207_11638_gb300 import binding as b
from paper_2207_11638_gb300 import synth
from tests.cnn_util import to_oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LIMIT = 1 << 21          # SM cycles: about a millisecond


@pytest.fixture(autouse=True)
def _hook_off():
    b.set_fault_injection(0)
    assert b.device_status() == b.CDCT_OK
    yield
    b.set_fault_injection(0)
    b.device_status()


@pytest.mark.parametrize("n,variant", [(8, "hat"), (16, "tilde"), (32, "hat")])
def test_stage_wait_times_out_once_then_recovers(n, variant):
    img = synth.ar1_image(96, 160, 0.95, seed=3)
    dev = torch.from_numpy(img).cuda()
    plan = b.Plan(n, variant)
    r = n * n // 4
    b.set_fault_injection(1, LIMIT)
    rec, _, ps = plan.fwd_zonal_inv(dev, r)
    assert b.device_status() == b.CDCT_ETIMEOUT
    assert b.device_status() == b.CDCT_OK            # reported once, then cleared
    assert np.isnan(float(ps.cpu()[0]))               # unfinished units' partials are NaN
    b.set_fault_injection(0)
    rec, _, ps = plan.fwd_zonal_inv(dev, r)
    assert b.device_status() == b.CDCT_OK
    ref = pl.fzi_integer(img, n, variant, r)
    np.testing.assert_array_equal(rec.cpu().numpy()[0], ref["recon"].astype(np.float32))
    want = pl.psnr_from_sse(pl.sse_integer(img, ref["z"], n), n, img.size)
    assert abs(float(ps.cpu()[0]) - want) <= 1e-4


def test_batch_stage_wait_times_out_once_then_recovers():
    imgs = [synth.ar1_image(h, w, 0.9, seed=20 + h) for h, w in ((40, 64), (96, 128))]
    devs = [torch.from_numpy(x).cuda() for x in imgs]
    recs = [torch.empty(x.shape, dtype=torch.float32, device="cuda") for x in imgs]
    plan = b.Plan(16, "hat")
    batch = b.Batch(plan, devs, recs)
    b.set_fault_injection(1, LIMIT)
    batch.run(64)
    assert b.device_status() == b.CDCT_ETIMEOUT
    assert b.device_status() == b.CDCT_OK
    b.set_fault_injection(0)
    batch.run(64)
    assert b.device_status() == b.CDCT_OK
    for x, rc in zip(imgs, recs):
        ref = pl.fzi_integer(x, 16, "hat", 64)
        np.testing.assert_array_equal(rc.cpu().numpy(), ref["recon"].astype(np.float32))


def test_gemm_commit_wait_times_out_once_then_recovers():
    B = 64
    regions = torch.from_numpy(synth.residual_regions_32(B, seed=12)).cuda()
    rng = np.random.default_rng(5)
    labels_h = rng.integers(0, 17, size=(2, B)).astype(np.uint8)
    labels = torch.from_numpy(labels_h).cuda()
    flat = synth.cnn_init_params(9, bias_std=0.1)
    net = b.Cnn(torch.from_numpy(flat).cuda())
    b.set_fault_injection(2, LIMIT)
    net.grad(regions, (0, 1), labels)
    assert b.device_status() == b.CDCT_ETIMEOUT
    assert b.device_status() == b.CDCT_OK
    b.set_fault_injection(0)
    g, loss = net.grad(regions, (0, 1), labels)
    assert b.device_status() == b.CDCT_OK
    ref_loss, _, _ = cnn.loss_and_grad(to_oracle(flat), regions.cpu().numpy(), labels_h, (0, 1), None, 0.0, bf=True)
    assert abs(float(loss.cpu()[0]) - ref_loss) <= 1e-4 * max(1.0, abs(ref_loss))
