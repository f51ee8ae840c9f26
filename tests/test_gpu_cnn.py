"""CNN size selector on the GPU against the CPU oracle (oracle/cnn.py), through the C ABI.

Tolerances.  Both sides round the same values to bfloat16 at the same
points; the GPU accumulates in float32 (tensor-core order), the oracle in
float64.  A rounding decision can therefore flip by one bfloat16 unit (2^-8
relative) where a pre-rounding value lies within float32 error of a rounding
midpoint.  Such flips are rare and each moves a logit by about |w| 2^-8, so
logits are held to 2e-2 absolute (on logits of size ~1-10) and gradients to
2e-2 of each tensor's largest entry (and 1e-2 in relative Frobenius norm).
Labels, an argmax, must agree wherever the oracle's best logit leads the
second by more than twice the logit tolerance; elsewhere the GPU's label must
be within that tolerance of the oracle's best.
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

TOL_LOGIT = 2e-2
TOL_GRAD = 2e-2


def _net(seed):
    flat = synth.cnn_init_params(seed, bias_std=0.1)
    net = b.Cnn(torch.from_numpy(flat).cuda())
    net.pack()
    return net, flat


def _check_labels(lab, ref_logits):
    srt = np.sort(ref_logits, axis=-1)
    margin = srt[..., -1] - srt[..., -2]
    best = ref_logits.argmax(axis=-1)
    sure = margin > 2 * TOL_LOGIT
    assert np.array_equal(lab[sure], best[sure])
    picked = np.take_along_axis(ref_logits, lab[..., None].astype(np.int64), axis=-1)[..., 0]
    assert np.all(srt[..., -1] - picked <= 2 * TOL_LOGIT)


@pytest.mark.parametrize("n_regions", [1, 16, 37])
def test_infer_matches_oracle(n_regions):
    regions = synth.residual_regions_32(n_regions, seed=11)
    net, flat = _net(7)
    slots = (0, 1, 2)
    lab, lg, mg = net.infer(torch.from_numpy(regions).cuda(), slots, logits=True, margin=True)
    torch.cuda.synchronize()
    ref = cnn.forward(to_oracle(flat), regions, slots, bf=True)["logits"]
    got = lg.cpu().numpy().astype(np.float64)
    err = float(np.max(np.abs(got - ref)))
    print(f"infer n={n_regions}: max |logit - oracle| = {err:.3e}, logit range {ref.min():.2f}..{ref.max():.2f}")
    assert err <= TOL_LOGIT
    lab = lab.cpu().numpy()
    _check_labels(lab, ref)
    # the margin output is the kernel's own top-2 gap
    srt = np.sort(got, axis=-1)
    np.testing.assert_allclose(mg.cpu().numpy(), srt[..., -1] - srt[..., -2], atol=1e-6)
    assert np.array_equal(lab, got.argmax(axis=-1))


def test_infer_many_groups_per_cta_matches_oracle():
    """3000 regions: more groups of 16 than SMs, so CTAs run two groups through
    the inference pipeline (pairs and the per-group head crossing a group
    boundary), and the last group is half full.

    The pipeline is checked exactly: regions at and around group boundaries,
    run again on their own (one group each), give the same logits bit for bit.
    Against the oracle the bound follows the rounding-flip model of this
    file: almost every region agrees to float32 rounding, and the few where a
    bfloat16 rounding decision flipped (sometimes twice in one region) stay
    within twice the logit tolerance."""
    n = 3000
    regions = synth.residual_regions_32(n, seed=23)
    net, flat = _net(9)
    slots = (0, 1, 2)
    lab, lg, mg = net.infer(torch.from_numpy(regions).cuda(), slots, logits=True, margin=True)
    got = lg.cpu().numpy()
    pick = np.array([0, 15, 16, 17, 31, 32, 2431, 2432, 2447, 2448, 2991, 2992, n - 1])
    _, lg1, _ = net.infer(torch.from_numpy(np.ascontiguousarray(regions[pick])).cuda(), slots, logits=True,
                          margin=True)
    assert np.array_equal(lg1.cpu().numpy(), got[:, pick])
    ref = cnn.forward(to_oracle(flat), regions, slots, bf=True)["logits"]
    e = np.abs(got.astype(np.float64) - ref).max(axis=(0, 2))            # per region
    print(f"infer n={n}: per-region max |logit - oracle| quantiles 50/99/100 % = "
          f"{np.quantile(e, 0.5):.2e} / {np.quantile(e, 0.99):.2e} / {e.max():.2e}")
    assert np.quantile(e, 0.9) <= 1e-5
    assert np.mean(e > 1e-3) <= 0.05
    assert e.max() <= 2 * TOL_LOGIT
    srt = np.sort(got.astype(np.float64), axis=-1)
    np.testing.assert_allclose(mg.cpu().numpy(), srt[..., -1] - srt[..., -2], atol=1e-6)
    _check_labels(lab.cpu().numpy(), ref)


@pytest.mark.parametrize("dtype", ["u8", "i16"])
def test_infer_ragged_images_and_slots(dtype):
    """Regions of images whose sides are not multiples of 32 (edge-replicated), and slot 3."""
    rng = np.random.default_rng(3)
    if dtype == "u8":
        imgs = np.stack([synth.ar1_image(70, 100, 0.9, seed=s) for s in (5, 6)])
    else:
        imgs = rng.integers(-255, 256, size=(2, 45, 33)).astype(np.int16)
    net, flat = _net(8)
    slots = (3, 0)
    lab, lg = net.infer(torch.from_numpy(imgs).cuda(), slots, logits=True)
    torch.cuda.synchronize()
    padded = pl.pad_replicate(imgs, 32)
    regs = padded.reshape(2, padded.shape[1] // 32, 32, padded.shape[2] // 32, 32).swapaxes(2, 3).reshape(-1, 32, 32)
    ref = cnn.forward(to_oracle(flat), regs, slots, bf=True)["logits"]
    err = float(np.max(np.abs(lg.cpu().numpy() - ref)))
    print(f"infer ragged {dtype}: max |logit - oracle| = {err:.3e}")
    assert err <= TOL_LOGIT
    _check_labels(lab.cpu().numpy(), ref)


def test_grad_matches_oracle():
    B = 64
    regions = synth.residual_regions_32(B, seed=12)
    rng = np.random.default_rng(5)
    slots = (0, 1, 3)
    labels = rng.integers(0, 17, size=(3, B)).astype(np.uint8)
    # partition costs: 128-bit integers around 2^70, as (low, high) words
    lo = rng.integers(0, 2 ** 63, size=(3, B, 17), dtype=np.int64)
    hi = rng.integers(40, 80, size=(3, B, 17), dtype=np.int64)
    words = np.stack([lo, hi], axis=-1)
    costs = np.empty((3, B, 17), dtype=object)
    for idx in np.ndindex(costs.shape):
        costs[idx] = int(hi[idx]) << 64 | int(lo[idx])
    net, flat = _net(9)
    g, loss = net.grad(torch.from_numpy(regions).cuda(), slots, torch.from_numpy(labels).cuda(),
                       torch.from_numpy(words).cuda(), mu=0.5)
    torch.cuda.synchronize()
    ref_loss, ref_g, _ = cnn.loss_and_grad(to_oracle(flat), regions, labels, slots, cnn.normalised_regret(costs),
                                           0.5, bf=True)
    got = to_oracle(g.cpu().numpy())
    lv = float(loss.cpu()[0])
    print(f"grad: loss {lv:.6f} vs oracle {ref_loss:.6f}")
    assert abs(lv - ref_loss) <= 1e-4 * max(1.0, abs(ref_loss))
    for name, _ in cnn.PARAM_SHAPES:
        r, q = ref_g[name], got[name]
        scale = float(np.max(np.abs(r)))
        err = float(np.max(np.abs(q - r)))
        rel = float(np.linalg.norm(q - r) / max(np.linalg.norm(r), 1e-30))
        print(f"  {name:8s} max|g| {scale:.3e}  max err {err:.3e}  rel norm {rel:.3e}")
        if name == "fc1_q":
            assert not np.any(q[:, 2])          # slot 2 not in the batch: no gradient
        assert err <= TOL_GRAD * scale + 1e-8, name
        assert rel <= 1e-2, name


def test_grad_is_deterministic():
    B = 128
    regions = torch.from_numpy(synth.residual_regions_32(B, seed=14)).cuda()
    labels = torch.randint(0, 17, (2, B), dtype=torch.uint8, device="cuda")
    net, _ = _net(10)
    g1, l1 = net.grad(regions, (1, 2), labels)
    g1, l1 = g1.clone(), l1.clone()
    g2, l2 = net.grad(regions, (1, 2), labels)
    torch.cuda.synchronize()
    assert torch.equal(g1, g2) and torch.equal(l1, l2)


def test_adam_matches_oracle():
    flat = synth.cnn_init_params(11)
    rng = np.random.default_rng(6)
    grads = [rng.standard_normal(flat.size).astype(np.float32) * s for s in (1e-2, 3e-3, 1e-1)]
    net = b.Cnn(torch.from_numpy(flat).cuda())
    p = {"w": flat.astype(np.float64)}
    st = {}
    for gi in grads:
        net.adam(torch.from_numpy(gi).cuda(), lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8)
        cnn.adam_step(p, {"w": gi.astype(np.float64)}, st, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8)
    torch.cuda.synchronize()
    np.testing.assert_allclose(net.params.cpu().numpy(), p["w"], rtol=2e-6, atol=2e-8)
    # m is a float32 running sum of terms of size |g| <= ~0.5: its rounding error is ~2^-24 |g|
    np.testing.assert_allclose(net.m.cpu().numpy(), st["m"]["w"], rtol=1e-5, atol=1e-8)


def test_training_on_rd_labels_reduces_the_loss():
    """A few hundred GPU steps on labels from the exhaustive search fit the training set."""
    regions = torch.from_numpy(synth.residual_regions_32(2048, seed=13)).cuda()
    qs = (8, 16, 32)
    labels = b.RdSearch("hat").search(regions, qs)
    net = b.Cnn(torch.from_numpy(synth.cnn_init_params(1)).cuda())
    B = 256
    losses = []
    for step in range(240):
        k = step % (2048 // B)
        loss = net.train_step(regions[k * B:(k + 1) * B], (0, 1, 2), labels[:, k * B:(k + 1) * B].contiguous(),
                              lr=2e-3)
        losses.append(loss.clone())
    torch.cuda.synchronize()
    lv = [float(x.cpu()[0]) for x in losses]
    first, last = np.mean(lv[:8]), np.mean(lv[-8:])
    print(f"training: mean loss of the first epoch {first:.4f}, of the last {last:.4f}")
    assert np.all(np.isfinite(lv))
    assert last < 0.8 * first
    # better than the best constant predictor: the entropy of each slot's label frequencies
    lab = labels.cpu().numpy()
    h = []
    for i in range(3):
        f = np.bincount(lab[i], minlength=17) / lab.shape[1]
        h.append(-np.sum(f[f > 0] * np.log(f[f > 0])))
    print(f"label entropy per slot {np.round(h, 4).tolist()} (mean {np.mean(h):.4f})")
    assert last < np.mean(h)
    net.pack()
    pred = net.infer(regions, (0, 1, 2))
    acc = float((pred == labels).float().mean())
    major = np.mean([np.bincount(lab[i], minlength=17).max() / lab.shape[1] for i in range(3)])
    print(f"training-set label accuracy {acc:.3f} (most frequent label per slot, averaged: {major:.3f})")


def test_checkpoint_resume_is_bit_identical(tmp_path):
    """Save the training state mid-run, resume it in a fresh selector: the weights after
    the remaining steps equal those of the uninterrupted run bit for bit."""
    regions = torch.from_numpy(synth.residual_regions_32(512, seed=15)).cuda()
    qs, slots = (8, 16, 32), (0, 1, 2)
    labels, costs = b.RdSearch("hat").search(regions, qs, costs=True)

    def step(net, k):
        i = k % 2
        net.train_step(regions[i * 256:(i + 1) * 256], slots, labels[:, i * 256:(i + 1) * 256].contiguous(),
                       lr=1e-3, costs=costs[:, i * 256:(i + 1) * 256].contiguous(), mu=10.0)

    net = b.Cnn(torch.from_numpy(synth.cnn_init_params(3)).cuda())
    for k in range(5):
        step(net, k)
    path = str(tmp_path / "selector.ckpt")
    net.save(path, {"next_batch": 5})
    for k in range(5, 10):
        step(net, k)
    torch.cuda.synchronize()
    net2, extra = b.Cnn.load(path)
    assert extra == {"next_batch": 5} and net2.step == 5
    for k in range(extra["next_batch"], 10):
        step(net2, k)
    torch.cuda.synchronize()
    assert torch.equal(net2.params, net.params) and torch.equal(net2.m, net.m) and torch.equal(net2.v, net.v)
