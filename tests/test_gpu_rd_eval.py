"""Coding with a given quadtree (cdct_rd_evaluate), the subset search and the
selector's fallback pick (cdct_cnn_select) against the oracle, through the C ABI.

Costs, distortions and rates are exact integers on both sides: bit-exact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import pipeline as pl
from oracle import rd
from paper_2207_11638_gb300 import binding as b
from paper_2207_11638_gb300 import synth

pytestmark = pytest.mark.gpu
QS = (8, 16, 32)


def oracle_partition(region, label, variant, q, kappa=(1, 2), valid=None):
    """(J', D on the J' scale, R) of one region coded with one labelled quadtree, block by block."""
    lam = rd.lambda_scaled(q, *kappa)
    flags = 1 if label == 0 else 5
    j, d, r = lam * flags, 0, flags
    for y, x, n in rd.partition_blocks(label):
        v = None if valid is None else valid[y:y + n, x:x + n]
        jb, db, rb = rd.block_cost(region[y:y + n, x:x + n], variant, q, *kappa, valid=v)
        j += jb
        d += (32 // n) ** 4 * db
        r += rb
    return j, d, r


def words(a):
    a = np.asarray(a).astype(np.uint64)
    return [int(h) << 64 | int(lo) for lo, h in zip(a[..., 0].ravel(), a[..., 1].ravel())]


@pytest.mark.parametrize("variant", ("tilde", "hat"))
def test_evaluate_matches_oracle(variant):
    regs = synth.residual_regions_32(12, seed=31)
    rng = np.random.default_rng(7)
    labels = rng.integers(0, 17, size=(len(QS), len(regs))).astype(np.uint8)
    labels[:, 0] = 0
    labels[:, 1] = 16
    labels[:, 2] = 1
    s = b.RdSearch(variant)
    dev = torch.from_numpy(regs).cuda()
    cost, dist, bits = s.evaluate(dev, QS, torch.from_numpy(labels).cuda())
    torch.cuda.synchronize()
    gc, gd, gb = words(cost.cpu().numpy()), words(dist.cpu().numpy()), bits.cpu().numpy().ravel().tolist()
    k = 0
    for qi, q in enumerate(QS):
        lam = rd.lambda_scaled(q, 1, 2)
        for ri, reg in enumerate(regs):
            lab = int(labels[qi, ri])
            j, d, r = oracle_partition(reg, lab, variant, q)
            # the block-by-block sum is the search's own partition cost
            assert j == rd.partition_costs(rd.region_block_costs(reg, variant, q, 1, 2), lam)[lab]
            assert (gc[k], gd[k], gb[k]) == (j, d, r), (q, ri, lab)
            k += 1


def test_evaluate_ragged_image_matches_oracle():
    rng = np.random.default_rng(8)
    img = rng.integers(-255, 256, size=(1, 45, 70)).astype(np.int16)
    s = b.RdSearch("hat")
    dev = torch.from_numpy(img).cuda()
    n = s.region_count(dev)
    labels = rng.integers(0, 17, size=(2, n)).astype(np.uint8)
    cost, dist, bits = s.evaluate(dev, (16, 24), torch.from_numpy(labels).cuda())
    torch.cuda.synchronize()
    padded = pl.pad_replicate(img, 32)[0]
    valid = np.zeros(padded.shape, dtype=bool)
    valid[:45, :70] = True
    gc, gd, gb = words(cost.cpu().numpy()), words(dist.cpu().numpy()), bits.cpu().numpy().ravel().tolist()
    k = 0
    for qi, q in enumerate((16, 24)):
        for t in range(n):
            ty, tx = divmod(t, padded.shape[1] // 32)
            sl = (slice(ty * 32, ty * 32 + 32), slice(tx * 32, tx * 32 + 32))
            want = oracle_partition(padded[sl], int(labels[qi, t]), "hat", q, valid=valid[sl])
            assert (gc[k], gd[k], gb[k]) == want
            k += 1


def test_evaluate_of_search_labels_is_the_minimum():
    regs = torch.from_numpy(synth.residual_regions_32(3000, seed=32)).cuda()
    s = b.RdSearch("hat")
    labels, pc = s.search(regs, QS, costs=True)
    cost, _, _ = s.evaluate(regs, QS, labels)
    torch.cuda.synchronize()
    pcs = b.rd_cost_ints(pc.cpu().numpy())
    got = words(cost.cpu().numpy())
    want = [min(pcs[qi][r]) for qi in range(len(QS)) for r in range(3000)]
    assert got == want


def test_subset_search_matches_full_search():
    regs = torch.from_numpy(synth.residual_regions_32(1000, seed=33)).cuda()
    s = b.RdSearch("hat")
    full, full_pc = s.search(regs, QS, costs=True)
    pick = np.arange(5, 1000, 7)
    idx = torch.from_numpy(pick.astype(np.int64)).cuda()
    cnt = torch.tensor([len(pick)], dtype=torch.int64, device="cuda")
    lab = torch.full((len(QS), 1000), 255, dtype=torch.uint8, device="cuda")
    pc = torch.zeros_like(full_pc)
    s.search_subset(regs, QS, idx, cnt, lab, pc)
    torch.cuda.synchronize()
    lab, full = lab.cpu().numpy(), full.cpu().numpy()
    assert np.array_equal(lab[:, pick], full[:, pick])
    rest = np.setdiff1d(np.arange(1000), pick)
    assert np.all(lab[:, rest] == 255)
    assert torch.equal(pc[:, pick].cpu(), full_pc[:, pick].cpu())
    # an empty list and out-of-range numbers change nothing
    cnt.zero_()
    s.search_subset(regs, QS, idx, cnt, lab_t := torch.full((len(QS), 1000), 7, dtype=torch.uint8, device="cuda"))
    bad = torch.tensor([-1, 1000, 5_000_000], dtype=torch.int64, device="cuda")
    s.search_subset(regs, QS, bad, torch.tensor([3], dtype=torch.int64, device="cuda"), lab_t)
    torch.cuda.synchronize()
    assert bool((lab_t == 7).all())


def test_cnn_select_picks_low_margins():
    rng = np.random.default_rng(9)
    margin = rng.exponential(1.0, size=(3, 5000)).astype(np.float32)
    idx, cnt = b.cnn_select(torch.from_numpy(margin).cuda(), 0.25)
    torch.cuda.synchronize()
    n = int(cnt.cpu()[0])
    got = np.sort(idx[:n].cpu().numpy())
    want = np.flatnonzero(margin.min(axis=0) < 0.25)
    assert np.array_equal(got, want)
