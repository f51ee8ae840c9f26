"""GPU rate-distortion quadtree search against the oracle (oracle/rd.py).

Labels and the 17 partition costs are exact integers on both sides, so they
must agree bit for bit: on seeded residual regions of the 32 x 32 region
workload (differences of AR(1) images), on images whose size is not a
multiple of 32 (edge-replicated regions, distortion over valid pixels), on
extreme and degenerate content, for both variants and several lambdas; and,
at the full 200 000-region size in the launch configuration the benchmark
times, on sampled regions.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rd
from paper_2207_11638_gb300 import binding as b
from paper_2207_11638_gb300 import synth

pytestmark = pytest.mark.gpu
QS = (8, 16, 32)


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run(variant, imgs, qs, kappa=(1, 2)):
    s = b.RdSearch(variant, *kappa)
    dev = torch.from_numpy(np.ascontiguousarray(imgs)).cuda()
    labels, pc = s.search(dev, qs, costs=True)
    torch.cuda.synchronize()
    return labels.cpu().numpy(), b.rd_cost_ints(pc.cpu().numpy())


def compare(got, want):
    gl, gc = got
    wl, wc = want
    np.testing.assert_array_equal(gl, wl)
    assert gc == [[list(map(int, r)) for r in q] for q in wc]


@pytest.mark.parametrize("variant", ("tilde", "hat"))
def test_rd_regions_match_oracle(variant):
    regs = synth.residual_regions_32(24, seed=4)
    compare(run(variant, regs, QS), rd.rd_search(regs, variant, QS))


@pytest.mark.parametrize("kappa", [(0, 0), (1, 4), (3, 1), (1024, 0)])
def test_rd_lambda_range(kappa):
    regs = synth.residual_regions_32(8, seed=21)
    compare(run("hat", regs, (4, 24), kappa), rd.rd_search(regs, "hat", (4, 24), *kappa))


@pytest.mark.parametrize("dtype,shape", [("u8", (1, 70, 100)), ("i16", (2, 33, 65)), ("u8", (1, 5, 7)),
                                         ("i16", (1, 64, 40))])
def test_rd_ragged_images_match_oracle(dtype, shape):
    rng = np.random.default_rng(sum(shape))
    if dtype == "u8":
        imgs = rng.integers(0, 256, size=shape).astype(np.uint8)
    else:
        imgs = rng.integers(-255, 256, size=shape).astype(np.int16)
    compare(run("hat", imgs, (8, 32)), rd.rd_search_image(imgs.astype(np.int64), "hat", (8, 32)))


def test_rd_extreme_and_degenerate_regions():
    regs = np.zeros((6, 32, 32), dtype=np.int16)
    regs[1] = 255
    regs[2] = -255
    yy, xx = np.mgrid[:32, :32]
    regs[3] = np.where((yy + xx) % 2 == 0, 255, -255)             # checkerboard: highest frequencies
    regs[4] = np.where(yy < 16, 255, -255)
    regs[5, :16, :16] = 200                                        # one busy quadrant
    for variant in ("tilde", "hat"):
        compare(run(variant, regs, (1, 8, 4096)), rd.rd_search(regs, variant, (1, 8, 4096)))


def test_rd_full_size_sampled():
    """200 000 regions in one launch (the region workload's size); sampled regions checked."""
    n = 200_000
    regs = synth.residual_regions_32(n, seed=4)
    s = b.RdSearch("hat")
    dev = torch.from_numpy(regs).cuda()
    labels, pc = s.search(dev, QS, costs=True)
    torch.cuda.synchronize()
    lab = labels.cpu().numpy()
    assert lab.shape == (3, n) and lab.max() < rd.N_PARTITIONS
    idx = np.random.default_rng(0).choice(n, size=12, replace=False)
    want_l, want_c = rd.rd_search(regs[idx], "hat", QS)
    np.testing.assert_array_equal(lab[:, idx], want_l)
    got_c = b.rd_cost_ints(pc[:, torch.from_numpy(idx).cuda()].cpu().numpy())
    assert got_c == [[list(map(int, r)) for r in q] for q in want_c]
    # every label's cost is the minimum of its region's 17 costs
    pcs = pc[:, :2000].cpu().numpy().astype(np.uint64)
    hi, lo = pcs[..., 1], pcs[..., 0]
    for qi in range(3):
        for r in range(2000):
            costs = [int(h) << 64 | int(l) for l, h in zip(lo[qi, r], hi[qi, r])]
            assert costs[lab[qi, r]] == min(costs)
