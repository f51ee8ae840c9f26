"""The learned size selector earns its place: trained briefly on the exhaustive
search's labels, on regions it has not seen its decision (the network, with
the exhaustive search re-deciding the 40 % of regions whose smallest margin
is lowest; the threshold is taken from the training regions) must

* code them at a lower Lagrangian RD cost J = D + lambda R than the best
  fixed partition (all 32 x 32, all 16 x 16 or all 8 x 8 blocks), and
* decide faster than the exhaustive search it replaces.

The network alone must beat the mean RD cost of the three fixed partitions.

The RD cost of a decision is measured by the library's own coder
(cdct_rd_evaluate): the same J the search minimises, so the exhaustive
labels are the optimum and every other decision costs at least as much.
"""
import numpy as np
import pytest

from paper_2207_11638_gb300 import binding as b
from paper_2207_11638_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

QS = (8, 16, 32)
SLOTS = (0, 1, 2)


def _j(words):
    """(low, high) int64 word pairs of 128-bit costs -> float64 totals per slot."""
    w = words.cpu().numpy().astype(np.uint64)
    return (w[..., 1].astype(np.float64) * 2.0 ** 64 + w[..., 0].astype(np.float64)).sum(axis=1)


def _timed(fn, reps=5):
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def test_learned_decision_beats_fixed_partitions_and_the_search_time():
    n, n_train, B = 49152, 40960, 512
    regs_h = synth.residual_regions_32(n, seed=21)
    regs_h = regs_h[np.random.default_rng(5).permutation(n)]
    regs = torch.from_numpy(regs_h).cuda()
    search = b.RdSearch("hat")
    labels, costs = search.search(regs, QS, costs=True)
    net = b.Cnn(torch.from_numpy(synth.cnn_init_params(3)).cuda())
    steps = n_train // B
    epochs = 8
    for ep in range(epochs):
        for k in range(steps):
            it = ep * steps + k
            lr = 2e-3 * 0.5 * (1.0 + np.cos(np.pi * it / (epochs * steps)))
            net.train_step(regs[k * B:(k + 1) * B], SLOTS, labels[:, k * B:(k + 1) * B].contiguous(), lr=lr,
                           costs=costs[:, k * B:(k + 1) * B].contiguous(), mu=300.0)
    torch.cuda.synchronize()
    b.check_device()
    net.pack()
    _, mg_train = net.infer(regs[:n_train], SLOTS, margin=True)
    tau = float(torch.quantile(mg_train.min(dim=0).values.float(), 0.4))
    held = regs[n_train:].contiguous()
    lab_ex = labels[:, n_train:].contiguous()

    def decide():
        lab, mg = net.infer(held, SLOTS, margin=True)
        idx, cnt = b.cnn_select(mg, tau)
        search.search_subset(held, QS, idx, cnt, lab)
        return lab, cnt

    lab_l, cnt = decide()
    lab_cnn = net.infer(held, SLOTS)
    j_ex = _j(search.evaluate(held, QS, lab_ex)[0])
    j_l = _j(search.evaluate(held, QS, lab_l)[0])
    j_cnn = _j(search.evaluate(held, QS, lab_cnn)[0])
    j_fixed = {name: _j(search.evaluate(held, QS, torch.full_like(lab_ex, lab))[0])
               for name, lab in (("all_32", 0), ("all_16", 1), ("all_8", 16))}
    pct = lambda j: 100.0 * (j.sum() / j_ex.sum() - 1.0)
    print(f"held-out RD cost over the exhaustive search: learned decision +{pct(j_l):.3f} % "
          f"({int(cnt.cpu()[0])} of {n - n_train} regions re-searched), network alone +{pct(j_cnn):.3f} %, fixed "
          + ", ".join(f"{k} +{pct(v):.3f} %" for k, v in j_fixed.items()))
    assert np.all(j_ex <= j_l) and np.all(j_ex <= j_cnn)    # the search is the optimum of the same J
    assert j_l.sum() < min(v.sum() for v in j_fixed.values())
    assert j_cnn.sum() < np.mean([v.sum() for v in j_fixed.values()])
    # decision time over the same held-out regions
    ms_l = _timed(decide)
    ms_search = _timed(lambda: search.search(held, QS))
    print(f"decision over {n - n_train} regions: learned {ms_l:.3f} ms, exhaustive search {ms_search:.3f} ms")
    assert ms_l < ms_search
