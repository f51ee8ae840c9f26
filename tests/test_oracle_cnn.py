"""Pins of the CNN size-selector oracle (oracle/cnn.py).

Each check comes from outside the oracle's own formulas: scipy's
correlate2d for the convolution, torch's float32 -> bfloat16 conversion for
the rounding, central finite differences for every gradient, and closed
forms for pooling, the softmax cross-entropy gradient and Adam's first step.
"""
import math

import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn


def _rand_params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    p = cnn.init_params(seed)
    for k in p:
        if k.endswith("_b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1 * scale
    return p


def test_param_count_and_layout():
    assert cnn.param_count() == 144 + 16 + 4608 + 32 + 9216 + 32 + 64 * 512 + 64 * 4 + 64 + 17 * 64 + 17
    p = cnn.init_params(0)
    assert [k for k, _ in cnn.PARAM_SHAPES] == list(p.keys())


def test_bf16_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    # exact midpoints between neighbouring bfloat16 values: ties go to even
    base = torch.tensor(rng.standard_normal(64).astype(np.float32)).to(torch.bfloat16).to(torch.float32).numpy()
    ulp = np.ldexp(1.0, np.frexp(base.astype(np.float64))[1] - 8)
    mids = (base.astype(np.float64) + 0.5 * ulp).astype(np.float32)
    x = np.concatenate([x, mids, -mids]).astype(np.float32)
    want = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = cnn.bf16(x.astype(np.float64))
    assert np.array_equal(got, want)


def test_conv_matches_scipy_correlate2d():
    rng = np.random.default_rng(2)
    a = rng.standard_normal((2, 7, 9, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    z = cnn.conv3x3(a, w, b)
    for n in range(2):
        for o in range(4):
            want = b[o] + sum(correlate2d(a[n, :, :, i], w[o, :, :, i], mode="same", boundary="fill")
                              for i in range(3))
            assert np.allclose(z[n, :, :, o], want, rtol=1e-12, atol=1e-12)


def test_maxpool_closed_form_and_first_maximum():
    r = np.array([[1, 5, 2, 2],
                  [3, 4, 2, 2],
                  [0, 0, 7, 1],
                  [0, 0, 1, 7]], dtype=np.float64)[None, :, :, None]
    p, arg = cnn.maxpool2(r)
    assert p[0, :, :, 0].tolist() == [[5, 2], [0, 7]]
    # windows in raster order (dy, dx): 5 at (0,1) -> 1; all-2 tie -> first (0); zeros -> 0; 7 tie -> 0
    assert arg[0, :, :, 0].tolist() == [[1, 0], [0, 0]]
    back = cnn.maxpool2_backward(np.array([[[[10.0], [20.0]], [[30.0], [40.0]]]]), arg)
    want = np.zeros((4, 4))
    want[0, 1], want[0, 2], want[2, 0], want[2, 2] = 10, 20, 30, 40
    assert np.array_equal(back[0, :, :, 0], want)


def test_normalised_regret_closed_form():
    costs = np.array([[[10, 12, 10] + [40] * 14]], dtype=object)
    rg = cnn.normalised_regret(costs)
    assert rg.shape == (1, 1, 17)
    assert rg[0, 0, 0] == 0 and rg[0, 0, 2] == 0 and math.isclose(rg[0, 0, 1], 0.2) and math.isclose(rg[0, 0, 5], 3.0)


def test_softmax_cross_entropy_gradient_closed_form():
    # all weights zero: logits = fc2_b for every sample, so dL/dfc2_b = mean(p - onehot)
    p = {k: np.zeros(s) for k, s in cnn.PARAM_SHAPES}
    p["fc2_b"] = np.linspace(-1, 1, 17)
    regions = np.zeros((3, 32, 32))
    labels = np.array([[0, 5, 16], [2, 2, 9]])
    loss, g, _ = cnn.loss_and_grad(p, regions, labels, (0, 3), bf=False)
    e = np.exp(p["fc2_b"] - p["fc2_b"].max())
    prob = e / e.sum()
    onehot_mean = np.bincount(labels.ravel(), minlength=17) / labels.size
    assert np.allclose(g["fc2_b"], prob - onehot_mean, atol=1e-15)
    assert math.isclose(loss, float(np.mean(-np.log(prob[labels.ravel()]))), rel_tol=1e-13)
    for k in ("fc2_w", "fc1_w", "fc1_q", "conv1_w"):
        assert not np.any(g[k])


def _loss(p, regions, labels, slots, rg, mu):
    return cnn.loss_and_grad(p, regions, labels, slots, rg, mu, bf=False)[0]


def test_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    p = _rand_params(3)
    regions = rng.integers(-120, 121, size=(2, 32, 32))
    slots = (0, 2)
    labels = rng.integers(0, 17, size=(2, 2))
    rg = rng.uniform(0, 0.3, size=(2, 2, 17))
    mu = 0.7
    _, g, _ = cnn.loss_and_grad(p, regions, labels, slots, rg, mu, bf=False)
    h = 1e-6
    for name, shape in cnn.PARAM_SHAPES:
        flat = p[name].reshape(-1)
        picks = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        if name == "fc1_q":
            picks = np.array([0 * 4 + 0, 5 * 4 + 2, 9 * 4 + 0, 13 * 4 + 2])   # slots in use
        for i in picks:
            old = flat[i]
            flat[i] = old + h
            lp = _loss(p, regions, labels, slots, rg, mu)
            flat[i] = old - h
            lm = _loss(p, regions, labels, slots, rg, mu)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 + 1e-5 * abs(an), (name, int(i), fd, an)
    # slots not evaluated get no gradient
    assert not np.any(g["fc1_q"][:, [1, 3]])


def test_adam_first_step_closed_form_and_quadratic():
    p = {"w": np.array([0.5, -2.0, 3.0])}
    g = {"w": np.array([0.1, -4.0, 1e-3])}
    st = {}
    cnn.adam_step(p, g, st, lr=0.01, eps=1e-8)
    # t = 1: m^ = g, v^ = g^2, so the step is lr g / (|g| + eps)
    want = np.array([0.5, -2.0, 3.0]) - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8)
    assert np.allclose(p["w"], want, rtol=0, atol=1e-15)
    # minimises a convex quadratic 0.5 ||w - c||^2
    c = np.array([1.0, -1.0, 0.25])
    p = {"w": np.zeros(3)}
    st = {}
    for _ in range(3000):
        cnn.adam_step(p, {"w": p["w"] - c}, st, lr=0.01)
    assert np.allclose(p["w"], c, atol=1e-3)


def test_bf16_forward_close_to_float64_forward():
    rng = np.random.default_rng(4)
    p = _rand_params(4)
    regions = rng.integers(-200, 201, size=(4, 32, 32))
    a = cnn.forward(p, regions, (0, 1, 2), bf=True)["logits"]
    b = cnn.forward(p, regions, (0, 1, 2), bf=False)["logits"]
    assert np.max(np.abs(a - b)) < 0.05 * max(1.0, np.max(np.abs(b)))


def test_training_steps_reduce_the_loss():
    rng = np.random.default_rng(5)
    p = cnn.init_params(5)
    regions = rng.integers(-100, 101, size=(8, 32, 32))
    labels = rng.integers(0, 17, size=(1, 8))
    st = {}
    first = None
    for _ in range(15):
        loss, g, _ = cnn.loss_and_grad(p, regions, labels, (1,), bf=True)
        first = loss if first is None else first
        cnn.adam_step(p, g, st, lr=3e-3)
    assert loss < 0.5 * first
