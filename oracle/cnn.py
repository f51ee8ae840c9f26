"""Learned transform-size selector: a small CNN over 32 x 32 residual regions.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): nothing in the product
path may import or call it.

The paper measures its transforms inside a codec whose encoder chooses the
transform size per region (Sec. 6.2, sizes 8, 16 and 32).  The library's
exhaustive search (``oracle/rd.py``) makes that choice by trying all 17
quadtrees; this network proposes it instead.  It is not in the paper; every
definition below is this library's, written out plainly in float64:

Network (activations NHWC, one region at a time; x is the int16 residual):
  a0 = x / 64
  for l = 1, 2, 3 (channels 1 -> 16 -> 32 -> 32):
      z_l[y, x, o] = b_l[o] + sum_{dy, dx in 0..2} sum_i W_l[o, dy, dx, i] a_{l-1}[y + dy - 1, x + dx - 1, i]
                     (zero outside the map: a 3 x 3 cross-correlation with zero padding)
      a_l = maxpool_2x2(relu(z_l))                   (32 -> 16 -> 8 -> 4 pixels a side)
  h = a_3 flattened in (y, x, channel) order          (512 features)
  u = Wf1 h                                          (64)
  for each quantiser slot k (one-hot input):  g_k = relu(u + bf1 + Wq[:, k])
      logits_k = Wf2 g_k + bf2                       (17, one per quadtree label of ``rd``)
Loss per (region, slot): cross-entropy of softmax(logits_k) with the search's
label, plus mu * sum_j p_j c_j, the expected normalised RD regret, where
c_j = (J_j - J_min) / J_min from the search's 17 partition costs.  The batch
loss is the mean over all (region, slot) samples.

Mixed precision (what the GPU kernels compute): weights are bfloat16 copies of
float32 master weights (biases stay float32); each stored activation (a_l, g_k)
and each gradient that feeds a matrix product (du, dh, da_2, da_1 and the
pre-pool gradients) is rounded to bfloat16, round to nearest even.  Those
rounding points are reproduced here when ``bf16=True``; the arithmetic between
them is float64.  Gradients treat each rounding as the identity (the usual
straight-through reading).  Max pooling routes the gradient to the first
maximum of its window in raster order.

Optimiser: Adam (Kingma and Ba, 2015) with bias correction, on the float32
master weights.

Pins: ``tests/test_oracle_cnn.py`` (convolution against scipy's correlate2d,
central finite differences of the loss for every parameter tensor, the
softmax/CE closed form, pooling and Adam closed forms, bfloat16 rounding
against torch's conversion).
"""
from __future__ import annotations

import numpy as np

IN_SCALE = 1.0 / 64.0
CHANNELS = (1, 16, 32, 32)
HIDDEN = 64
N_LABELS = 17
Q_SLOTS = 4
FEATURES = 4 * 4 * 32

# parameter tensors in the order of the library's flat float32 vector
PARAM_SHAPES = (
    ("conv1_w", (16, 3, 3, 1)), ("conv1_b", (16,)),
    ("conv2_w", (32, 3, 3, 16)), ("conv2_b", (32,)),
    ("conv3_w", (32, 3, 3, 32)), ("conv3_b", (32,)),
    ("fc1_w", (HIDDEN, FEATURES)), ("fc1_q", (HIDDEN, Q_SLOTS)), ("fc1_b", (HIDDEN,)),
    ("fc2_w", (N_LABELS, HIDDEN)), ("fc2_b", (N_LABELS,)),
)
WEIGHTS = ("conv1_w", "conv2_w", "conv3_w", "fc1_w", "fc1_q", "fc2_w")   # stored as bfloat16


def param_count() -> int:
    return int(sum(np.prod(s) for _, s in PARAM_SHAPES))


def bf16(x):
    """Nearest bfloat16 (8 significant bits, ties to even) of float64 values, as float64.

    Normal range only (the network's values are far from bfloat16's under- and
    overflow thresholds)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                  # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.round(m * 256.0), e - 8)


def init_params(seed: int = 0) -> dict:
    """He-normal weights, zero biases (float32 values held in float64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = {}
    for name, shape in PARAM_SHAPES:
        if name.endswith("_b"):
            p[name] = np.zeros(shape)
        else:
            fan_in = int(np.prod(shape[1:]))
            if name == "fc1_q":
                fan_in = FEATURES
            p[name] = rng.standard_normal(shape) * np.sqrt(2.0 / fan_in)
        p[name] = p[name].astype(np.float32).astype(np.float64)
    return p


def _weights(params, bf):
    return {k: (bf16(v) if (bf and k in WEIGHTS) else np.asarray(v, dtype=np.float64)) for k, v in params.items()}


def conv3x3(a: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """z[n, y, x, o] = b[o] + sum_{dy,dx,i} w[o, dy, dx, i] a[n, y+dy-1, x+dx-1, i], zero padded."""
    n, h, wd, _ = a.shape
    ap = np.zeros((n, h + 2, wd + 2, a.shape[3]))
    ap[:, 1:h + 1, 1:wd + 1, :] = a
    z = np.zeros((n, h, wd, w.shape[0])) + b
    for dy in range(3):
        for dx in range(3):
            z += np.einsum("nyxi,oi->nyxo", ap[:, dy:dy + h, dx:dx + wd, :], w[:, dy, dx, :])
    return z


def conv3x3_backward(a: np.ndarray, w: np.ndarray, dz: np.ndarray):
    """(da, dw, db) of conv3x3 for the upstream gradient dz."""
    n, h, wd, _ = a.shape
    ap = np.zeros((n, h + 2, wd + 2, a.shape[3]))
    ap[:, 1:h + 1, 1:wd + 1, :] = a
    dw = np.zeros(w.shape)
    dap = np.zeros(ap.shape)
    for dy in range(3):
        for dx in range(3):
            dw[:, dy, dx, :] = np.einsum("nyxo,nyxi->oi", dz, ap[:, dy:dy + h, dx:dx + wd, :])
            dap[:, dy:dy + h, dx:dx + wd, :] += np.einsum("nyxo,oi->nyxi", dz, w[:, dy, dx, :])
    return dap[:, 1:h + 1, 1:wd + 1, :], dw, dz.sum(axis=(0, 1, 2))


def maxpool2(r: np.ndarray):
    """(pooled, argmax) over 2 x 2 windows; argmax in 0..3 = 2 dy + dx, first maximum wins."""
    n, h, w, c = r.shape
    win = r.reshape(n, h // 2, 2, w // 2, 2, c).transpose(0, 1, 3, 5, 2, 4).reshape(n, h // 2, w // 2, c, 4)
    return win.max(axis=-1), win.argmax(axis=-1)


def maxpool2_backward(dp: np.ndarray, arg: np.ndarray) -> np.ndarray:
    n, h2, w2, c = dp.shape
    win = np.zeros((n, h2, w2, c, 4))
    np.put_along_axis(win, arg[..., None], dp[..., None], axis=-1)
    return win.reshape(n, h2, w2, c, 2, 2).transpose(0, 1, 4, 2, 5, 3).reshape(n, 2 * h2, 2 * w2, c)


def forward(params: dict, regions: np.ndarray, slots, bf: bool = True) -> dict:
    """Forward pass of a batch.  regions [n, 32, 32] integers; slots: the one-hot
    quantiser slots evaluated for every region.  Returns the activations and
    logits [len(slots), n, 17]."""
    rnd = bf16 if bf else (lambda v: v)
    w = _weights(params, bf)
    a = rnd(np.asarray(regions, dtype=np.float64)[..., None] * IN_SCALE)
    cache = {"a0": a}
    for l in (1, 2, 3):
        z = conv3x3(a, w[f"conv{l}_w"], w[f"conv{l}_b"])
        r = rnd(np.maximum(z, 0.0))
        a, arg = maxpool2(r)
        cache[f"r{l}"], cache[f"arg{l}"], cache[f"a{l}"] = r, arg, a
    h = a.reshape(a.shape[0], FEATURES)
    u = h @ w["fc1_w"].T
    g = np.stack([rnd(np.maximum(u + w["fc1_b"] + w["fc1_q"][:, k], 0.0)) for k in slots])
    logits = g @ w["fc2_w"].T + w["fc2_b"]
    cache.update(h=h, u=u, g=g, logits=logits, slots=tuple(slots), w=w)
    return cache


def softmax(logits: np.ndarray) -> np.ndarray:
    e = np.exp(logits - logits.max(axis=-1, keepdims=True))
    return e / e.sum(axis=-1, keepdims=True)


def normalised_regret(costs) -> np.ndarray:
    """c_j = (J_j - J_min) / J_min per (slot, region) from exact partition costs [..., 17]."""
    c = np.asarray(costs, dtype=object)
    out = np.zeros(c.shape, dtype=np.float64)
    for idx in np.ndindex(c.shape[:-1]):
        row = [int(v) for v in c[idx]]
        jmin = min(row)
        out[idx] = [(v - jmin) / jmin if jmin > 0 else 0.0 for v in row]
    return out


def loss_and_grad(params: dict, regions, labels, slots, regret=None, mu: float = 0.0, bf: bool = True):
    """Mean loss over the (slot, region) samples and its gradient (dict like params).

    labels [len(slots), n]; regret [len(slots), n, 17] (normalised, or None)."""
    rnd = bf16 if bf else (lambda v: v)
    c = forward(params, regions, slots, bf)
    w = c["w"]
    labels = np.asarray(labels)
    ns, n = labels.shape
    m = ns * n
    p = softmax(c["logits"])
    onehot = np.zeros_like(p)
    np.put_along_axis(onehot, labels[..., None].astype(np.int64), 1.0, axis=-1)
    ce = -np.log(np.take_along_axis(p, labels[..., None].astype(np.int64), axis=-1)[..., 0])
    dl = p - onehot
    loss = ce.sum()
    if regret is not None and mu != 0.0:
        rg = np.asarray(regret, dtype=np.float64)
        er = (p * rg).sum(axis=-1)
        loss += mu * er.sum()
        dl = dl + mu * p * (rg - er[..., None])
    loss /= m
    dl /= m
    grad = {}
    grad["fc2_w"] = np.einsum("sno,snh->oh", dl, c["g"])
    grad["fc2_b"] = dl.sum(axis=(0, 1))
    dg = (dl @ w["fc2_w"]) * (c["g"] > 0)                       # [s, n, 64]
    grad["fc1_b"] = dg.sum(axis=(0, 1))
    grad["fc1_q"] = np.zeros((HIDDEN, Q_SLOTS))
    for si, k in enumerate(c["slots"]):
        grad["fc1_q"][:, k] += dg[si].sum(axis=0)
    du = rnd(dg.sum(axis=0))                                     # [n, 64]
    grad["fc1_w"] = du.T @ c["h"]
    dh = rnd(du @ w["fc1_w"])                                    # [n, 512]
    da = dh.reshape(c["a3"].shape)
    for l in (3, 2, 1):
        dr = maxpool2_backward(da, c[f"arg{l}"]) * (c[f"r{l}"] > 0)
        dz = rnd(dr)
        da_prev, grad[f"conv{l}_w"], grad[f"conv{l}_b"] = conv3x3_backward(c[f"a{l - 1}"], w[f"conv{l}_w"], dz)
        da = rnd(da_prev)
    return loss, grad, c


def adam_step(params: dict, grad: dict, state: dict, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8) -> None:
    """One Adam update in place: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
    theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for k in params:
        m = state.setdefault("m", {}).get(k, np.zeros_like(params[k]))
        v = state.setdefault("v", {}).get(k, np.zeros_like(params[k]))
        m = beta1 * m + (1 - beta1) * grad[k]
        v = beta2 * v + (1 - beta2) * grad[k] * grad[k]
        state["m"][k], state["v"][k] = m, v
        params[k] = params[k] - lr * (m / (1 - beta1 ** t)) / (np.sqrt(v / (1 - beta2 ** t)) + eps)


def predict(params: dict, regions, slots, bf: bool = True) -> np.ndarray:
    """Labels [len(slots), n]: the argmax of the logits (first maximum)."""
    return forward(params, regions, slots, bf)["logits"].argmax(axis=-1).astype(np.uint8)
