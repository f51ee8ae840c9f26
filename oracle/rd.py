"""Exhaustive rate-distortion quadtree search over 32 x 32 regions.

TEST INFRASTRUCTURE ONLY (see the package docstring): nothing in the product
path may import or call it.

The paper evaluates its transforms inside a codec whose block size is
chosen per region (the HEVC experiment of Sec. 6.2, transform sizes 8, 16
and 32).  It prints no rate-distortion search, so this module defines one
from plain parts, each written out with no fast algorithm:

* transform of a block A (paper convention, Sec. 5.1):  Y = T A U with
  U = N T^-1, and the scaled coefficients B = C A C^-1 = diag(s) Y diag(s)^-1 / N
  where C = diag(s) T and s_i = (T T^T)_ii^(-1/2)  (Sec. 3.1 / 6.1);
* quantiser: L = round(B / q) with the paper's round() (sign(x) floor(|x| + 1/2),
  Sec. 3), evaluated exactly:  |L| = max{k >= 0 : k = 0 or
  4 Y_ij^2 d_j >= (2k - 1)^2 N^2 q^2 d_i}, d = diag(T T^T);
* decoder: B' = q L; its integer form Y'_ij = N q L_ij c_ij with the fixed-point
  scale c_ij = round(2^F sqrt(d_i / d_j)), F = 12, so that Y' ~ 2^F N diag(s)^-1 B' diag(s);
  reconstruction Z' = U Y' T  (A' = Z' / (2^F N^2), the paper's C^-1 B' C);
* distortion: the pixel-domain squared error, as the integer
  sum_px (2^F N^2 A - Z')^2 = (2^F N^2)^2 SSE;
* rate: a coded-block flag (1 bit) per block; one significance bit for each
  zig-zag position (the generalised order of Sec. 5.1) up to and including
  the last nonzero level; per nonzero level 2 floor(log2 |L|) + 2 bits (a
  signed Exp-Golomb code of order 0); and one split flag per quadtree node
  that may split (the 32 x 32 node and each 16 x 16 node);
* cost J = SSE + lambda R with lambda = kappa q^2, all on the common integer
  scale 2^(2F) 32^4:
      J'_block = (32 / N)^4 sum (2^F N^2 A - Z')^2 + lambda' R_block,
      lambda' = kappa q^2 2^(2F + 20),  kappa = kappa_num / 2^kappa_log2_den;
* partitions: the 17 quadtrees  32 | four quadrants each 16 or four 8s.
  Label 0 is the unsplit region; label 1 + m splits it, with bit k of m set
  when quadrant k (raster order: top-left, top-right, bottom-left,
  bottom-right) is split into 8 x 8 blocks.  The chosen label minimises J';
  ties go to the larger transform (at each node the unsplit choice wins).

Every quantity is an exact integer (Python ints), so labels and costs are
defined without rounding ambiguity.  Pins: ``tests/test_oracle_rd.py``.
"""
from __future__ import annotations

import functools
import math

import numpy as np

from . import matrices as mx
from . import pipeline as pl

FRAC_BITS = 12           # F: fractional bits of the dequantisation scale
REGION = 32
SIZES = (32, 16, 8)
N_PARTITIONS = 17


@functools.lru_cache(maxsize=None)
def _t_u(variant: str, n: int):
    return mx.T_N(variant, n).astype(np.int64), mx.U_N(variant, n).astype(np.int64)


@functools.lru_cache(maxsize=None)
def row_norms2(variant: str, n: int) -> list[int]:
    """d_i = (T_N T_N^T)_ii (so s_i = d_i^(-1/2), Sec. 3.1)."""
    t = _t_u(variant, n)[0]
    return [int(v) for v in np.diag(t @ t.T)]


@functools.lru_cache(maxsize=None)
def dequant_scale(variant: str, n: int, frac_bits: int = FRAC_BITS) -> list[list[int]]:
    """c_ij = round(2^F sqrt(d_i / d_j)): the largest c with (2c - 1)^2 d_j <= 4^(F+1) d_i."""
    d = row_norms2(variant, n)
    lim = 4 ** (frac_bits + 1)
    out = []
    for i in range(n):
        row = []
        for j in range(n):
            c = int(math.floor(2 ** frac_bits * math.sqrt(d[i] / d[j]) + 0.5))
            while (2 * (c + 1) - 1) ** 2 * d[j] <= lim * d[i]:
                c += 1
            while c > 0 and (2 * c - 1) ** 2 * d[j] > lim * d[i]:
                c -= 1
            row.append(c)
        out.append(row)
    return out


def quant_level(y: int, di: int, dj: int, n: int, q: int) -> int:
    """round(B_ij / q) for B_ij = y s_i / (n s_j), exactly (paper's round, Sec. 3)."""
    a = abs(int(y))
    lhs = 4 * a * a * dj
    unit = n * n * q * q * di
    k = int(math.floor(a * math.sqrt(dj / di) / (n * q) + 0.5))   # estimate, then exact correction
    while (2 * (k + 1) - 1) ** 2 * unit <= lhs:
        k += 1
    while k > 0 and (2 * k - 1) ** 2 * unit > lhs:
        k -= 1
    return k if y >= 0 else -k


def level_bits(level: int) -> int:
    """Bits of one level: 0 for a zero, else 2 floor(log2 |L|) + 2 (signed Exp-Golomb, order 0)."""
    a = abs(int(level))
    return 0 if a == 0 else 2 * (a.bit_length() - 1) + 2


@functools.lru_cache(maxsize=None)
def _scan(n: int):
    return tuple(pl.zigzag_order(n))


def block_rate(levels, n: int) -> int:
    """Bits of one block: coded-block flag, significance bits up to the last nonzero level in
    zig-zag order, and the bits of every nonzero level."""
    scan = [levels[i][j] for i, j in _scan(n)]
    last = max((k for k, v in enumerate(scan) if v != 0), default=-1)
    return 1 + (last + 1) + sum(level_bits(v) for v in scan)


def lambda_scaled(q: int, kappa_num: int, kappa_log2_den: int, frac_bits: int = FRAC_BITS) -> int:
    """lambda' = kappa q^2 2^(2F + 20) (an integer for kappa_log2_den <= 2F + 20)."""
    e = 2 * frac_bits + 20 - kappa_log2_den
    if e < 0:
        raise ValueError("kappa denominator too large for the integer cost scale")
    return kappa_num * q * q * (1 << e)


def block_cost(a: np.ndarray, variant: str, q: int, kappa_num: int, kappa_log2_den: int,
               frac_bits: int = FRAC_BITS, valid=None):
    """(J'_block, D, R) of one N x N block a (N = a.shape[0]) on the common scale.

    D = sum (2^F N^2 A - Z')^2 over the pixels where ``valid`` (default: all)
    is true, unscaled; R = block_rate of the levels.
    """
    n = a.shape[0]
    t, u = _t_u(variant, n)
    d = row_norms2(variant, n)
    c = dequant_scale(variant, n, frac_bits)
    y = t @ a.astype(np.int64) @ u                       # Y = T A U (exact)
    lv = [[quant_level(int(y[i, j]), d[i], d[j], n, q) for j in range(n)] for i in range(n)]
    yd = [[n * q * lv[i][j] * c[i][j] for j in range(n)] for i in range(n)]
    if max(abs(v) for row in yd for v in row) >= 1 << 44:       # keeps U Y' T inside int64
        raise OverflowError("dequantised coefficient out of range")
    yd = np.array(yd, dtype=np.int64)
    z = u @ yd @ t                                       # Z' = U Y' T (exact in int64)
    e = (a.astype(np.int64) << frac_bits) * (n * n) - z
    if valid is not None:
        e = np.where(valid, e, 0)
    dist = sum(int(v) * int(v) for v in e.ravel())
    rate = block_rate(lv, n)
    scale = (REGION // n) ** 4
    return scale * dist + lambda_scaled(q, kappa_num, kappa_log2_den, frac_bits) * rate, dist, rate


def region_block_costs(region: np.ndarray, variant: str, q: int, kappa_num: int, kappa_log2_den: int,
                       valid=None):
    """J' of the 21 blocks of a 32 x 32 region: {32: [J], 16: [4, raster], 8: [16, raster]}."""
    out = {}
    for n in SIZES:
        k = REGION // n
        out[n] = [block_cost(region[by * n:(by + 1) * n, bx * n:(bx + 1) * n], variant, q,
                             kappa_num, kappa_log2_den,
                             valid=None if valid is None else valid[by * n:(by + 1) * n, bx * n:(bx + 1) * n])[0]
                  for by in range(k) for bx in range(k)]
    return out


def quadrant_8_blocks(k: int) -> list[int]:
    """Raster indices (in the 4 x 4 grid of 8 x 8 blocks) of the four 8 x 8 blocks of quadrant k."""
    qy, qx = k >> 1, k & 1
    return [(2 * qy + dy) * 4 + (2 * qx + dx) for dy in range(2) for dx in range(2)]


def partition_costs(bc, lam: int) -> list[int]:
    """J' of the 17 partitions from the block costs (flags: one per node that may split)."""
    out = [lam + bc[32][0]]
    for m in range(16):
        j = lam
        for k in range(4):
            if (m >> k) & 1:
                j += lam + sum(bc[8][b] for b in quadrant_8_blocks(k))
            else:
                j += lam + bc[16][k]
        out.append(j)
    return out


def dp_label(bc, lam: int) -> int:
    """Bottom-up choice: each quadrant keeps its 16 x 16 block unless four 8 x 8 blocks cost
    less; the region stays whole unless the best split costs less."""
    m, split_cost = 0, lam
    for k in range(4):
        j16 = lam + bc[16][k]
        j8 = lam + sum(bc[8][b] for b in quadrant_8_blocks(k))
        if j8 < j16:
            m |= 1 << k
            split_cost += j8
        else:
            split_cost += j16
    return 0 if lam + bc[32][0] <= split_cost else 1 + m


def rd_search(regions: np.ndarray, variant: str, qs, kappa_num: int = 1, kappa_log2_den: int = 2):
    """Labels [len(qs), n] (uint8) and partition costs [len(qs), n, 17] (Python ints)."""
    regions = np.asarray(regions)
    labels = np.zeros((len(qs), len(regions)), dtype=np.uint8)
    costs = np.empty((len(qs), len(regions), N_PARTITIONS), dtype=object)
    for qi, q in enumerate(qs):
        lam = lambda_scaled(q, kappa_num, kappa_log2_den)
        for r, reg in enumerate(regions):
            bc = region_block_costs(reg, variant, q, kappa_num, kappa_log2_den)
            labels[qi, r] = dp_label(bc, lam)
            costs[qi, r, :] = partition_costs(bc, lam)
    return labels, costs


def rd_search_image(imgs: np.ndarray, variant: str, qs, kappa_num: int = 1, kappa_log2_den: int = 2):
    """rd_search over the 32 x 32 regions of images [B, H, W], tiled from the top-left corner:
    pixels beyond H x W are edge-replicated and left out of the distortion.  Regions are
    numbered image by image, row-major.  Returns labels [len(qs), R] and costs [len(qs), R, 17]."""
    imgs = np.asarray(imgs)
    _, h, w = imgs.shape
    padded = pl.pad_replicate(imgs, REGION)
    valid = np.zeros(padded.shape[1:], dtype=bool)
    valid[:h, :w] = True
    regions, masks = [], []
    for img in padded:
        for ty in range(padded.shape[1] // REGION):
            for tx in range(padded.shape[2] // REGION):
                sl = (slice(ty * REGION, (ty + 1) * REGION), slice(tx * REGION, (tx + 1) * REGION))
                regions.append(img[sl])
                masks.append(valid[sl])
    labels = np.zeros((len(qs), len(regions)), dtype=np.uint8)
    costs = np.empty((len(qs), len(regions), N_PARTITIONS), dtype=object)
    for qi, q in enumerate(qs):
        lam = lambda_scaled(q, kappa_num, kappa_log2_den)
        for r, (reg, m) in enumerate(zip(regions, masks)):
            bc = region_block_costs(reg, variant, q, kappa_num, kappa_log2_den, valid=None if m.all() else m)
            labels[qi, r] = dp_label(bc, lam)
            costs[qi, r, :] = partition_costs(bc, lam)
    return labels, costs


def partition_blocks(label: int):
    """The (y, x, size) blocks a label's partition consists of."""
    if label == 0:
        return [(0, 0, 32)]
    m = label - 1
    out = []
    for k in range(4):
        qy, qx = 16 * (k >> 1), 16 * (k & 1)
        if (m >> k) & 1:
            out += [(qy + dy, qx + dx, 8) for dy in (0, 8) for dx in (0, 8)]
        else:
            out.append((qy, qx, 16))
    return out
