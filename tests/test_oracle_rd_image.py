"""Pins of the RD oracle's image path (oracle/rd.py: rd_search_image and the
``valid`` mask of block_cost) to definitions that share none of its code:

* tiling: an image whose sides are multiples of 32 gives exactly the region
  search over its 32 x 32 tiles, taken image by image and row-major from the
  top-left corner;
* padding (reading A9: pad by edge replication, measure only the original
  pixels): the padded value at (y, x) is the pixel at (min(y, H-1),
  min(x, W-1)), written out index by index here;
* distortion over original pixels only: with a quantiser step so large that
  every level is zero, each partition cost has a closed form in the energy
  of the region's original pixels; with a moderate step, the all-8x8
  partition of every edge region equals a brute-force pure-Python sum built
  from the printed T_8 and the printed inverse chain (Eqs. 4-7), the paper's
  round() of the float scaled coefficients B = C A C^-1 / q (Sec. 3,
  Sec. 5.1), the JPEG zig-zag fixture and Exp-Golomb codewords built bit by bit.

A plausible mistake anywhere on this path (counting replicated pixels in D,
padding with zeros or from the wrong edge, tiling from another corner,
numbering regions column-major) fails one of these tests.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import rd
from tests import golden_io
from tests.test_oracle_pins import G, _printed_inverse_chain_8

ZZ = golden_io.grid("jpeg_zigzag_8x8.txt")      # scan position of (row, col), JPEG order
F = rd.FRAC_BITS


def residual_image(h, w, seed, amp=255):
    rng = np.random.default_rng(seed)
    return rng.integers(-amp, amp + 1, size=(h, w)).astype(np.int16)


def smooth_residual(h, w, seed):
    """A correlated residual (difference of two smoothed random fields), so that
    quantised blocks keep a handful of levels rather than none or all."""
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(h + 4, w + 4))
    k = np.ones(5) / 5.0
    x = np.apply_along_axis(lambda r: np.convolve(r, k, mode="valid"), 1, x)
    x = np.apply_along_axis(lambda c: np.convolve(c, k, mode="valid"), 0, x)
    return np.clip(np.rint(60.0 * x / x.std()), -255, 255).astype(np.int16)


def tile(img, ty, tx):
    """The 32 x 32 region (ty, tx) of img with edge replication, pixel by pixel,
    and its mask of original pixels."""
    h, w = img.shape
    reg = [[int(img[min(32 * ty + y, h - 1)][min(32 * tx + x, w - 1)]) for x in range(32)] for y in range(32)]
    valid = [[32 * ty + y < h and 32 * tx + x < w for x in range(32)] for y in range(32)]
    return reg, valid


def label_shape(label):
    """(split flags charged, number of blocks) of a quadtree label."""
    if label == 0:
        return 1, 1
    m = label - 1
    return 5, sum(4 if (m >> k) & 1 else 1 for k in range(4))


# ---------------------------------------------------------------------------
# tiling and numbering
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("variant", ("tilde", "hat"))
def test_whole_tiles_equal_region_search(variant):
    imgs = np.stack([residual_image(64, 96, seed=1), residual_image(64, 96, seed=2)])
    qs = (8, 32)
    labels, costs = rd.rd_search_image(imgs, variant, qs)
    regions = np.array([imgs[b, 32 * ty:32 * ty + 32, 32 * tx:32 * tx + 32]
                        for b in range(2) for ty in range(2) for tx in range(3)])
    want_l, want_c = rd.rd_search(regions, variant, qs)
    assert labels.shape == (2, 12)
    assert np.array_equal(labels, want_l)
    assert costs.tolist() == want_c.tolist()


# ---------------------------------------------------------------------------
# distortion over original pixels only: all levels zero
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("h,w", [(45, 70), (33, 31), (7, 100)])
def test_ragged_all_zero_levels_closed_form(h, w):
    """q so large that every |B| / q < 1/2: each block codes only its flag (R = 1),
    Z' = 0, and D = (2^F N^2)^2 sum A^2 over the block's original pixels, so that
    every partition costs lambda' (flags + blocks) + 2^2F 32^4 sum A^2 over the
    region's original pixels."""
    img = residual_image(h, w, seed=h * 1000 + w)
    q = 1 << 14
    lam = rd.lambda_scaled(q, 1, 2)
    labels, costs = rd.rd_search_image(img[None], "hat", (q,))
    nty, ntx = -(-h // 32), -(-w // 32)
    assert costs.shape == (1, nty * ntx, rd.N_PARTITIONS)
    for ty in range(nty):
        for tx in range(ntx):
            reg, valid = tile(img, ty, tx)
            energy = sum(reg[y][x] ** 2 for y in range(32) for x in range(32) if valid[y][x])
            for label in range(rd.N_PARTITIONS):
                flags, nblk = label_shape(label)
                want = lam * (flags + nblk) + 2 ** (2 * F) * 32 ** 4 * energy
                assert costs[0, ty * ntx + tx, label] == want, (ty, tx, label)
            assert labels[0, ty * ntx + tx] == 0


# ---------------------------------------------------------------------------
# distortion over original pixels only: brute force, N = 8 from the printed matrices
# ---------------------------------------------------------------------------

def brute_2d(left, a, right):
    n = len(a)
    return [[sum(left[k][i] * a[i][j] * right[j][l] for i in range(n) for j in range(n))
             for l in range(n)] for k in range(n)]


def eg_bits(level):
    """Signed Exp-Golomb (order 0) length of a nonzero level: codeword of |L| - 1, plus a sign bit."""
    b = bin(abs(level))[2:]                      # binary of (|L| - 1) + 1
    return len("0" * (len(b) - 1) + b) + 1


def block_j8_brute(block, valid, variant, q):
    """(J'_block, D, R) of one 8 x 8 block by brute force from the printed matrices."""
    t = [[int(v) for v in row] for row in G[f"T8_{variant}"][0]]
    u = [[int(x * 8) for x in row] for row in _printed_inverse_chain_8(variant)]      # U_8 = 8 T_8^-1
    d = [sum(v * v for v in row) for row in t]                                         # diag(T T^T)
    s = [1.0 / math.sqrt(di) for di in d]
    # B = C A C^-1 = diag(s) T A U diag(s)^-1 / 8  (Sec. 5.1, C = diag(s) T), in float64
    y = brute_2d(t, block, u)
    lv = [[0] * 8 for _ in range(8)]
    for i in range(8):
        for j in range(8):
            if d[i] == d[j]:                      # B / q = Y / (8 q) is rational: exact round, ties included
                x = Fraction(y[i][j], 8 * q)
                k = math.floor(abs(x) + Fraction(1, 2))
                lv[i][j] = k if x >= 0 else -k
                continue
            x = s[i] * y[i][j] / (8.0 * s[j]) / q   # irrational ratio: the float is far from a tie
            frac = abs(x) - math.floor(abs(x))
            assert abs(frac - 0.5) > 1e-9, "float too close to a tie; pick another seed"
            lv[i][j] = int(math.copysign(math.floor(abs(x) + 0.5), x))      # paper's round()
    c = [[math.floor(2 ** F * math.sqrt(d[i] / d[j]) + 0.5) for j in range(8)] for i in range(8)]
    yd = [[8 * q * lv[i][j] * c[i][j] for j in range(8)] for i in range(8)]
    z = brute_2d(u, yd, t)                                                               # Z' = U Y' T
    dist = sum((2 ** F * 64 * block[i][j] - z[i][j]) ** 2
               for i in range(8) for j in range(8) if valid[i][j])
    scan = [0] * 64
    for i in range(8):
        for j in range(8):
            scan[int(ZZ[i][j])] = lv[i][j]
    last = max((k for k in range(64) if scan[k] != 0), default=-1)
    rate = 1 + (last + 1) + sum(eg_bits(v) for v in scan if v != 0)
    lam = rd.lambda_scaled(q, 1, 2)
    return (32 // 8) ** 4 * dist + lam * rate, dist, rate


@pytest.mark.parametrize("variant", ("tilde", "hat"))
def test_ragged_edge_regions_brute_force_8(variant):
    """The all-8x8 partition (label 16) of every edge region of a ragged image equals
    the brute-force cost of its sixteen 8 x 8 blocks plus five split flags; the
    block_cost of each block with its mask equals the brute-force (J, D, R)."""
    h, w = 45, 70
    img = smooth_residual(h, w, seed=5)
    q = 16
    lam = rd.lambda_scaled(q, 1, 2)
    labels, costs = rd.rd_search_image(img[None], variant, (q,))
    nty, ntx = -(-h // 32), -(-w // 32)
    nonzero_blocks = 0
    for ty in range(nty):
        for tx in range(ntx):
            reg, valid = tile(img, ty, tx)
            if all(all(r) for r in valid):
                continue                                          # interior: covered by the tiling test
            total = 5 * lam
            for by in range(4):
                for bx in range(4):
                    blk = [row[8 * bx:8 * bx + 8] for row in reg[8 * by:8 * by + 8]]
                    vm = [row[8 * bx:8 * bx + 8] for row in valid[8 * by:8 * by + 8]]
                    j, dist, rate = block_j8_brute(blk, vm, variant, q)
                    got = rd.block_cost(np.array(blk, dtype=np.int64), variant, q, 1, 2, valid=np.array(vm))
                    assert got == (j, dist, rate), (ty, tx, by, bx)
                    nonzero_blocks += rate > 1
                    total += j
            assert costs[0, ty * ntx + tx, 16] == total, (ty, tx)
    assert nonzero_blocks > 5          # the levels are not trivially all zero


def test_padding_is_edge_replication():
    """The padded pixels enter the transform as the nearest edge pixel: a region
    whose original part is constant per row codes like the fully constant-row
    region, and differs from zero padding."""
    h, w = 40, 20
    img = np.repeat(np.arange(h, dtype=np.int16)[:, None] * 3 - 60, w, axis=1)     # constant rows
    q = 8
    _, costs = rd.rd_search_image(img[None], "hat", (q,))
    # tile (0, 0): rows 0..31 all valid, columns 20..31 replicated from column 19
    reg, valid = tile(img, 0, 0)
    assert [r[31] for r in reg] == [int(v) for v in img[:32, 19]]
    region = np.repeat(img[:32, :1], 32, axis=1).astype(np.int64)       # every row constant out to column 31
    bc_pad = rd.region_block_costs(region, "hat", q, 1, 2, valid=np.array(valid))
    assert costs[0, 0].tolist() == rd.partition_costs(bc_pad, rd.lambda_scaled(q, 1, 2))
    zero_pad = region.copy()
    zero_pad[:, w:] = 0
    bc_zero = rd.region_block_costs(zero_pad, "hat", q, 1, 2, valid=np.array(valid))
    assert rd.partition_costs(bc_zero, rd.lambda_scaled(q, 1, 2)) != costs[0, 0].tolist()
