"""Pins of the rate-distortion quadtree oracle (oracle/rd.py) to definitions
independent of its own arithmetic: the quantiser against the paper's round()
applied to B = C A C^-1 computed with float matrices (Sec. 3, Sec. 3.1), the
fixed-point decoder against the float inverse C^-1 B' C, Exp-Golomb code
lengths against codewords built bit by bit, closed forms for all-zero levels,
and the bottom-up partition choice against brute force over all 17 quadtrees.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import matrices as mx
from oracle import rd
from paper_2207_11638_gb300 import synth


def c_hat(variant, n):
    t = mx.T_N(variant, n).astype(np.float64)
    s = 1.0 / np.sqrt(np.diag(t @ t.T))
    return s[:, None] * t


def paper_round(x):
    """round(x) = sign(x) floor(|x| + 1/2) (Sec. 3), elementwise."""
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def blocks(n, count, seed, lo=-255, hi=255):
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(count, n, n)).astype(np.int64)


@pytest.mark.parametrize("variant", mx.VARIANTS)
@pytest.mark.parametrize("n", rd.SIZES)
def test_quantiser_is_paper_round_of_scaled_coefficients(variant, n):
    c = c_hat(variant, n)
    ci = np.linalg.inv(c)
    t, u = (mx.T_N(variant, n).astype(np.int64), mx.U_N(variant, n).astype(np.int64))
    d = rd.row_norms2(variant, n)
    checked = 0
    for q in (3, 8, 16, 32):
        for a in blocks(n, 3, seed=n * 100 + q):
            b = c @ a.astype(np.float64) @ ci               # B = C A C^-1, float
            want = paper_round(b / q)
            y = t @ a @ u
            got = np.array([[rd.quant_level(int(y[i, j]), d[i], d[j], n, q) for j in range(n)]
                            for i in range(n)])
            frac = np.abs(b / q) - np.floor(np.abs(b / q))
            clear = np.abs(frac - 0.5) > 1e-9                # away from ties the float answer is sure
            assert np.array_equal(got[clear], want[clear])
            checked += int(clear.sum())
            # where d_i = d_j, B / q = Y / (N q) is rational: exact round, ties included
            for i, j in itertools.product(range(n), range(n)):
                if d[i] == d[j]:
                    x = Fraction(int(y[i, j]), n * q)
                    k = math.floor(abs(x) + Fraction(1, 2))
                    assert got[i, j] == (k if x >= 0 else -k)
                    checked += 0 if clear[i, j] else 1
    assert checked == 4 * 3 * n * n


@pytest.mark.parametrize("n", rd.SIZES)
def test_quantiser_ties_round_away_from_zero(n):
    d = rd.row_norms2("hat", n)
    for q in (2, 8, 32):
        for k in (1, 2, 7):
            y = (2 * k - 1) * n * q // 2                   # |B / q| = k - 1/2 exactly on the diagonal
            assert rd.quant_level(y, d[0], d[0], n, q) == k
            assert rd.quant_level(-y, d[0], d[0], n, q) == -k
            assert rd.quant_level(y - 1, d[0], d[0], n, q) == k - 1


def eg0_codeword(v):
    """Exp-Golomb order-0 codeword of v >= 0: (len(bin(v+1)) - 1) zeros, then bin(v+1)."""
    b = bin(v + 1)[2:]
    return "0" * (len(b) - 1) + b


def test_level_bits_are_exp_golomb_plus_sign():
    assert rd.level_bits(0) == 0
    for lv in list(range(1, 300)) + [1023, 1024, 65535, 65536]:
        want = len(eg0_codeword(lv - 1)) + 1
        assert rd.level_bits(lv) == want and rd.level_bits(-lv) == want


def test_block_rate_counts_significance_to_last_nonzero():
    n = 8
    lv = [[0] * n for _ in range(n)]
    assert rd.block_rate(lv, n) == 1                          # coded-block flag only
    lv[0][0] = 1
    assert rd.block_rate(lv, n) == 1 + 1 + 2
    lv[2][0] = -3                                             # zig-zag position 3 (JPEG order)
    assert rd.block_rate(lv, n) == 1 + 4 + 2 + 4


@pytest.mark.parametrize("variant", mx.VARIANTS)
@pytest.mark.parametrize("n", rd.SIZES)
def test_dequant_scale_is_rounded_ratio(variant, n):
    d = rd.row_norms2(variant, n)
    c = rd.dequant_scale(variant, n)
    for i, j in itertools.product(range(n), range(n)):
        x = 2 ** rd.FRAC_BITS * np.sqrt(d[i] / d[j])
        assert abs(c[i][j] - np.floor(x + 0.5)) == 0
        assert abs(c[i][j] - x) <= 0.5
    assert all(c[i][i] == 2 ** rd.FRAC_BITS for i in range(n))


@pytest.mark.parametrize("variant", mx.VARIANTS)
@pytest.mark.parametrize("n", rd.SIZES)
def test_decoder_converges_to_float_inverse(variant, n):
    """With many fractional bits the integer decoder reproduces A' = C^-1 (q L) C."""
    c = c_hat(variant, n)
    ci = np.linalg.inv(c)
    t, u = (mx.T_N(variant, n).astype(np.int64), mx.U_N(variant, n).astype(np.int64))
    d = rd.row_norms2(variant, n)
    fb = 20
    cs = rd.dequant_scale(variant, n, fb)
    q = 16
    for a in blocks(n, 2, seed=7 + n, lo=-40, hi=40):
        y = t @ a @ u
        lv = np.array([[rd.quant_level(int(y[i, j]), d[i], d[j], n, q) for j in range(n)] for i in range(n)])
        want = ci @ (q * lv.astype(np.float64)) @ c                # A' = C^-1 B' C
        yd = np.array([[n * q * lv[i, j] * cs[i][j] for j in range(n)] for i in range(n)], dtype=np.int64)
        got = (u @ yd @ t) / float(2 ** fb * n * n)
        assert np.max(np.abs(got - want)) < 1e-3
        # the default F = 12 decoder stays within its rounding bound (relative 2^-12 per coefficient)
        _, dist, _ = rd.block_cost(a, variant, q, 1, 2)
        sse_float = float(np.sum((a - want) ** 2))
        sse_fixed = dist / float(2 ** rd.FRAC_BITS * n * n) ** 2
        assert abs(sse_fixed - sse_float) <= 0.02 * sse_float + 1.0


@pytest.mark.parametrize("variant", mx.VARIANTS)
def test_all_zero_levels_closed_form(variant):
    region = synth.residual_regions_32(1, seed=9)[0].astype(np.int64)
    q = 1 << 14                                                  # every |B| / q < 1/2
    lam = rd.lambda_scaled(q, 1, 2)
    bc = rd.region_block_costs(region, variant, q, 1, 2)
    energy = int(np.sum(region ** 2))
    scale = 2 ** (2 * rd.FRAC_BITS) * 32 ** 4
    assert bc[32][0] == scale * energy + lam
    for k in range(4):
        qy, qx = 16 * (k >> 1), 16 * (k & 1)
        assert bc[16][k] == scale * int(np.sum(region[qy:qy + 16, qx:qx + 16] ** 2)) + lam
    costs = rd.partition_costs(bc, lam)
    assert costs[0] == 2 * lam + scale * energy
    assert costs[16] == lam + 4 * lam + 16 * lam + scale * energy
    assert rd.dp_label(bc, lam) == 0


def test_zero_region_is_unsplit():
    z = np.zeros((1, 32, 32), dtype=np.int16)
    labels, costs = rd.rd_search(z, "hat", (8,))
    lam = rd.lambda_scaled(8, 1, 2)
    assert labels[0, 0] == 0 and costs[0, 0, 0] == 2 * lam


def test_partitions_tile_the_region():
    for label in range(rd.N_PARTITIONS):
        cover = np.zeros((32, 32), dtype=int)
        for y, x, s in rd.partition_blocks(label):
            cover[y:y + s, x:x + s] += 1
        assert np.all(cover == 1)
    assert len({tuple(rd.partition_blocks(l)) for l in range(rd.N_PARTITIONS)}) == rd.N_PARTITIONS


@pytest.mark.parametrize("variant", mx.VARIANTS)
def test_bottom_up_choice_equals_brute_force(variant):
    regions = synth.residual_regions_32(6, seed=11)
    for q in (8, 16, 32):
        lam = rd.lambda_scaled(q, 1, 2)
        for reg in regions:
            bc = rd.region_block_costs(reg, variant, q, 1, 2)
            # brute force: every quadtree's cost from its own blocks, flags counted per node
            brute = []
            for label in range(rd.N_PARTITIONS):
                j = lam * (1 if label == 0 else 5)
                for y, x, s in rd.partition_blocks(label):
                    j += rd.block_cost(reg[y:y + s, x:x + s], variant, q, 1, 2)[0]
                brute.append(j)
            assert brute == rd.partition_costs(bc, lam)
            label = rd.dp_label(bc, lam)
            assert brute[label] == min(brute)
            ties = [l for l in range(rd.N_PARTITIONS) if brute[l] == min(brute)]
            assert label == ties[0] or len(ties) == 1
