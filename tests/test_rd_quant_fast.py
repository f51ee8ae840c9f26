"""The RD search's quantiser shortcut (csrc/rd.cu, quant_level_fast) against the
exact definition of the level.

The level of a forward coefficient y of row i, column j of an N-point block at
step q is the paper's round() of B / q (Sec. 3), decided exactly as
|L| = max{k : 4 y^2 d_j >= (2k - 1)^2 N^2 q^2 d_i}, d = diag(T T^T).  The
kernel first forms t = fmaf(float(|y|), est, 1/2) in float32, est =
sqrtf(d_j) * (1 / (float(N q) * sqrtf(d_i))), and takes floor(t) whenever
t -+ t 2^-20 round down to the same integer; only otherwise does it run the
integer test.  numpy's float32 operations round like the GPU's (IEEE, round to
nearest even; the fma is formed exactly in float64, as a 26 x 24-bit product
plus 1/2 is exact there, then rounded once), so this test replays the
shortcut bit for bit and checks it never disagrees with the definition, on
random coefficients and on coefficients placed at and around every rounding
boundary.
"""
import math

import numpy as np
import pytest

from oracle import matrices as mx


def exact_level(a, dj, di, n, q):
    lhs = 4 * a * a * dj
    unit = n * n * q * q * di
    k = math.isqrt(lhs // unit) // 2 + 2 if a else 0
    while k > 0 and (2 * k - 1) ** 2 * unit > lhs:
        k -= 1
    while (2 * k + 1) ** 2 * unit <= lhs:
        k += 1
    return k


def fast_level(a, dj, di, n, q):
    """None where the kernel falls back to the integer test."""
    f = np.float32
    est_i = f(1.0) / (f(n * q) * np.sqrt(f(di)))
    est = np.sqrt(f(dj)) * est_i
    t = f(float(f(a)) * float(est) + 0.5)           # fmaf(float(a), est, 0.5f)
    d = t * f(2.0 ** -20)
    lo, hi = np.floor(t - d), np.floor(t + d)
    return int(lo) if lo == hi else None


@pytest.mark.parametrize("variant", ("hat", "tilde"))
@pytest.mark.parametrize("n", (8, 16, 32))
def test_quantiser_shortcut_matches_the_exact_level(variant, n):
    t = mx.T_N(variant, n).astype(np.int64)
    d = (t * t).sum(axis=1)
    rng = np.random.default_rng(n + (variant == "hat"))
    checked = fallback = typical = typical_fallback = 0
    for q in (1, 2, 3, 8, 16, 32, 64):
        for i in range(n):
            for j in range(n):
                di, dj = int(d[i]), int(d[j])
                small = [int(a) for a in rng.integers(0, 4096, size=40)]
                cands = list(rng.integers(0, 1 << 26, size=40)) + small
                # coefficients at and around the boundaries x + 1/2 = k of the first levels and far up
                for k in list(range(1, 40)) + [1000, 10 ** 5, 10 ** 6]:
                    b = (k - 0.5) * n * q * math.sqrt(di / dj)
                    for a in (math.floor(b) - 1, math.floor(b), math.ceil(b), math.ceil(b) + 1):
                        if 0 <= a < (1 << 26):
                            cands.append(a)
                typical += len(small)
                typical_fallback += sum(fast_level(a, dj, di, n, q) is None for a in small)
                for a in cands:
                    a = int(a)
                    fl = fast_level(a, dj, di, n, q)
                    checked += 1
                    if fl is None:
                        fallback += 1
                        continue
                    assert fl == exact_level(a, dj, di, n, q), (a, dj, di, n, q)
    print(f"{variant} N={n}: {checked} coefficients, {fallback} decided by the integer test "
          f"({typical_fallback} of {typical} random ones with |y| < 4096)")
    # the shortcut must decide nearly all coefficients of everyday size
    assert typical_fallback < typical // 20


@pytest.mark.parametrize("n", (8, 16, 32))
def test_zigzag_key_orders_like_the_position(n):
    """The search tracks the last significant coefficient of a block by a key
    64 (i + j) + (i on odd diagonals, 63 - i on even ones), one add per
    coefficient, and turns the block's largest key back into a position once.
    The key must order like the zig-zag position of oracle.pipeline and
    decode to it."""
    from oracle import pipeline as pl
    pos = {rc: p for p, rc in enumerate(pl.zigzag_order(n))}
    key = {}
    for i in range(n):
        for j in range(n):
            d = i + j
            key[(i, j)] = 64 * d + (i if d % 2 else 63 - i)
    order = sorted(key, key=key.get)
    assert [pos[rc] for rc in order] == list(range(n * n))
    for (i, j), k in key.items():
        d, sub = k >> 6, k & 63
        ii = sub if d % 2 else 63 - sub
        assert (ii, d - ii) == (i, j)
