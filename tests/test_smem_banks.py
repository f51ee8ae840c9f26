"""Shared-memory bank model of the pipelined fused kernel.

A CPU model of the addresses the kernel computes (lane -> block / row / sub-
block maps, padded exchange-buffer layouts, staged-row pitches).  It counts
the wavefronts one warp-wide 128-bit access needs (one per quarter warp at
best), checks the exchanges never need more, and that every layout is
injective and fits its buffer.
"""
import itertools

import pytest


def wavefronts(addrs, width=16):
    phases = {4: [range(32)], 8: [range(16), range(16, 32)],
              16: [range(8 * i, 8 * i + 8) for i in range(4)]}[width]
    total = 0
    for ph in phases:
        banks = {}
        for lane in ph:
            for w in range(width // 4):
                word = addrs[lane] // 4 + w
                banks.setdefault(word % 32, set()).add(word)
        total += max(len(s) for s in banks.values())
    return total


# ---- N = 16: lanes (lbw = lane & 7 block, p = lane >> 3); blocks 65 chunks apart
def addr16(lane, s, row, ch):
    return 16 * ((lane & 7) * 65 + (s * 8 + row) * 2 + ch)


# ---- N = 32: lanes (lbw = lane >> 4 block, p = lane & 15); blocks 288 chunks apart
def l1(hr, row, c, ch):
    return (hr * 16 + row) * 9 + 2 * c + ch


def l2(q, row, ch):
    return q * 17 + 2 * row + (row >> 2) + ch


def addr32(lane, chunk):
    return 16 * ((lane >> 4) * 288 + chunk)


def test_layouts_are_injective_and_fit():
    a16 = [(s * 8 + r) * 2 + c for s in range(4) for r in range(8) for c in range(2)]
    assert len(set(a16)) == 64 and max(a16) < 65
    a1 = [l1(h, r, c, ch) for h in range(2) for r in range(16) for c in range(4) for ch in range(2)]
    a2 = [l2(q, r, ch) for q in range(16) for r in range(8) for ch in range(2)]
    assert len(set(a1)) == 256 and max(a1) < 288
    assert len(set(a2)) == 256 and max(a2) < 288


def test_n16_exchanges_conflict_free():
    for b, ch in itertools.product(range(2), range(2)):
        # fold writes: lane writes sub-block (a, b) rows p and 7-p
        for a in range(2):
            for row_of in (lambda p: p, lambda p: 7 - p):
                ad = [addr16(l, a * 2 + b, row_of(l >> 3), ch) for l in range(32)]
                assert wavefronts(ad) == 4
    # core reads / writes: lane (lbw, s = p) touches sub-block s rows 0..7
    for i, ch in itertools.product(range(8), range(2)):
        ad = [addr16(l, l >> 3, i, ch) for l in range(32)]
        assert wavefronts(ad) == 4


def test_n32_exchanges_conflict_free():
    for c, ch in itertools.product(range(4), range(2)):
        # first-fold writes: half 0 row p, half 1 row 15 - p
        assert wavefronts([addr32(l, l1(0, l & 15, c, ch)) for l in range(32)]) == 4
        assert wavefronts([addr32(l, l1(1, 15 - (l & 15), c, ch)) for l in range(32)]) == 4
    for i, ch in itertools.product(range(8), range(2)):
        # second-fold reads: q = lane & 15; rows ra, rb of half hr, class c
        for which in range(2):
            ad = []
            for l in range(32):
                q = l & 15
                hr, ar, c = q >> 3, (q >> 2) & 1, q & 3
                ra, rb = (7 - i, 8 + i) if ar else (i, 15 - i)
                ad.append(addr32(l, l1(hr, ra if which == 0 else rb, c, ch)))
            assert wavefronts(ad) == 4
        # core output writes
        assert wavefronts([addr32(l, l2(l & 15, i, ch)) for l in range(32)]) == 4
    # unfold reads: lane p reads top row rt of q_t and bottom row rb of q_b
    for hr, c, ch, which in itertools.product(range(2), range(4), range(2), range(2)):
        ad = []
        for l in range(32):
            p = l & 15
            m = p if hr == 0 else 15 - p
            rt, rb = (m, 7 - m) if m < 8 else (15 - m, m - 8)
            q = hr * 8 + (0 if which == 0 else 4) + c
            ad.append(addr32(l, l2(q, rt if which == 0 else rb, ch)))
        assert wavefronts(ad) == 4


@pytest.mark.parametrize("esize", (1, 2))
def test_staged_row_reads(esize):
    """128-bit reads of the staged rows: N = 8 and N = 32 conflict free, N = 16 i16 two-way."""
    # N = 8: lane = block, row r, 8 pixels per block
    if esize == 2:
        assert wavefronts([l * 16 for l in range(32)]) == 4
    # N = 32: lane p (< 16) reads row p of block lane >> 4; pitch = row bytes + 16
    rowb = 256 * esize
    ad = [(l & 15) * (rowb + 16) + (l >> 4) * 32 * esize for l in range(32)]
    assert wavefronts(ad) == 4
    # N = 16: lanes of a quarter warp read one row of 8 consecutive blocks
    ad = [(l >> 3) * 4 * 512 * esize + (l & 7) * 16 * esize for l in range(32)]
    assert wavefronts(ad) == (8 if esize == 2 else 4)
