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


# ---- separable packed bodies (csrc/sep_body.cuh), paper convention, r = N^2/4
# N = 32: lane -> (block lane >> 4, column pair lane & 15); pass-B task
# t = min(lane, 23) -> (block t // 12, row pair t % 12).  Exchange words:
# xA b*472 + c*28 + i; xB chunk b*212 + c*13 + r; mask table pairs
# b*312 + r*26 + j (two copies).
def sep32_task(l):
    t = min(l, 23)
    return t // 12, t % 12


def test_sep32_accesses_conflict_free():
    for i in range(32):      # pass A: staged row i (528-byte pitch), 4 bytes per lane
        assert wavefronts([(l >> 4) * 64 + 4 * (l & 15) + i * 528 for l in range(32)], 4) == 1
    for q in range(6):       # xA writes, 4 rows per 128-bit store
        assert wavefronts([4 * ((l >> 4) * 472 + (l & 15) * 28 + 4 * q) for l in range(32)]) == 4
    for cp in range(16):     # pass B reads of xA (rows 2r, 2r + 1)
        ad = [4 * (sep32_task(l)[0] * 472 + 2 * sep32_task(l)[1] + cp * 28) for l in range(32)]
        assert wavefronts(ad, 8) == 2
    for j in range(0, 23, 2):  # mask pairs j, j + 1 of the lane's row pair
        ad = [8 * (sep32_task(l)[0] * 312 + sep32_task(l)[1] * 26 + j) for l in range(32)]
        assert wavefronts(ad) == 4
    for cp in range(16):     # xB writes by the 24 pass-B lanes
        ad = {l: 16 * (sep32_task(l)[0] * 212 + cp * 13 + sep32_task(l)[1]) for l in range(24)}
        assert wavefronts_subset(ad) == 3
    for rp in range(12):     # pass C reads of xB
        assert wavefronts([16 * ((l >> 4) * 212 + (l & 15) * 13 + rp) for l in range(32)]) == 4
    xa = {b * 472 + c * 28 + i for b in range(2) for c in range(16) for i in range(24)}
    xb = {(b * 212 + c * 13 + r) for b in range(2) for c in range(16) for r in range(12)}
    assert len(xa) == 2 * 16 * 24 and max(xa) < 1680
    assert len(xb) == 2 * 16 * 12 and 4 * max(xb) + 3 < 1680
    assert (12 * 26 * 8 // 16) % 8 == 4    # second mask copy 156 chunks on: rows r and r + 8 split banks


# N = 16: lane -> (block (l & 3) + 4 (l >> 4), column quad (l >> 2) & 3);
# pass-B task t (rounds of 32) -> (block t & 7, row pair t >> 3), t < 48.
# xA words cp*104 + b*12 + i; xB chunks 208 + b*49 + cp*6 + r.
def sep16_lane(l):
    return (l & 3) + 4 * (l >> 4), (l >> 2) & 3


def test_sep16_accesses_conflict_free():
    for i in range(16):      # pass A: staged row i, 8 bytes per lane (columns 4q .. 4q+3)
        ad = [sep16_lane(l)[0] * 32 + 8 * sep16_lane(l)[1] + i * 1024 for l in range(32)]
        assert wavefronts(ad, 8) == 2
    for h, t in itertools.product(range(2), range(3)):   # xA writes, column pair 2q + h
        ad = [4 * ((2 * sep16_lane(l)[1] + h) * 104 + sep16_lane(l)[0] * 12 + 4 * t) for l in range(32)]
        assert wavefronts(ad) == 4
    for rd in range(2):
        tasks = [min(rd * 32 + l, 47) for l in range(32)]
        for cp in range(8):  # pass B reads of xA
            assert wavefronts([4 * (cp * 104 + (t & 7) * 12 + 2 * (t >> 3)) for t in tasks], 8) == 2
            ad = {l: 16 * (208 + (t & 7) * 49 + cp * 6 + (t >> 3)) for l, t in enumerate(tasks)
                  if rd * 32 + l < 48}
            assert wavefronts_subset(ad) == (4 if rd == 0 else 2)
    for h, rp in itertools.product(range(2), range(6)):  # pass C reads of xB
        ad = [16 * (208 + sep16_lane(l)[0] * 49 + (2 * sep16_lane(l)[1] + h) * 6 + rp) for l in range(32)]
        assert wavefronts(ad) == 4
    xa = {cp * 104 + b * 12 + i for cp in range(8) for b in range(8) for i in range(12)}
    xb = {208 + b * 49 + cp * 6 + r for b in range(8) for cp in range(8) for r in range(6)}
    assert len(xa) == 8 * 8 * 12 and max(xa) < 832
    assert len(xb) == 8 * 8 * 6 and min(xb) * 4 >= 832 and 4 * max(xb) + 3 < 832 + 4 * 8 * 49


def wavefronts_subset(addrs, width=16):
    """wavefronts of a 128-bit access by the lanes present in `addrs` (lane -> byte address)"""
    total = 0
    for ph in [range(8 * i, 8 * i + 8) for i in range(4)]:
        banks = {}
        for lane in ph:
            if lane not in addrs:
                continue
            for w in range(width // 4):
                word = addrs[lane] // 4 + w
                banks.setdefault(word % 32, set()).add(word)
        if banks:
            total += max(len(s) for s in banks.values())
    return total
