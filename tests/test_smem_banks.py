"""Shared-memory bank model of the fused kernels' transposes and staged reads.

A CPU model of the addresses the kernels compute (lane -> block/slab map,
tile strides, XOR chunk swizzle): it counts the wavefronts one warp-wide
access needs (32-bit: one per warp, 64-bit: per half warp, 128-bit: per
quarter warp) and checks the transposes need no more than the minimum.
"""
import pytest


def wavefronts(addrs, width):
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


MIN = {4: 1, 8: 2, 16: 4}


def lane_map(n, tid):
    if n == 16:                      # slab-major: 8 blocks x 4 slabs per warp
        w, l = tid >> 5, tid & 31
        return w * 8 + (l & 7), l >> 3
    return tid // 16, tid % 16       # N = 32: 2 blocks x 16 slabs per warp


GEOM = {16: dict(W=4, CH=4, STRIDE=16 * 16 + 4), 32: dict(W=2, CH=8, STRIDE=32 * 32)}


def swz(n, r):
    g = GEOM[n]
    return (r // g["W"]) & (g["CH"] - 1)


@pytest.mark.parametrize("n", (16, 32))
def test_transposes_conflict_free(n):
    g = GEOM[n]
    for warp in range(4):
        tids = [warp * 32 + l for l in range(32)]
        # rows -> cols: row-slab writes of 16-byte chunks
        for k in range(g["W"]):
            for c in range(g["CH"]):
                ad = []
                for t in tids:
                    lb, p = lane_map(n, t)
                    r = p * g["W"] + k
                    ad.append(4 * (lb * g["STRIDE"] + r * n + 4 * (c ^ swz(n, r))))
                assert wavefronts(ad, 16) == MIN[16]
        # column-slab reads (W words per row): 16 B for N = 16, 8 B for N = 32
        width = 4 * g["W"]
        for i in range(n):
            ad = []
            for t in tids:
                lb, p = lane_map(n, t)
                c, off = (p * g["W"]) >> 2, (p * g["W"]) & 3
                ad.append(4 * (lb * g["STRIDE"] + i * n + 4 * (c ^ swz(n, i)) + off))
            assert wavefronts(ad, width) == MIN[width]


def test_staged_row_reads():
    """128-bit reads of the staged int16 rows: N = 8 conflict free, N = 16 / 32 two-way."""
    ad8 = [0 * 2048 + l * 16 for l in range(32)]
    assert wavefronts(ad8, 16) == MIN[16]
    ad16 = []
    for l in range(32):
        lb, p = lane_map(16, l)
        ad16.append((4 * p) * 1024 + lb * 32)
    assert wavefronts(ad16, 16) == 2 * MIN[16]
    ad32 = []
    for l in range(32):
        lb, p = lane_map(32, l)
        ad32.append((2 * p) * (512 + 16) + lb * 64)
    assert wavefronts(ad32, 16) == 2 * MIN[16]
