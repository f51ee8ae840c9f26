"""The operand layouts of the tcgen05 inference kernel (csrc/cnn_infer_tc.cuh),
modelled on the CPU.

A tcgen05 MMA reads its operands from shared memory through descriptors:
K-major, no swizzle, core matrices of 8 rows x 16 bytes, `lbo` bytes apart
along K and `sbo` bytes apart along M (or N), element (row, k) of the
operand at start + (k / 8) lbo + (row / 8) sbo + (row % 8) 16 + (k % 8) 2.
This test builds the kernel's shared-memory images (the expanded region E,
the parity-split conv2 input map of a pair, the side-by-side conv3 map, and
the packed B operands, including conv2's zero-padded N = 128 operand per
receptive-field offset), reads every MMA operand through that descriptor
formula, multiplies, pools the accumulator rows as the epilogues do, and
checks the result against a direct 3 x 3 convolution and 2 x 2 max pool.
It pins the address arithmetic of the design, not the CUDA code.
"""
import numpy as np


def desc_read(mem, addr, lbo, sbo, rows, k):
    out = np.zeros((rows, k))
    for r in range(rows):
        for kk in range(k):
            out[r, kk] = mem[(addr + (kk // 8) * lbo + (r // 8) * sbo + (r % 8) * 16 + (kk % 8) * 2) // 2]
    return out


def b_off(n, k):
    return (k >> 3) * 128 + (n >> 3) * 256 + (n & 7) * 16 + (k & 7) * 2


def conv_pool(x, w):
    """x [C][H][W], w [O][C][3][3] -> max over 2 x 2 of the zero-padded correlation."""
    c, h, wd = x.shape
    xp = np.zeros((c, h + 2, wd + 2))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((w.shape[0], h, wd))
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("oc,chw->ohw", w[:, :, dy, dx], xp[:, dy:dy + h, dx:dx + wd])
    return y.reshape(w.shape[0], h // 2, 2, wd // 2, 2).max(axis=(2, 4))


# conv2 input map of a pair: offset of padded pixel (R, C) of region s, channel plane p
CPAR, RS, RP = 144, 288, 576
RPAR, PLANE = 9 * RP, 2 * 9 * RP


def a1_off(s, p, r, c):
    return p * PLANE + (r & 1) * RPAR + (r >> 1) * RP + s * RS + (c & 1) * CPAR + (c >> 1) * 16


def test_conv1_conv2_conv3_operand_layouts():
    rng = np.random.default_rng(0)
    w1 = rng.standard_normal((16, 1, 3, 3))
    w2 = rng.standard_normal((32, 16, 3, 3))
    w3 = rng.standard_normal((32, 32, 3, 3))
    regions = [rng.standard_normal((32, 32)) for _ in range(2)]
    mem = np.zeros(1 << 17)
    # ---- conv1: E[17][16] entries of 16 B per region, B1 = 64 x 16 ----------
    erow, ebytes, e0, b1 = 256, 17 * 256, 0, 20000
    for s, img in enumerate(regions):
        p = np.zeros((34, 34))
        p[1:33, 1:33] = img
        for j in range(17):
            for u in range(16):
                for c in range(4):
                    for h in range(2):
                        mem[(e0 + s * ebytes + j * erow + u * 16 + (2 * c + h) * 2) // 2] = p[2 * j + h, 2 * u + c]
    for n in range(64):
        for k in range(16):
            g, o = n >> 4, n & 15
            ry, rx = 2 * (k >> 3) + (k & 1), (k >> 1) & 3
            dy, dx = ry - (g >> 1), rx - (g & 1)
            mem[(b1 + b_off(n, k)) // 2] = w1[o, 0, dy, dx] if 0 <= dy <= 2 and 0 <= dx <= 2 else 0.0
    a1 = 40000
    bmat = desc_read(mem, b1, 128, 256, 64, 16)
    for s in range(2):
        for t in range(2):
            d = desc_read(mem, e0 + s * ebytes + t * 8 * erow, erow, 128, 128, 16) @ bmat.T
            for m in range(128):                       # lane m = 16 v_local + u
                v, u = 8 * t + (m >> 4), m & 15
                pooled = d[m].reshape(4, 16).max(axis=0)
                for ch in range(16):
                    mem[(a1 + a1_off(s, ch // 8, v + 1, u + 1) + (ch % 8) * 2) // 2] = pooled[ch]
    act1 = [conv_pool(img[None], w1) for img in regions]
    for s in range(2):
        got = np.array([[[mem[(a1 + a1_off(s, ch // 8, v + 1, u + 1) + (ch % 8) * 2) // 2] for u in range(16)]
                         for v in range(16)] for ch in range(16)])
        np.testing.assert_allclose(got, act1[s], atol=1e-9)
    # ---- conv2: one N = 128 MMA per receptive-field offset (ry, rx) -----------
    b2 = 90000
    d2 = np.zeros((128, 128))
    for off in range(16):
        ry, rx = off >> 2, off & 3
        for n in range(128):
            g, o = n >> 5, n & 31
            dy, dx = ry - (g >> 1), rx - (g & 1)
            for c in range(16):
                mem[(b2 + off * 4096 + b_off(n, c)) // 2] = w2[o, c, dy, dx] if 0 <= dy <= 2 and 0 <= dx <= 2 else 0.0
        a = desc_read(mem, a1 + (ry & 1) * RPAR + (ry >> 1) * RP + (rx & 1) * CPAR + (rx >> 1) * 16, PLANE, RS, 128, 16)
        d2 += a @ desc_read(mem, b2 + off * 4096, 128, 256, 128, 16).T
    act2 = [conv_pool(x, w2) for x in act1]
    a3plane, a3 = 3200, 160000
    for m in range(128):                               # lane m = 8 i + u, i = 2 v + s
        i, u = m >> 3, m & 7
        v, s = i >> 1, i & 1
        pooled = d2[m].reshape(4, 32).max(axis=0)
        np.testing.assert_allclose(pooled, act2[s][:, v, u], atol=1e-9)
        for ch in range(32):
            mem[(a3 + (ch // 8) * a3plane + ((v + 1) * 20 + 10 * s + u + 1) * 16 + (ch % 8) * 2) // 2] = pooled[ch]
    # ---- conv3: pixel-tiled, the pair side by side, 18 MMAs of N = 32 ---------
    b3 = 180000
    d3 = np.zeros((128, 32))
    for j in range(18):
        tap, h = j >> 1, j & 1
        for o in range(32):
            for c in range(16):
                mem[(b3 + j * 1024 + b_off(o, c)) // 2] = w3[o, 16 * h + c, tap // 3, tap % 3]
        a = desc_read(mem, a3 + ((tap // 3) * 20 + tap % 3) * 16 + 2 * h * a3plane, a3plane, 160, 128, 16)
        d3 += a @ desc_read(mem, b3 + j * 1024, 128, 256, 32, 16).T
    feat = [conv_pool(x, w3) for x in act2]
    for m in range(0, 128):                            # core matrix k = m // 8: region k & 1, output row k >> 1
        k, x = m >> 3, m & 7
        s, yrow = k & 1, k >> 1
        if yrow % 2 or x % 2:
            continue                                   # the window's top-left lane
        partners = [m, m ^ 1, m ^ 16, m ^ 17]          # x neighbour one lane away, y neighbour 16 lanes away
        pooled = d3[partners].max(axis=0)
        np.testing.assert_allclose(pooled, feat[s][:, yrow // 2, x // 2], atol=1e-9)


def test_training_gemm_tma_stage_layout():
    """The training GEMM's A stages (csrc/cnn_train.cu): TMA writes a box of
    8 K x 128 rows as 128 rows of 16 contiguous bytes, box c of a 64-K stage
    at c * 2048.  Read with lbo = 2048 and sbo = 128 from chunk 2 kk, the K = 16
    operand kk of the stage is rows x K[16 kk .. 16 kk + 15] of the tile; the B
    slab layout (lbo 128, sbo 256) gives W[n][16 kk ..]."""
    rng = np.random.default_rng(1)
    m, kdim, bn = 200, 144, 32
    a = rng.standard_normal((m, kdim))
    b = rng.standard_normal((bn, kdim))
    want = a @ b.T
    got = np.zeros((256, bn))
    mem = np.zeros(1 << 16)
    bbase = 0
    for kc in range(kdim // 8):                      # B: slab kc/2, core matrices 128 B along K, 256 B along N
        for r in range(bn):
            for e in range(8):
                mem[(bbase + (kc >> 1) * bn * 32 + (r >> 3) * 256 + (kc & 1) * 128 + (r & 7) * 16 + e * 2) // 2] = \
                    b[r, 8 * kc + e]
    sa = 40000
    for tile in range(2):                            # rows past m read as zero (TMA fill)
        for k0 in range(0, kdim, 64):
            kn = min(64, kdim - k0)
            for c in range(kn // 8):                 # one box per 8 K
                for r in range(128):
                    row = tile * 128 + r
                    for e in range(8):
                        mem[(sa + c * 2048 + r * 16 + e * 2) // 2] = a[row, k0 + 8 * c + e] if row < m else 0.0
            for kk in range(kn // 16):
                am = desc_read(mem, sa + 2 * kk * 2048, 2048, 128, 128, 16)
                bm = desc_read(mem, bbase + (k0 // 16 + kk) * bn * 32, 128, 256, bn, 16)
                got[tile * 128:tile * 128 + 128] += am @ bm.T
    np.testing.assert_allclose(got[:m], want, atol=1e-9)
    assert not got[m:].any()
