"""The JPEG-like block pipeline of Sec. 5.1, as explicit matrix products.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

For an N x N block A, with T = T_N (integer), U = N T_N^{-1} (integer) and
s = diag(S_N):

* PAPER convention (Sec. 5.1 writes B = C A C^{-1} and A' = C^{-1} B C with
  C = diag(s) T):  Y = T A U, so B = diag(s) Y diag(s)^{-1} / N;
  Z = U Ym T, so the reconstruction is Z / N^2.
* TRANSPOSE convention (the usual B = C A C^T, A' = C^{-1} B C^{-T}):
  Y = T A T^T, B = diag(s) Y diag(s); Z = U Ym U^T, reconstruction Z / N^2.

Ym keeps the first r coefficients in zig-zag order and zeroes the rest.  S is
diagonal and the mask elementwise, so S cancels exactly in the
reconstruction; it only enters the scaled coefficients B.

Sizes not divisible by N are padded by replicating the last row / column; the
reconstruction and the PSNR cover the original H x W pixels only.  The
exact-DCT variant uses C_8^II in float64: B = C A C^T, A' = C^T Bm C.
"""
from __future__ import annotations

import math

import numpy as np

from . import matrices as mx

CONVS = ("paper", "transpose")


# ---------------------------------------------------------------------------
# zig-zag order and zonal mask (Sec. 5.1)
# ---------------------------------------------------------------------------

def zigzag_order(n: int):
    """Zig-zag scan of an n x n grid as a list of (row, col).

    Anti-diagonals d = row + col in increasing order; on an even d the row
    index decreases along the diagonal, on an odd d it increases.  For n = 8
    this is the standard JPEG sequence the paper cites.
    """
    order = []
    for d in range(2 * n - 1):
        rows = range(max(0, d - n + 1), min(d, n - 1) + 1)
        rows = reversed(rows) if d % 2 == 0 else rows
        for i in rows:
            order.append((i, d - i))
    return order


def zonal_mask(n: int, r: int) -> np.ndarray:
    """n x n 0/1 mask keeping the first r zig-zag positions."""
    if not 1 <= r <= n * n:
        raise ValueError("r must be in [1, N*N]")
    m = np.zeros((n, n), dtype=np.int64)
    for i, j in zigzag_order(n)[:r]:
        m[i, j] = 1
    return m


# ---------------------------------------------------------------------------
# image <-> blocks
# ---------------------------------------------------------------------------

def pad_replicate(img: np.ndarray, n: int) -> np.ndarray:
    """Pad the last two axes up to multiples of n by repeating the edge."""
    h, w = img.shape[-2:]
    hp, wp = -(-h // n) * n, -(-w // n) * n
    pad = [(0, 0)] * (img.ndim - 2) + [(0, hp - h), (0, wp - w)]
    return np.pad(img, pad, mode="edge")


def to_blocks(img: np.ndarray, n: int) -> np.ndarray:
    """[..., H', W'] -> [..., H'/n, W'/n, n, n] (block-major view copy)."""
    *lead, hp, wp = img.shape
    b = img.reshape(*lead, hp // n, n, wp // n, n)
    return np.moveaxis(b, -3, -2).copy()


def from_blocks(blocks: np.ndarray) -> np.ndarray:
    """Inverse of ``to_blocks``."""
    *lead, nby, nbx, n, _ = blocks.shape
    b = np.moveaxis(blocks, -2, -3)
    return b.reshape(*lead, nby * n, nbx * n)


# ---------------------------------------------------------------------------
# 2-D transforms on blocks (explicit matrix products)
# ---------------------------------------------------------------------------

def forward_blocks(a: np.ndarray, t: np.ndarray, u: np.ndarray, conv: str) -> np.ndarray:
    """Integer coefficients Y per block: T A U (paper) or T A T^T (transpose)."""
    a = a.astype(np.int64)
    right = u if conv == "paper" else t.T
    return t @ a @ right


def inverse_blocks(ym: np.ndarray, t: np.ndarray, u: np.ndarray, conv: str) -> np.ndarray:
    """Integer Z = N^2 * reconstruction: U Ym T (paper) or U Ym U^T (transpose)."""
    right = t if conv == "paper" else u.T
    return u @ ym.astype(np.int64) @ right


def scaled_coeffs(y: np.ndarray, s: np.ndarray, n: int, conv: str) -> np.ndarray:
    """Scaled coefficients B (float64) from Y (Sec. 3.1 scale S applied)."""
    y = y.astype(np.float64)
    if conv == "paper":
        return s[:, None] * y / s[None, :] / n
    return s[:, None] * y * s[None, :]


def kept_coeffs(ym: np.ndarray, n: int, r: int) -> np.ndarray:
    """The first r coefficients of each block in zig-zag order, [..., r]."""
    idx = zigzag_order(n)[:r]
    rows = np.array([i for i, _ in idx])
    cols = np.array([j for _, j in idx])
    return ym[..., rows, cols]


# ---------------------------------------------------------------------------
# full pipeline
# ---------------------------------------------------------------------------

def fzi_integer(img: np.ndarray, n: int, variant: str, r: int, conv: str = "paper"):
    """Forward -> zonal(r) -> inverse on an integer image [..., H, W].

    Returns a dict with the block-major integer arrays ``y``, ``ym``, ``z``
    (shape [..., nby, nbx, n, n]) and the float64 reconstruction ``recon``
    (shape [..., H, W]) = Z / N^2 cropped to the original size.
    """
    t = mx.T_N(variant, n)
    u = mx.U_N(variant, n)
    h, w = img.shape[-2:]
    a = to_blocks(pad_replicate(np.asarray(img).astype(np.int64), n), n)
    y = forward_blocks(a, t, u, conv)
    ym = y * zonal_mask(n, r)
    z = inverse_blocks(ym, t, u, conv)
    recon = from_blocks(z).astype(np.float64) / float(n * n)
    return {"y": y, "ym": ym, "z": z, "recon": recon[..., :h, :w]}


def fzi_exact(img: np.ndarray, r: int, n: int = 8):
    """Exact DCT variant: B = C A C^T, Bm = mask o B, A' = C^T Bm C (float64)."""
    c = mx.dct2_matrix(n)
    h, w = img.shape[-2:]
    a = to_blocks(pad_replicate(np.asarray(img).astype(np.float64), n), n)
    b = c @ a @ c.T
    bm = b * zonal_mask(n, r)
    rec = c.T @ bm @ c
    return {"b": b, "bm": bm, "recon": from_blocks(rec)[..., :h, :w]}


# ---------------------------------------------------------------------------
# error and PSNR (Sec. 5.1)
# ---------------------------------------------------------------------------

def sse_integer(img: np.ndarray, z_blocks: np.ndarray, n: int) -> int:
    """Exact sum over the original pixels of (N^2 A - Z)^2, a Python int.

    ``img`` is one image [H, W]; ``z_blocks`` its [nby, nbx, n, n] Z.
    """
    h, w = img.shape
    z = from_blocks(z_blocks)[:h, :w]
    e = (n * n) * np.asarray(img).astype(np.int64) - z
    e2 = (e * e).ravel()                      # |e| < 2^31, so e^2 < 2^62
    lo = e2 & ((1 << 31) - 1)
    hi = e2 >> 31
    return int(np.sum(hi, dtype=np.int64)) * (1 << 31) + int(np.sum(lo, dtype=np.int64))


def psnr_from_sse(sse_num: int, n: int, npix: int, peak: float = 255.0) -> float:
    """PSNR in dB from the exact numerator sum (N^2 A - Z)^2; +inf if zero.

    MSE = sse_num / (N^4 npix); PSNR = 10 log10(peak^2 / MSE).
    """
    if sse_num == 0:
        return math.inf
    return 10.0 * (math.log10(peak * peak) + math.log10(n ** 4 * npix) - math.log10(sse_num))


def psnr_float(ref: np.ndarray, recon: np.ndarray, peak: float = 255.0) -> float:
    """PSNR of a float64 reconstruction against the reference; +inf if equal."""
    d = np.asarray(ref, dtype=np.float64) - np.asarray(recon, dtype=np.float64)
    mse = float(np.mean(d * d))
    return math.inf if mse == 0.0 else 10.0 * math.log10(peak * peak / mse)


def psnr_integer_path(img: np.ndarray, n: int, variant: str, r: int, conv: str = "paper"):
    """Per-image PSNR list for a batch [B, H, W] (or one image) via exact SSE."""
    res = fzi_integer(img, n, variant, r, conv)
    imgs = img if img.ndim == 3 else img[None]
    zs = res["z"] if img.ndim == 3 else res["z"][None]
    h, w = imgs.shape[-2:]
    return [psnr_from_sse(sse_integer(imgs[b], zs[b], n), n, h * w) for b in range(imgs.shape[0])]
