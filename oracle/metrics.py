"""Assessment measures of Secs. 3.1 and 4 (test pins for the matrices).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import math

import numpy as np

from . import matrices as mx


def deviation_from_diagonality(m: np.ndarray) -> float:
    """delta(M) = 1 - ||diag M||_F^2 / ||M||_F^2 (Sec. 3.1)."""
    m = np.asarray(m, dtype=np.float64)
    return 1.0 - float(np.sum(np.diag(m) ** 2)) / float(np.sum(m * m))


def total_error_energy(c_approx: np.ndarray) -> float:
    """epsilon_total = pi ||C - C_approx||_F^2 against the exact DCT (Sec. 4.1)."""
    n = c_approx.shape[0]
    d = mx.dct2_matrix(n) - np.asarray(c_approx, dtype=np.float64)
    return math.pi * float(np.sum(d * d))


def ar1_covariance(n: int, rho: float) -> np.ndarray:
    """R_x with entries rho^|m - n| (first-order Markov model, Sec. 4.1)."""
    idx = np.arange(n)
    return rho ** np.abs(idx[:, None] - idx[None, :]).astype(np.float64)


def coding_gain(c: np.ndarray, rho: float, synthesis: str = "rows") -> float:
    """Unified coding gain in dB (Sec. 4.1).

    h_k is row k of C; g_k is row k of C^{-1} as the paper states
    (``synthesis="rows"``) or column k (``"cols"``, the usual synthesis
    basis).  A_k = su[(h_k^T h_k) o R_x] = h_k R_x h_k^T, B_k = ||g_k||^2,
    C_g = 10 log10 prod_k (A_k B_k)^(-1/N).
    """
    c = np.asarray(c, dtype=np.float64)
    n = c.shape[0]
    r = ar1_covariance(n, rho)
    cinv = np.linalg.inv(c)
    total = 0.0
    for k in range(n):
        h = c[k]
        g = cinv[k] if synthesis == "rows" else cinv[:, k]
        a_k = float(np.sum(np.outer(h, h) * r))
        b_k = float(g @ g)
        total += math.log10(a_k * b_k)
    return -10.0 * total / n


def klt_coding_gain(n: int, rho: float) -> float:
    """Coding gain of the KLT of R_x: 10 log10 of mean over geometric mean of
    the eigenvalues (the variance of the AR(1) model is one)."""
    lam = np.linalg.eigvalsh(ar1_covariance(n, rho))
    return 10.0 * (math.log10(float(np.mean(lam))) - float(np.mean(np.log10(lam))))


def stage_adds(m: np.ndarray) -> int:
    """Additions to apply one sparse stage: sum over rows of (nonzeros - 1)."""
    nnz = np.count_nonzero(np.asarray(m), axis=1)
    return int(np.sum(np.maximum(nnz - 1, 0)))


def stage_list(variant: str, n: int):
    """Elementary stages (applied right to left) of T_N for the fast algorithm.

    N = 8: [P_8, M_1, M_2, M_3, M_4, B_8] (Eqs. 4-5).  N > 8: the stages of
    diag(T_{N/2}, T_{N/2}) (each stage block-diagonal), the M^per_N interleave
    on the left and M^add_N on the right (Sec. 6).
    """
    if n == 8:
        a, b, g = mx.params(variant)
        return mx.chen_factors(a, b, g)
    inner = stage_list(variant, n // 2)
    return [mx.M_per(n)] + [mx.block_diag(s, s) for s in inner] + [mx.M_add(n)]


def additive_complexity(variant: str, n: int) -> int:
    """Total additions of the fast algorithm for T_N (Tables 2 and 4)."""
    return sum(stage_adds(s) for s in stage_list(variant, n))


# ---------------------------------------------------------------------------
# SSIM (Sec. 5.1 compares reconstructions by PSNR and by the structural
# similarity index of Wang et al. 2004).  The paper cites the index without
# restating it; the standard form is used: an 11 x 11 circularly symmetric
# Gaussian window (sigma = 1.5, unit sum), K1 = 0.01, K2 = 0.03, L = 255,
# local statistics only where the window lies inside the image, and the mean
# of the SSIM map.
# ---------------------------------------------------------------------------

SSIM_WIN, SSIM_SIGMA, SSIM_K1, SSIM_K2, SSIM_L = 11, 1.5, 0.01, 0.03, 255.0


def ssim_window(size: int = SSIM_WIN, sigma: float = SSIM_SIGMA) -> np.ndarray:
    """w(i, j) proportional to exp(-((i - c)^2 + (j - c)^2) / (2 sigma^2)), summing to one."""
    r = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-(r[:, None] ** 2 + r[None, :] ** 2) / (2.0 * sigma * sigma))
    return g / g.sum()


def _window_filter(a: np.ndarray, w: np.ndarray) -> np.ndarray:
    """sum_{k,l} w[k, l] a[i + k, j + l] for every window lying inside a."""
    from numpy.lib.stride_tricks import sliding_window_view
    return np.einsum("ijkl,kl->ij", sliding_window_view(a, w.shape), w)


def ssim_map(x: np.ndarray, y: np.ndarray, peak: float = SSIM_L) -> np.ndarray:
    """Local SSIM = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2))."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    w = ssim_window()
    mx_, my_ = _window_filter(x, w), _window_filter(y, w)
    sxx = _window_filter(x * x, w) - mx_ * mx_
    syy = _window_filter(y * y, w) - my_ * my_
    sxy = _window_filter(x * y, w) - mx_ * my_
    c1, c2 = (SSIM_K1 * peak) ** 2, (SSIM_K2 * peak) ** 2
    return ((2 * mx_ * my_ + c1) * (2 * sxy + c2)) / ((mx_ * mx_ + my_ * my_ + c1) * (sxx + syy + c2))


def ssim(x: np.ndarray, y: np.ndarray, peak: float = SSIM_L) -> float:
    """Mean SSIM of one image pair (at least 11 x 11)."""
    return float(np.mean(ssim_map(x, y, peak)))
