"""Exactness of the separable packed kernels (csrc/sep_body.cuh).

They run the paper-convention transform (Sec. 5.1) as four 1-D passes,
  A  X  = T A          (columns; two 16-bit lanes per 32-bit word)
  B  2Y = X W, mask, Q = 2Ym T     (rows; float pairs)
  C  4Z = W Q          (columns; float pairs)
each a chain of the paper's sparse stage matrices (Eqs. 3-7, the JAM
recursion of Sec. 6.1; W = 2U).  Float arithmetic on integers is exact while
every value stays below 2^24, and the 16-bit lanes of pass A decode exactly
while every output X stays within [-2^15, 2^15).

For inputs |A| <= 255 the worst case of any linear intermediate is 255 times
the l1 norm of its coefficients over the block's pixels.  Before the mask
the 2-D map is separable (outer products of a T row and a stage row), after
it the coefficients of pass C are summed explicitly, so the bounds below are
exact, not estimates.
"""
import numpy as np
import pytest

from oracle import matrices as mx
from oracle import pipeline as pl
from tests.test_int32_headroom import t_stages, transposed, w_stages


def partial_products(stages):
    out, p = [], np.eye(stages[0].shape[1], dtype=np.int64)
    for s in stages:
        p = s.astype(np.int64) @ p
        out.append(p.copy())
    return out


def worst_cases(variant, n, r):
    t = mx.T_N(variant, n).astype(np.int64)
    w = 2 * mx.U_N(variant, n).astype(np.int64)
    ts, ws = t_stages(variant, n), w_stages(variant, n)
    mask = pl.zonal_mask(n, r).astype(np.int64)
    out = {}
    pa = partial_products(ts)
    assert np.array_equal(pa[-1], t)
    out["A"] = max(255 * np.abs(p).sum(1).max() for p in pa)
    out["X"] = 255 * np.abs(t).sum(1).max()
    row_l1 = np.abs(t).sum(1)
    pb = partial_products(transposed(ws))
    assert np.array_equal(pb[-1], w.T)
    out["B_fwd"] = max(255 * row_l1.max() * np.abs(p).sum(1).max() for p in pb)
    pc = partial_products(transposed(ts))
    assert np.array_equal(pc[-1], t.T)
    worst_b, rows = 0, {}
    for i in range(n):
        mi = mask[i][:, None] * w.T               # masked 2Y[i][j] = sum_{m,k} T[i][m] A[m][k] W[k][j] mask[i][j]
        for p in pc:
            worst_b = max(worst_b, 255 * row_l1[i] * np.abs(p @ mi).sum(1).max())
        rows[i] = pc[-1] @ mi                     # Q[i][l] = sum_{m,k} T[i][m] rows[i][l][k] A[m][k]
    out["B_inv"] = worst_b
    pd = partial_products(ws)
    assert np.array_equal(pd[-1], w)
    worst_c = 0
    for l in range(n):
        cs = np.stack([np.outer(t[i], rows[i][l]) for i in range(n)])
        for p in pd:
            worst_c = max(worst_c, 255 * np.abs(np.einsum("si,imk->smk", p, cs)).sum((1, 2)).max())
    out["C"] = worst_c
    return out


@pytest.mark.parametrize("variant", ("tilde", "hat"))
@pytest.mark.parametrize("n", (16, 32))
def test_separable_order_is_exact_in_float32(variant, n):
    r = n * n // 4
    w = worst_cases(variant, n, r)
    assert w["X"] < 2 ** 15                     # pass A lanes decode exactly
    assert w["X"] == 255 * n                    # the DC row of T_N is all ones
    for k in ("B_fwd", "B_inv", "C"):
        assert w[k] < 2 ** 24, (k, w[k])


def test_bounds_are_attained_by_sign_patterns():
    """The pass-C bound is a worst case that an input reaches: the sign pattern
    of the worst coefficient matrix, times 255, gives exactly that value."""
    variant, n, r = "hat", 16, 64
    t = mx.T_N(variant, n).astype(np.int64)
    w = 2 * mx.U_N(variant, n).astype(np.int64)
    mask = pl.zonal_mask(n, r).astype(np.int64)
    # 4Z = W (mask o (T A W)) T for the paper convention (W = 2U)
    # coefficients of 4Z[0][0] over A: c[m][k] = sum_{i,j} W[0][i] mask[i][j] T[i][m] W[k][j] T[j][0]
    c = np.einsum("i,ij,im,kj,j->mk", w[0], mask, t, w, t[:, 0])
    a = 255 * np.sign(c)
    z4 = w @ (mask * (t @ a @ w)) @ t
    assert z4[0, 0] == 255 * np.abs(c).sum()
    res = pl.fzi_integer(a.astype(np.int64), n, variant, r)
    assert res["z"][0, 0, 0, 0] * 4 == z4[0, 0]
