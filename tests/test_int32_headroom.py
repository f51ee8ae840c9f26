"""Every int32 intermediate of the fused kernels stays below 2^31.

The kernels apply, per block, a row pass, a column pass, the zonal mask, an
inverse column pass and an inverse row pass, each a chain of the paper's
sparse stage matrices (Eqs. 3-7 and the JAM recursion of Sec. 6.1), with U
carried as W = 2U.  For inputs |A| <= 255 the largest value any stage can
produce is bounded by the absolute row sums of the partial products, applied
pass by pass (masking can only shrink the bound).  The inverse stages are
the paper's printed factors, doubled.
"""
import numpy as np
import pytest

from oracle import matrices as mx
from oracle import metrics as me
from tests import golden_io

G = golden_io.matrices()


def w8_stages(v):
    """2 U_8 = B_8 (2M_4^-1)(2M_3^-1)(2M_2^-1) M_1^T P_8^T, first-applied first."""
    m3 = G["M3_tilde"][0] if v == "tilde" else G["M3_hat_inv"][0]   # 2 M~_3^{-1} = M~_3
    return [mx.P8().T, mx.M1().T, G[f"M2_{v}_inv"][0], m3, G["M4_inv"][0], mx.B8()]


def t_stages(v, n):
    return list(reversed(me.stage_list(v, n)))


def w_stages(v, n):
    if n == 8:
        return w8_stages(v)
    inner = w_stages(v, n // 2)
    return [mx.M_per(n).T] + [mx.block_diag(s, s) for s in inner] + [mx.M_add(n)]


def transposed(stages):
    return [s.T for s in reversed(stages)]


def chain_bounds(stages, xb):
    out, p = [], np.eye(len(xb), dtype=np.int64)
    for s in stages:
        p = s.astype(np.int64) @ p
        out.append(np.abs(p) @ xb)
    return out, p


@pytest.mark.parametrize("variant", ("tilde", "hat"))
@pytest.mark.parametrize("n", (8, 16, 32))
@pytest.mark.parametrize("conv", ("paper", "transpose"))
def test_int32_headroom(variant, n, conv):
    wst = w_stages(variant, n)
    _, wp = chain_bounds(wst, np.ones(n))
    np.testing.assert_array_equal(wp, 2 * mx.U_N(variant, n))
    fr = transposed(wst) if conv == "paper" else t_stages(variant, n)
    fc, ic = t_stages(variant, n), wst
    ir = transposed(t_stages(variant, n)) if conv == "paper" else wst
    worst = 0.0
    b, _ = chain_bounds(fr, np.full(n, 255.0))
    worst = max(worst, max(x.max() for x in b))
    b2 = np.zeros((n, n))
    for j in range(n):
        bb, _ = chain_bounds(fc, np.full(n, b[-1][j]))
        worst = max(worst, max(x.max() for x in bb))
        b2[:, j] = bb[-1]
    b3 = np.zeros((n, n))
    for j in range(n):
        bb, _ = chain_bounds(ic, b2[:, j])
        worst = max(worst, max(x.max() for x in bb))
        b3[:, j] = bb[-1]
    for i in range(n):
        bb, _ = chain_bounds(ir, b3[i, :])
        worst = max(worst, max(x.max() for x in bb))
    assert worst < 2 ** 31 - 1, worst
