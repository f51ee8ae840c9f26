"""Pins of the CPU oracle against what the paper prints and what mathematics fixes.

No GPU.  Every expected value here is either typed from the paper
(tests/golden/, cited there), a closed form, or brute force on a tiny input.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import matrices as mx
from oracle import metrics as me
from oracle import pipeline as pl
from tests import golden_io

G = golden_io.matrices()
S = golden_io.scalars()
VARIANTS = ("tilde", "hat")


def frac_mat(arr, scale):
    return [[Fraction(int(v)) * scale for v in row] for row in arr]


def frac_matmul(a, b):
    n, k, m = len(a), len(b), len(b[0])
    return [[sum(a[i][t] * b[t][j] for t in range(k)) for j in range(m)] for i in range(n)]


def frac_of(arr):
    return [[Fraction(int(v)) for v in row] for row in np.asarray(arr)]


def frac_block_diag(a, b):
    n, m = len(a), len(b)
    z = Fraction(0)
    top = [list(r) + [z] * m for r in a]
    bot = [[z] * n + list(r) for r in b]
    return top + bot


# ---------------------------------------------------------------------------
# Sec. 2-3: factors and the two 8-point approximations
# ---------------------------------------------------------------------------

def test_exact_parameters_give_twice_the_dct():
    """T_C at the exact Chen constants equals 2 C_8^II (Sec. 3)."""
    a, b, g = mx.chen_params_exact()
    np.testing.assert_allclose(mx.T_C(a, b, g), 2.0 * mx.dct2_matrix(8), atol=1e-12)


def test_dct_matrices_orthonormal():
    for n in (4, 8, 16, 32):
        for c in (mx.dct2_matrix(n), mx.dct4_matrix(n)):
            np.testing.assert_allclose(c @ c.T, np.eye(n), atol=1e-12)


def test_chen_dct4_factorization():
    """Eqs. 1-2 with orthonormal C_4 blocks hold up to the printed scale.

    Reading: with C_N^II / C_N^IV normalised as in Sec. 2, Eq. 1 holds with
    1/sqrt(2) in place of 1/2, and Eq. 2 as Q A_1 A_2 A_3 = sqrt(2) C_4^IV
    I-bar_4.  Eq. 3 (the one the method uses) holds exactly: see
    ``test_exact_parameters_give_twice_the_dct``.
    """
    a, b, _ = mx.chen_params_exact()
    j4 = mx.counter_identity(4).astype(float)
    lhs = mx.Q4() @ mx.A1(b) @ mx.A2() @ mx.A3(a)
    np.testing.assert_allclose(lhs, math.sqrt(2.0) * mx.dct4_matrix(4) @ j4, atol=1e-12)
    mid = mx.block_diag(mx.dct2_matrix(4), j4 @ mx.dct4_matrix(4) @ j4)
    np.testing.assert_allclose(mx.P8() @ mid @ mx.B8() / math.sqrt(2.0), mx.dct2_matrix(8),
                               atol=1e-12)


def test_parameter_vectors():
    """sign() gives all ones; round() gives (1, 1,1,1,0, 1,0) (beta_3 rounds to 0)."""
    assert mx.sign_params() == (1, [1, 1, 1, 1], [1, 1])
    assert mx.round_params() == (1, [1, 1, 1, 0], [1, 0])
    # the paper's round is half away from zero, as in C
    assert [mx.paper_round(x) for x in (0.5, -0.5, 1.5, -2.5, 0.49)] == [1, -1, 2, -3, 0]


@pytest.mark.parametrize("variant", VARIANTS)
def test_stage_matrices_match_printed(variant):
    a, b, g = mx.params(variant)
    np.testing.assert_array_equal(mx.M2(b), G[f"M2_{variant}"][0])
    np.testing.assert_array_equal(mx.M3(a, g), G[f"M3_{variant}"][0])
    np.testing.assert_array_equal(mx.M4(a), G["M4"][0])
    np.testing.assert_array_equal(mx.P8(), G["P8"][0])


@pytest.mark.parametrize("variant", VARIANTS)
def test_T8_matches_printed(variant):
    """P_8 M_1 M_2 M_3 M_4 B_8 reproduces the printed T~_8 / T^_8 (Eqs. 4-5)."""
    np.testing.assert_array_equal(mx.T8(variant), G[f"T8_{variant}"][0])


def test_printed_inverse_factor_identities():
    """M~_3^{-1} = M~_3 / 2, B_8^{-1} = B_8^T / 2, M_1^{-1} = M_1^T, P_8^{-1} = P_8^T."""
    m3t = frac_of(G["M3_tilde"][0])
    half = [[x / 2 for x in row] for row in m3t]
    ident = [[Fraction(int(i == j)) for j in range(8)] for i in range(8)]
    assert frac_matmul(m3t, half) == ident
    b8 = frac_of(mx.B8())
    assert frac_matmul(b8, [[x / 2 for x in row] for row in frac_of(mx.B8().T)]) == ident
    assert frac_matmul(frac_of(mx.M1()), frac_of(mx.M1().T)) == ident
    assert frac_matmul(frac_of(mx.P8()), frac_of(mx.P8().T)) == ident


@pytest.mark.parametrize("variant", VARIANTS)
def test_printed_inverse_factors_are_inverses(variant):
    """Each printed inverse factor of Eqs. 6-7 inverts its stage matrix."""
    ident = [[Fraction(int(i == j)) for j in range(8)] for i in range(8)]
    m2inv = frac_mat(*G[f"M2_{variant}_inv"])
    assert frac_matmul(frac_of(G[f"M2_{variant}"][0]), m2inv) == ident
    m4inv = frac_mat(*G["M4_inv"])
    assert frac_matmul(frac_of(G["M4"][0]), m4inv) == ident
    if variant == "hat":
        m3inv = frac_mat(*G["M3_hat_inv"])
        assert frac_matmul(frac_of(G["M3_hat"][0]), m3inv) == ident


def _printed_inverse_chain_8(variant):
    """(1/2) B_8^T M_4^{-1} M_3^{-1} M_2^{-1} M_1^T P_8^T from the printed factors (Eqs. 6-7)."""
    if variant == "tilde":
        m3inv = [[x / 2 for x in row] for row in frac_of(G["M3_tilde"][0])]
    else:
        m3inv = frac_mat(*G["M3_hat_inv"])
    chain = [frac_of(G["P8"][0]) and [[x / 2 for x in row] for row in frac_of(mx.B8().T)],
             frac_mat(*G["M4_inv"]), m3inv, frac_mat(*G[f"M2_{variant}_inv"]),
             frac_of(mx.M1().T), frac_of(G["P8"][0].T)]
    out = chain[0]
    for f in chain[1:]:
        out = frac_matmul(out, f)
    return out


@pytest.mark.parametrize("variant", VARIANTS)
def test_U8_equals_printed_inverse_chain(variant):
    """U_8 = 8 T_8^{-1} equals 8 x the product of the printed inverse factors."""
    inv = _printed_inverse_chain_8(variant)
    u = mx.U_N(variant, 8)
    assert [[x * 8 for x in row] for row in inv] == frac_of(u)
    # and it inverts the printed T_8
    assert frac_matmul(frac_of(G[f"T8_{variant}"][0]), inv) == frac_of(np.eye(8, dtype=np.int64))


# ---------------------------------------------------------------------------
# Sec. 3.1: near orthogonality and the diagonal scale
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("variant", VARIANTS)
def test_scale_and_deviation_from_diagonality(variant):
    t = G[f"T8_{variant}"][0]
    ttt = mx.T8(variant) @ mx.T8(variant).T
    expected_diag, _ = S[f"diagTTt_{variant}"]
    np.testing.assert_array_equal(np.diag(ttt), expected_diag)
    np.testing.assert_allclose(mx.scale_S(mx.T8(variant)), 1.0 / np.sqrt(expected_diag), rtol=1e-15)
    val, tol = S[f"delta_TTt_{variant}"]
    assert abs(me.deviation_from_diagonality(ttt) - val) <= tol
    # T T^T is NOT diagonal (the paper's point in Sec. 3.1); delta of a diagonal matrix is 0
    assert np.count_nonzero(ttt - np.diag(np.diag(ttt))) > 0
    assert me.deviation_from_diagonality(np.diag([3.0, 4.0, 5.0])) == 0.0
    del t


@pytest.mark.parametrize("variant", VARIANTS)
def test_total_error_energy(variant):
    val, tol = S[f"eps_total_{variant}"]
    assert abs(me.total_error_energy(mx.C_hat(variant, 8)) - val) <= tol
    # the exact DCT has zero error energy
    assert me.total_error_energy(mx.dct2_matrix(8)) < 1e-25


def test_coding_gain_dct_and_klt():
    v, tol = S["coding_gain_dct"]
    assert abs(me.coding_gain(mx.dct2_matrix(8), 0.95) - v) <= tol
    assert abs(me.coding_gain(mx.dct2_matrix(8), 0.95, "cols") - v) <= tol
    v, tol = S["coding_gain_klt"]
    assert abs(me.klt_coding_gain(8, 0.95) - v) <= tol
    # the unified formula on the KLT basis itself gives the KLT gain
    _, vecs = np.linalg.eigh(me.ar1_covariance(8, 0.95))
    assert abs(me.coding_gain(vecs.T, 0.95) - v) <= tol
    # identity transform: no gain
    assert abs(me.coding_gain(np.eye(8), 0.95)) < 1e-12


@pytest.mark.parametrize("variant", VARIANTS)
def test_coding_gain_approximations_below_klt(variant):
    """Parity unpinned by the paper (Fig. 3 is not available); only ordering checked."""
    cg = me.coding_gain(mx.C_hat(variant, 8), 0.95)
    assert 0.0 < cg < me.klt_coding_gain(8, 0.95)


# ---------------------------------------------------------------------------
# Tables 2 and 4: additive complexity; multiplierless entries
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n", (8, 16, 32))
def test_additive_complexity(variant, n):
    val, _ = S[f"adds_{variant}_{n}"]
    assert me.additive_complexity(variant, n) == int(val)
    # the stage list really is a factorization of T_N
    prod = None
    for s in me.stage_list(variant, n):
        prod = s if prod is None else prod @ s
    np.testing.assert_array_equal(prod, mx.T_N(variant, n))


def test_exact_chen_counts():
    """16 multiplications (non-trivial entries) and 26 additions in Eq. 3."""
    a, b, g = mx.chen_params_exact()
    facs = mx.chen_factors(a, b, g)
    adds = sum(me.stage_adds(f) for f in facs)

    def row_mults(row):
        # a common non-unit factor is applied once after the additions
        mags = {round(abs(v), 12) for v in row if abs(v) > 1e-12}
        nonunit = [m for m in mags if abs(m - 1.0) > 1e-12]
        if not nonunit:
            return 0
        return 1 if len(mags) == 1 else sum(1 for v in row if abs(abs(v) - 1) > 1e-12 and abs(v) > 1e-12)

    mults = sum(row_mults(row) for f in facs for row in np.asarray(f, dtype=float))
    assert adds == int(S["adds_exact_8"][0])
    assert mults == int(S["mults_exact_8"][0])


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n", (8, 16, 32))
def test_multiplierless_entries(variant, n):
    """T_N entries in {0, +-1, +-2}; every inverse factor in (1/2){0, +-1, +-2} (Sec. 6.1).

    The product T_N^{-1} itself has entries in {0, +-1/8, +-1/4} x 8/N, so only
    the factors are in the paper's set P (reading A5).
    """
    t = mx.T_N(variant, n)
    assert set(np.unique(t)) <= {-2, -1, 0, 1, 2}
    for f in me.stage_list(variant, n):
        inv = mx.exact_inverse(f)
        assert all(x * 2 in {-4, -2, -1, 0, 1, 2, 4} or x * 2 == 0 for row in inv for x in row)
        assert all((2 * x).denominator == 1 for row in inv for x in row)
    inv = mx.exact_inverse(t)
    assert {abs(x) * n for row in inv for x in row} <= {Fraction(0), Fraction(1), Fraction(2)}


# ---------------------------------------------------------------------------
# Sec. 6.1: JAM-scaled 16- and 32-point transforms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n", (16, 32))
def test_expanded_factorization_and_inverse(variant, n):
    """T_N = P M1 M2 M3 M4 B (expanded) and T_N^{-1} = (4/N) B^T M4^-1 M3^-1 M2^-1 M1^T P^T,
    with the inverse stages block-diagonal copies of the printed 8-point inverse factors."""
    p, m1, m2, m3, m4, b = mx.jam_factors(variant, n)
    np.testing.assert_array_equal(p @ m1 @ m2 @ m3 @ m4 @ b, mx.T_N(variant, n))
    if variant == "tilde":
        m3inv8 = [[x / 2 for x in row] for row in frac_of(G["M3_tilde"][0])]
    else:
        m3inv8 = frac_mat(*G["M3_hat_inv"])
    blocks = {"m2": frac_mat(*G[f"M2_{variant}_inv"]), "m3": m3inv8, "m4": frac_mat(*G["M4_inv"])}
    reps = n // 8
    for k in blocks:
        m = blocks[k]
        for _ in range(reps.bit_length() - 1):
            m = frac_block_diag(m, m)
        blocks[k] = m
    chain = [frac_of(b.T), blocks["m4"], blocks["m3"], blocks["m2"], frac_of(m1.T), frac_of(p.T)]
    inv = chain[0]
    for f in chain[1:]:
        inv = frac_matmul(inv, f)
    inv = [[x * Fraction(4, n) for x in row] for row in inv]
    assert [[x * n for x in row] for row in inv] == frac_of(mx.U_N(variant, n))


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n", (16, 32))
def test_jam_rows_follow_dct_frequencies(variant, n):
    """Reading of M^per: row k of C_N is near DCT-II row k (|cosine| > 0.5 for
    every row, > 0.7 on average); stacking the halves instead of interleaving
    them leaves most rows orthogonal to the DCT row of the same index."""
    c = mx.C_hat(variant, n)
    d = mx.dct2_matrix(n)
    cos = np.abs(np.sum(c * d, axis=1))
    assert cos.min() > 0.5 and cos.mean() > 0.7, cos
    wrong = np.vstack([c[0::2], c[1::2]])
    assert np.median(np.abs(np.sum(wrong * d, axis=1))) < 0.1


# ---------------------------------------------------------------------------
# Sec. 5.1: zig-zag, blocks, forward / zonal / inverse, PSNR
# ---------------------------------------------------------------------------

def test_zigzag_is_jpeg_order():
    pos = golden_io.grid("jpeg_zigzag_8x8.txt")
    order = pl.zigzag_order(8)
    for k, (i, j) in enumerate(order):
        assert pos[i, j] == k


@pytest.mark.parametrize("n", (4, 8, 16, 32))
def test_zigzag_properties(n):
    order = pl.zigzag_order(n)
    assert sorted(order) == [(i, j) for i in range(n) for j in range(n)]
    diag = [i + j for i, j in order]
    assert diag == sorted(diag)
    for (i0, j0), (i1, j1) in zip(order, order[1:]):
        if i0 + j0 == i1 + j1:          # within an anti-diagonal: unit diagonal step
            assert abs(i1 - i0) == 1 and abs(j1 - j0) == 1
    m = pl.zonal_mask(n, n * n // 4)
    assert m.sum() == n * n // 4


def test_blocks_roundtrip_and_padding():
    rng = np.random.default_rng(0)
    img = rng.integers(0, 256, size=(2, 13, 21))
    p = pl.pad_replicate(img, 8)
    assert p.shape == (2, 16, 24)
    np.testing.assert_array_equal(p[:, :13, :21], img)
    np.testing.assert_array_equal(p[:, 15, :21], img[:, 12])
    np.testing.assert_array_equal(p[:, :13, 23], img[:, :, 20])
    np.testing.assert_array_equal(pl.from_blocks(pl.to_blocks(p, 8)), p)
    b = pl.to_blocks(p, 8)
    np.testing.assert_array_equal(b[1, 1, 2], p[1, 8:16, 16:24])


def _brute_2d(a, left, right):
    """Four-index sum Y[k][l] = sum_ij left[k][i] a[i][j] right[j][l], pure Python."""
    n = len(a)
    return [[sum(left[k][i] * a[i][j] * right[j][l] for i in range(n) for j in range(n))
             for l in range(n)] for k in range(n)]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("conv", pl.CONVS)
def test_forward_inverse_brute_force_8(variant, conv):
    """Y and Z from the printed T_8 and the printed inverse chain by brute force."""
    rng = np.random.default_rng(7)
    a = rng.integers(-255, 256, size=(8, 8))
    t = G[f"T8_{variant}"][0]
    u = [[int(x * 8) for x in row] for row in _printed_inverse_chain_8(variant)]
    tl = t.tolist()
    right_f = u if conv == "paper" else t.T.tolist()
    y_bf = _brute_2d(a.tolist(), tl, right_f)
    y = pl.forward_blocks(a, mx.T8(variant), mx.U_N(variant, 8), conv)
    assert y.tolist() == y_bf
    ym = y * pl.zonal_mask(8, 10)
    right_i = tl if conv == "paper" else np.array(u).T.tolist()
    z_bf = _brute_2d(ym.tolist(), u, right_i)
    z = pl.inverse_blocks(ym, mx.T8(variant), mx.U_N(variant, 8), conv)
    assert z.tolist() == z_bf


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("conv", pl.CONVS)
@pytest.mark.parametrize("n", (8, 16, 32))
def test_perfect_reconstruction_all_coefficients(variant, conv, n):
    rng = np.random.default_rng(n)
    img = rng.integers(-255, 256, size=(2, 2 * n + 3, 3 * n - 5))
    res = pl.fzi_integer(img, n, variant, n * n, conv)
    np.testing.assert_array_equal(res["recon"], img.astype(np.float64))
    padded = pl.to_blocks(pl.pad_replicate(img, n), n)
    np.testing.assert_array_equal(res["z"], n * n * padded)
    assert all(math.isinf(p) for p in pl.psnr_integer_path(img, n, variant, n * n, conv))


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n", (8, 16, 32))
def test_dc_only_gives_block_means(variant, n):
    """r = 1: rows 1.. of T_N sum to zero and row 0 is all ones, so the
    reconstruction is the block mean (a closed form)."""
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, size=(2 * n, 2 * n))
    for conv in pl.CONVS:
        rec = pl.fzi_integer(img, n, variant, 1, conv)["recon"]
        means = img.reshape(2, n, 2, n).mean(axis=(1, 3))
        np.testing.assert_allclose(rec, np.kron(means, np.ones((n, n))), atol=1e-12)


def test_exact_dct_variant():
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, size=(16, 24)).astype(np.float64)
    np.testing.assert_allclose(pl.fzi_exact(img, 64)["recon"], img, atol=1e-10)
    rec1 = pl.fzi_exact(img, 1)["recon"]
    means = img.reshape(2, 8, 3, 8).mean(axis=(1, 3))
    np.testing.assert_allclose(rec1, np.kron(means, np.ones((8, 8))), atol=1e-10)
    # Parseval: orthonormal C keeps the block energy
    b = pl.fzi_exact(img, 64)["b"]
    blocks = pl.to_blocks(img, 8)
    np.testing.assert_allclose(np.sum(b * b), np.sum(blocks * blocks), rtol=1e-12)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n", (8, 16))
def test_paper_convention_against_float_similarity(variant, n):
    """B = C A C^{-1} and A' = C^{-1} Bm C computed in float64 with numpy's own
    inverse of C = S T agree with the integer route (S cancels)."""
    rng = np.random.default_rng(11)
    a = rng.integers(0, 256, size=(n, n))
    c = mx.C_hat(variant, n)
    cinv = np.linalg.inv(c)
    b = c @ a @ cinv
    y = pl.forward_blocks(a, mx.T_N(variant, n), mx.U_N(variant, n), "paper")
    s = mx.scale_S(mx.T_N(variant, n))
    np.testing.assert_allclose(pl.scaled_coeffs(y, s, n, "paper"), b, atol=1e-9)
    mask = pl.zonal_mask(n, n * n // 4)
    rec = cinv @ (b * mask) @ c
    res = pl.fzi_integer(a, n, variant, n * n // 4, "paper")
    np.testing.assert_allclose(res["recon"], rec, atol=1e-9)
    # transpose convention: B = C A C^T, A' = C^{-1} Bm C^{-T}
    bt = c @ a @ c.T
    yt = pl.forward_blocks(a, mx.T_N(variant, n), mx.U_N(variant, n), "transpose")
    np.testing.assert_allclose(pl.scaled_coeffs(yt, s, n, "transpose"), bt, atol=1e-9)
    rect = cinv @ (bt * mask) @ cinv.T
    np.testing.assert_allclose(pl.fzi_integer(a, n, variant, n * n // 4, "transpose")["recon"],
                               rect, atol=1e-9)


def test_psnr_exact_matches_float_and_closed_form():
    rng = np.random.default_rng(2)
    img = rng.integers(0, 256, size=(3, 40, 56))
    for n, variant, r in ((8, "hat", 6), (16, "tilde", 64), (32, "hat", 256)):
        res = pl.fzi_integer(img, n, variant, r)
        exact = pl.psnr_integer_path(img, n, variant, r)
        for b in range(3):
            assert abs(exact[b] - pl.psnr_float(img[b], res["recon"][b])) < 1e-9
    # closed form: a uniform error of 1 everywhere gives 20 log10(255)
    ref = np.zeros((8, 8))
    assert abs(pl.psnr_float(ref, ref + 1.0) - 20 * math.log10(255)) < 1e-12
    assert pl.psnr_from_sse(64 * 64 * 4, 8, 4) == pytest.approx(20 * math.log10(255), abs=1e-12)


def test_kept_coefficients_order():
    y = np.arange(64).reshape(8, 8)
    pos = golden_io.grid("jpeg_zigzag_8x8.txt")
    kept = pl.kept_coeffs(y, 8, 64)
    for k in range(64):
        i, j = np.argwhere(pos == k)[0]
        assert kept[k] == y[i, j]
