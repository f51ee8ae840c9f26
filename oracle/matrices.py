"""Transform matrices of the paper, built from their definitions.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Every matrix is written as the paper defines it and multiplied out with
plain matrix products; nothing is factored into butterflies.  Integer
matrices are ``numpy.int64``; exact inverses use ``fractions.Fraction``.

Readings of the paper taken here (each listed in the design notes):

* Sec. 3 prints round(alpha, beta, gamma) as [1 1 0 1 1 1 0]; the entry that
  rounds to zero is beta_3 = cos(7 pi/16) = 0.195, not beta_1.  The printed
  M^_2 and T^_8 follow (1, 1,1,1,0, 1,0), which is what ``round_params``
  yields by applying the paper's round() to the exact constants.
* Sec. 6: M^per_N is printed in a garbled block form; it is read as the
  even/odd interleave (output row 2k <- row k of the upper half, output row
  2k+1 <- row k of the lower half).
* Eq. app_N (Sec. 6.1) drops the 1/sqrt(2) of the JAM recursion; T_N is kept
  integer, as printed.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

VARIANTS = ("tilde", "hat")


# ---------------------------------------------------------------------------
# Sec. 2: elementary matrices
# ---------------------------------------------------------------------------

def identity(n: int) -> np.ndarray:
    """I_n."""
    return np.eye(n, dtype=np.int64)


def counter_identity(n: int) -> np.ndarray:
    """Counter-identity I-bar_n (Sec. 2): ones on the anti-diagonal."""
    return np.fliplr(np.eye(n, dtype=np.int64))


def block_diag(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """[[a, 0], [0, b]] for square a, b."""
    n, m = a.shape[0], b.shape[0]
    out = np.zeros((n + m, n + m), dtype=np.result_type(a, b))
    out[:n, :n] = a
    out[n:, n:] = b
    return out


def dct2_matrix(n: int) -> np.ndarray:
    """C_N^II, Sec. 2: sqrt(2/N) c_m cos(m (2n+1) pi / (2N)), c_0 = 1/sqrt 2."""
    out = np.zeros((n, n), dtype=np.float64)
    for m in range(n):
        cm = 1.0 / math.sqrt(2.0) if m == 0 else 1.0
        for k in range(n):
            out[m, k] = math.sqrt(2.0 / n) * cm * math.cos(m * (2 * k + 1) * math.pi / (2 * n))
    return out


def dct4_matrix(n: int) -> np.ndarray:
    """C_N^IV, Sec. 2: sqrt(2/N) cos((2m+1)(2n+1) pi / (4N))."""
    out = np.zeros((n, n), dtype=np.float64)
    for m in range(n):
        for k in range(n):
            out[m, k] = math.sqrt(2.0 / n) * math.cos((2 * m + 1) * (2 * k + 1) * math.pi / (4 * n))
    return out


# ---------------------------------------------------------------------------
# Eq. 1 (Wang) and Eq. 2 (Chen): fixed matrices and parametric ones
# ---------------------------------------------------------------------------

def perm_from_rows(cols) -> np.ndarray:
    """Permutation matrix whose row i has its single one in column cols[i]."""
    n = len(cols)
    out = np.zeros((n, n), dtype=np.int64)
    for i, c in enumerate(cols):
        out[i, c] = 1
    return out


def P8() -> np.ndarray:
    """P_8 of Eq. 1 (row i has a one in the listed column)."""
    return perm_from_rows([0, 7, 1, 6, 2, 5, 3, 4])


def B8() -> np.ndarray:
    """B_8 = [[I_4, I-bar_4], [I-bar_4, -I_4]] of Eq. 1."""
    i4, j4 = identity(4), counter_identity(4)
    return np.block([[i4, j4], [j4, -i4]])


def Q4() -> np.ndarray:
    """Q of Eq. 2 (swaps the middle two entries)."""
    return perm_from_rows([0, 2, 1, 3])


def A1(beta) -> np.ndarray:
    """A_1(beta) of Eq. 2."""
    b0, b1, b2, b3 = beta
    return np.array([[b0, 0, 0, b3],
                     [0, b2, b1, 0],
                     [0, b1, -b2, 0],
                     [b3, 0, 0, -b0]], dtype=_dtype_of(beta))


def A2() -> np.ndarray:
    """A_2 of Eq. 2."""
    return np.array([[1, 1, 0, 0],
                     [1, -1, 0, 0],
                     [0, 0, -1, 1],
                     [0, 0, 1, 1]], dtype=np.int64)


def A3(alpha) -> np.ndarray:
    """A_3(alpha) of Eq. 2."""
    a = alpha
    return np.array([[0, 0, 0, 1],
                     [0, a, a, 0],
                     [0, -a, a, 0],
                     [1, 0, 0, 0]], dtype=_dtype_of([alpha]))


def P4() -> np.ndarray:
    """P_4 of Eq. 3."""
    return perm_from_rows([0, 3, 1, 2])


def B4() -> np.ndarray:
    """B_4 = [[I_2, I-bar_2], [I-bar_2, -I_2]] of Eq. 3."""
    i2, j2 = identity(2), counter_identity(2)
    return np.block([[i2, j2], [j2, -i2]])


def Ctilde(alpha, gamma) -> np.ndarray:
    """C-tilde(alpha, gamma) of Eq. 3 (the 4x4 block inside M_3)."""
    a = alpha
    g0, g1 = gamma
    return np.array([[a, a, 0, 0],
                     [a, -a, 0, 0],
                     [0, 0, -g0, g1],
                     [0, 0, g1, g0]], dtype=_dtype_of([alpha, g0, g1]))


def M1() -> np.ndarray:
    """M_1 = diag(I_4, I-bar_4 Q) of Eq. 3."""
    return block_diag(identity(4), counter_identity(4) @ Q4())


def M2(beta) -> np.ndarray:
    """M_2(beta) = diag(P_4, A_1(beta)) of Eq. 3."""
    return block_diag(P4(), A1(beta))


def M3(alpha, gamma) -> np.ndarray:
    """M_3(alpha, gamma) = diag(C-tilde, A_2) of Eq. 3."""
    return block_diag(Ctilde(alpha, gamma), A2())


def M4(alpha) -> np.ndarray:
    """M_4(alpha) = diag(B_4, A_3(alpha)) of Eq. 3."""
    return block_diag(B4(), A3(alpha))


def _dtype_of(vals):
    return np.int64 if all(float(v).is_integer() for v in vals) else np.float64


# ---------------------------------------------------------------------------
# Sec. 3: the parametric map T_C and its two approximations
# ---------------------------------------------------------------------------

def chen_params_exact():
    """(alpha, beta, gamma) of the exact Chen factorization (Sec. 3)."""
    alpha = math.cos(math.pi / 4)
    beta = [math.cos((2 * n + 1) * math.pi / 16) for n in range(4)]
    gamma = [math.cos((2 * n + 1) * math.pi / 8) for n in range(2)]
    return alpha, beta, gamma


def paper_sign(x: float) -> int:
    """sign(x) of Sec. 3: 1, 0, -1."""
    return 1 if x > 0 else (-1 if x < 0 else 0)


def paper_round(x: float) -> int:
    """round(x) = sign(x) floor(|x| + 1/2) of Sec. 3 (half away from zero)."""
    return paper_sign(x) * math.floor(abs(x) + 0.5)


def sign_params():
    """(alpha~, beta~, gamma~) = sign of the exact constants (Sec. 3)."""
    a, b, g = chen_params_exact()
    return paper_sign(a), [paper_sign(v) for v in b], [paper_sign(v) for v in g]


def round_params():
    """(alpha^, beta^, gamma^) = round of the exact constants (Sec. 3)."""
    a, b, g = chen_params_exact()
    return paper_round(a), [paper_round(v) for v in b], [paper_round(v) for v in g]


def params(variant: str):
    if variant == "tilde":
        return sign_params()
    if variant == "hat":
        return round_params()
    raise ValueError(variant)


def chen_factors(alpha, beta, gamma):
    """The factor list [P_8, M_1, M_2, M_3, M_4, B_8] of the map T_C (Sec. 3)."""
    return [P8(), M1(), M2(beta), M3(alpha, gamma), M4(alpha), B8()]


def T_C(alpha, beta, gamma) -> np.ndarray:
    """T_C(alpha, beta, gamma) = P_8 M_1 M_2 M_3 M_4 B_8 (Sec. 3)."""
    out = None
    for f in chen_factors(alpha, beta, gamma):
        out = f if out is None else out @ f
    return out


def T8(variant: str) -> np.ndarray:
    """T~_8 (Eq. 4) or T^_8 (Eq. 5) as an int64 matrix."""
    a, b, g = params(variant)
    t = T_C(a, b, g)
    assert t.dtype == np.int64
    return t


# ---------------------------------------------------------------------------
# Sec. 6 / 6.1: JAM recursion for N > 8
# ---------------------------------------------------------------------------

def M_add(n: int) -> np.ndarray:
    """M^add_N = [[I_{N/2}, I-bar_{N/2}], [I-bar_{N/2}, -I_{N/2}]] (Sec. 6)."""
    h = n // 2
    i, j = identity(h), counter_identity(h)
    return np.block([[i, j], [j, -i]])


def M_per(n: int) -> np.ndarray:
    """M^per_N read as the even/odd interleave (Sec. 6).

    Column k (k < N/2) of the upper half goes to row 2k and column N/2 + k of
    the lower half goes to row 2k + 1.
    """
    h = n // 2
    out = np.zeros((n, n), dtype=np.int64)
    for k in range(h):
        out[2 * k, k] = 1
        out[2 * k + 1, h + k] = 1
    return out


def T_N(variant: str, n: int) -> np.ndarray:
    """T_N of Eq. app_N: M^per_N diag(T_{N/2}, T_{N/2}) M^add_N, T_8 at the base."""
    if n == 8:
        return T8(variant)
    if n < 8 or n & (n - 1):
        raise ValueError("N must be a power of two >= 8")
    half = T_N(variant, n // 2)
    return M_per(n) @ block_diag(half, half) @ M_add(n)


def jam_factors(variant: str, n: int):
    """Stage matrices of Eqs. transformation_N_sign / _round (Sec. 6.1).

    Returns [P-check_N, M^(1)_N, M^(2)_N, M^(3)_N, M^(4)_N, B-check_N]; at
    N = 8 these are [P_8, M_1, M_2, M_3, M_4, B_8] of Eqs. 4-5.
    """
    if n == 8:
        a, b, g = params(variant)
        return chen_factors(a, b, g)
    p, m1, m2, m3, m4, b = jam_factors(variant, n // 2)
    return [M_per(n) @ block_diag(p, p),
            block_diag(m1, m1), block_diag(m2, m2), block_diag(m3, m3), block_diag(m4, m4),
            block_diag(b, b) @ M_add(n)]


# ---------------------------------------------------------------------------
# Exact inverses, U_N = N T_N^{-1}, scale S_N
# ---------------------------------------------------------------------------

def exact_inverse(m: np.ndarray):
    """Exact inverse of an integer matrix by Gauss-Jordan over the rationals.

    Returns a list of lists of ``Fraction``.
    """
    n = m.shape[0]
    a = [[Fraction(int(m[i, j])) for j in range(n)] + [Fraction(int(i == j)) for j in range(n)]
         for i in range(n)]
    for col in range(n):
        piv = next(r for r in range(col, n) if a[r][col] != 0)
        a[col], a[piv] = a[piv], a[col]
        pv = a[col][col]
        a[col] = [x / pv for x in a[col]]
        for r in range(n):
            if r != col and a[r][col] != 0:
                f = a[r][col]
                a[r] = [x - f * y for x, y in zip(a[r], a[col])]
    return [row[n:] for row in a]


def U_N(variant: str, n: int) -> np.ndarray:
    """U_N = N T_N^{-1}, checked to be an integer matrix (int64)."""
    inv = exact_inverse(T_N(variant, n))
    out = np.zeros((n, n), dtype=np.int64)
    for i in range(n):
        for j in range(n):
            v = inv[i][j] * n
            if v.denominator != 1:
                raise AssertionError("N T_N^-1 is not integral")
            out[i, j] = int(v)
    return out


def scale_S(t: np.ndarray) -> np.ndarray:
    """Diagonal of S' = sqrt(diag(T T^T)^{-1}) (Sec. 3.1, and S_N of Sec. 6.1)."""
    d = np.diag(t.astype(np.int64) @ t.astype(np.int64).T).astype(np.float64)
    return 1.0 / np.sqrt(d)


def C_hat(variant: str, n: int) -> np.ndarray:
    """Near-orthogonal approximation C = S T (float64), Sec. 3.1 / 6.1."""
    t = T_N(variant, n)
    return scale_S(t)[:, None] * t.astype(np.float64)
