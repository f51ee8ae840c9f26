"""Write the generated reports of Sec. 4.1: the coding gain relative to the
KLT over the correlation coefficient (the curves of Fig. 3), and the total
error energy table.  Every number comes from ``oracle/`` alone.

    python -m tests.golden.make_reports          # rewrites the two report files

Fig. 3 itself is not in the paper's text (the image is missing), so the
curves are the paper's definitions evaluated, not a transcription.  They
cover the exact DCT and the two approximations C^ = S T^ and C~ = S T~ of
Sec. 3.1, for N = 8 and, through the JAM recursion of Sec. 6.1, N = 16 and 32
(the paper plots N = 8 only).  The comparison transforms of Fig. 3 (HT, WHT,
SDCT, BAS) are not part of this build.  The synthesis basis g_k is read as
row k of C^-1, as Sec. 4.1 prints it; the column reading is reported beside
it.
"""
from __future__ import annotations

import os

from oracle import matrices as mx
from oracle import metrics as me

HERE = os.path.dirname(os.path.abspath(__file__))
CODING_GAIN_FILE = os.path.join(HERE, "report_coding_gain.txt")
EPS_FILE = os.path.join(HERE, "report_eps_total.txt")

RHOS = tuple(round(0.05 * k, 2) for k in range(20)) + (0.99,)   # 0 <= rho < 1
SIZES = (8, 16, 32)


def transforms(n):
    """(name, matrix) of the transforms the curves compare at size n."""
    return (("dct", mx.dct2_matrix(n)), ("hat", mx.C_hat("hat", n)), ("tilde", mx.C_hat("tilde", n)))


def coding_gain_rows():
    """[(n, rho, klt, {name: (rows, cols)})]: C_g(transform) - C_g(KLT) in dB."""
    out = []
    for n in SIZES:
        mats = transforms(n)
        for rho in RHOS:
            klt = me.klt_coding_gain(n, rho)
            rel = {name: (me.coding_gain(c, rho, "rows") - klt, me.coding_gain(c, rho, "cols") - klt)
                   for name, c in mats}
            out.append((n, rho, klt, rel))
    return out


def eps_rows():
    """[(n, variant, epsilon_total, delta)] for the approximations of Secs. 3.1 and 6.1."""
    out = []
    for n in SIZES:
        for v in ("hat", "tilde"):
            t = mx.T_N(v, n)
            out.append((n, v, me.total_error_energy(mx.C_hat(v, n)),
                        me.deviation_from_diagonality(t.astype(float) @ t.T.astype(float))))
    return out


def format_coding_gain(rows) -> str:
    lines = ["# Coding gain relative to the KLT, C_g(C) - C_g(KLT) in dB (Sec. 4.1, Fig. 3).",
             "# AR(1) model R_x = rho^|m-n|.  C_g(KLT) in dB, then per transform the row and the",
             "# column reading of the synthesis basis.  Written by tests/golden/make_reports.py.",
             "# n rho klt dct_rows dct_cols hat_rows hat_cols tilde_rows tilde_cols"]
    for n, rho, klt, rel in rows:
        vals = [klt] + [x for name in ("dct", "hat", "tilde") for x in rel[name]]
        lines.append(f"{n} {rho:.2f} " + " ".join(f"{x:.10f}" for x in vals))
    return "\n".join(lines) + "\n"


def format_eps(rows) -> str:
    lines = ["# Total error energy epsilon_total = pi ||C - C_approx||_F^2 against the exact DCT",
             "# (Sec. 4.1) and the deviation from diagonality delta of T T^T (Sec. 3.1), for",
             "# C_approx = S T, N = 8 (printed in the paper) and 16, 32 (JAM recursion, Sec. 6.1).",
             "# Written by tests/golden/make_reports.py.",
             "# n variant eps_total delta"]
    for n, v, eps, delta in rows:
        lines.append(f"{n} {v} {eps:.10f} {delta:.10f}")
    return "\n".join(lines) + "\n"


def parse(path):
    rows = []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append(line.split())
    return rows


def main():
    with open(CODING_GAIN_FILE, "w") as f:
        f.write(format_coding_gain(coding_gain_rows()))
    with open(EPS_FILE, "w") as f:
        f.write(format_eps(eps_rows()))


if __name__ == "__main__":
    main()
