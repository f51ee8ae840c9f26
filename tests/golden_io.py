"""Readers for the text fixtures under tests/golden/ (values typed from the paper)."""
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for raw in f:
            s = raw.strip()
            if s and not s.startswith("#"):
                yield s


def matrices(name="paper_matrices.txt"):
    """{name: (int64 entries, Fraction scale)} from a 'matrix' fixture file."""
    out = {}
    it = iter(_lines(name))
    for head in it:
        parts = head.split()
        assert parts[0] == "matrix", head
        key, rows, cols = parts[1], int(parts[2]), int(parts[3])
        scale = Fraction(parts[5]) if len(parts) > 4 and parts[4] == "scale" else Fraction(1)
        data = [[int(x) for x in next(it).split()] for _ in range(rows)]
        arr = np.array(data, dtype=np.int64)
        assert arr.shape == (rows, cols), key
        out[key] = (arr, scale)
    return out


def scalars(name="paper_scalars.txt"):
    """{name: (value, tolerance)}; list-valued entries come back as tuples."""
    out = {}
    for s in _lines(name):
        key, val, tol = s.split()
        if "," in val:
            out[key] = (tuple(int(v) for v in val.split(",")), float(tol))
        else:
            out[key] = (float(val), float(tol))
    return out


def grid(name):
    return np.array([[int(x) for x in s.split()] for s in _lines(name)], dtype=np.int64)
