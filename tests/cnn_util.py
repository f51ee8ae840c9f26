"""Test helper: the library's flat CNN parameter vector as the oracle's tensors."""
import numpy as np

from oracle import cnn


def to_oracle(flat) -> dict:
    flat = np.asarray(flat, dtype=np.float64)
    out, off = {}, 0
    for name, shape in cnn.PARAM_SHAPES:
        n = int(np.prod(shape))
        out[name] = flat[off:off + n].reshape(shape).copy()
        off += n
    assert off == flat.size
    return out


def from_oracle(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in cnn.PARAM_SHAPES])
