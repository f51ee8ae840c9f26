"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no transform arithmetic; it only draws images.  Both the
CUDA path (tests, bench) and the CPU oracle consume what it returns.

The image model is the first-order Markov (AR(1)) process the paper uses for
its coding-gain analysis (Sec. 4.1), extended separably to two dimensions:
a unit-variance field with correlation rho^|dy| rho^|dx|, mapped to mean 128
and standard deviation 40, rounded half up and clipped to [0, 255].  The
paper's own test images (30 standard 512x512 pictures, Sec. 5.1) and video
sequences (Sec. 6.2) are not available; these fields stand in for them.

Generation is on the host with NumPy's PCG64, so it is reproducible across
machines.
"""
from __future__ import annotations

import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np
from scipy.signal import lfilter

MEAN, STD = 128.0, 40.0


def _ar1_along(x: np.ndarray, rho: float, axis: int) -> np.ndarray:
    """Stationary AR(1) filter along ``axis``: y0 = x0, y_n = rho y_{n-1} + sqrt(1-rho^2) x_n."""
    c = math.sqrt(1.0 - rho * rho)
    first = np.take(x, [0], axis=axis)
    return lfilter([c], [1.0, -rho], x, axis=axis, zi=(1.0 - c) * first)[0]


def ar1_field(h: int, w: int, rho: float, rng: np.random.Generator) -> np.ndarray:
    """Unit-variance separable 2-D AR(1) Gaussian field, float64 [h, w]."""
    eps = rng.standard_normal((h, w))
    return _ar1_along(_ar1_along(eps, rho, axis=1), rho, axis=0)


def to_u8(z: np.ndarray) -> np.ndarray:
    return np.clip(np.floor(MEAN + STD * z + 0.5), 0, 255).astype(np.uint8)


def ar1_image(h: int, w: int, rho: float = 0.95, seed: int = 1) -> np.ndarray:
    """One uint8 AR(1) image (the 512x512, rho = 0.95 still-image workload)."""
    return to_u8(ar1_field(h, w, rho, np.random.Generator(np.random.PCG64(seed))))


def ar1_frame_420(h: int, w: int, rho: float, seed: int):
    """A 4:2:0 frame: luma [h, w] and two chroma planes [h/2, w/2], uint8."""
    rng = np.random.Generator(np.random.PCG64(seed))
    y = to_u8(ar1_field(h, w, rho, rng))
    u = to_u8(ar1_field(h // 2, w // 2, rho, rng))
    v = to_u8(ar1_field(h // 2, w // 2, rho, rng))
    return y, u, v


def frame_rhos(n_frames: int, seed: int, lo: float = 0.90, hi: float = 0.97) -> np.ndarray:
    """Per-frame correlation drawn uniformly from [lo, hi]."""
    return np.random.Generator(np.random.PCG64(seed)).uniform(lo, hi, size=n_frames)


def residual_frames_420(n_frames: int = 64, h: int = 1080, w: int = 1920, seed: int = 2,
                        threads: int = 8):
    """int16 residual batch: frame A (seed 2f) minus frame B (seed 2f + 1).

    Frame f uses rho_f ~ U[0.90, 0.97] for both A and B.  Returns
    (luma [F, h, w], chroma [2F, h/2, w/2]) with chroma ordered U_0, V_0,
    U_1, V_1, ...; values lie in [-255, 255].
    """
    rhos = frame_rhos(n_frames, seed)
    luma = np.empty((n_frames, h, w), dtype=np.int16)
    chroma = np.empty((2 * n_frames, h // 2, w // 2), dtype=np.int16)

    def one(f):
        a = ar1_frame_420(h, w, float(rhos[f]), seed * 1_000_003 + 2 * f)
        b = ar1_frame_420(h, w, float(rhos[f]), seed * 1_000_003 + 2 * f + 1)
        luma[f] = a[0].astype(np.int16) - b[0].astype(np.int16)
        chroma[2 * f] = a[1].astype(np.int16) - b[1].astype(np.int16)
        chroma[2 * f + 1] = a[2].astype(np.int16) - b[2].astype(np.int16)

    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, range(n_frames)))
    return luma, chroma


def uneven_sizes(n_images: int = 4096, seed: int = 3, lo: int = 64, hi: int = 2048,
                 multiple: int = 32):
    """Image sizes (h, w) log-uniform in [lo, hi], rounded to a multiple, and rho per image."""
    rng = np.random.Generator(np.random.PCG64(seed))
    logs = rng.uniform(math.log(lo), math.log(hi), size=(n_images, 2))
    sides = np.clip(np.round(np.exp(logs) / multiple) * multiple, lo, hi).astype(np.int64)
    rhos = rng.uniform(0.85, 0.97, size=n_images)
    return sides[:, 0], sides[:, 1], rhos


def residual_regions_32(n_regions: int, seed: int = 4, side: int = 512):
    """int16 32x32 residual regions: differences of pairs of AR(1) 512^2 images
    (rho = 0.95), each pair cut into (side/32)^2 regions; [n, 32, 32]."""
    per = (side // 32) ** 2
    n_pairs = -(-n_regions // per)
    out = np.empty((n_pairs * per, 32, 32), dtype=np.int16)
    for p in range(n_pairs):
        a = ar1_image(side, side, 0.95, seed * 1_000_003 + 2 * p).astype(np.int16)
        b = ar1_image(side, side, 0.95, seed * 1_000_003 + 2 * p + 1).astype(np.int16)
        d = (a - b).reshape(side // 32, 32, side // 32, 32).swapaxes(1, 2).reshape(per, 32, 32)
        out[p * per:(p + 1) * per] = d
    return out[:n_regions]


# Parameter tensors of the CNN size selector in the order of the library's
# flat float32 vector (include/cdct.h): (name, element count, fan-in).
CNN_LAYOUT = (("W1", 16 * 9, 9), ("b1", 16, 0), ("W2", 32 * 144, 144), ("b2", 32, 0),
              ("W3", 32 * 288, 288), ("b3", 32, 0), ("Wf1", 64 * 512, 512), ("Wq", 64 * 4, 512),
              ("bf1", 64, 0), ("Wf2", 17 * 64, 64), ("bf2", 17, 0))


def cnn_init_params(seed: int = 0, bias_std: float = 0.0) -> np.ndarray:
    """Seeded He-normal weights (std sqrt(2 / fan-in)) and N(0, bias_std) biases,
    as the flat float32 vector of the CNN size selector."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for _, n, fan_in in CNN_LAYOUT:
        if fan_in:
            parts.append(rng.standard_normal(n) * math.sqrt(2.0 / fan_in))
        else:
            parts.append(rng.standard_normal(n) * bias_std)
    return np.concatenate(parts).astype(np.float32)
