"""Autotuner of the fused kernel's pipeline schedule, with a JSON cache.

For a plan and a representative input it times each candidate schedule
(staging depth of the shared-memory input ring, resident CTAs per SM) with
CUDA events on the caller's stream, in ROUNDS interleaved rounds, and keeps
the candidate with the fastest median.  The kernel's default schedule is
kept unless another is faster by more than MARGIN: candidates that differ by
less than the timing noise would otherwise be picked at random from run to
run.  The choice is applied to the plan and recorded in a JSON cache keyed
by GPU name, N, variant, convention, pixel type and r.  The schedule never
changes results, only speed.  A missing, unreadable or corrupt cache file is
treated as empty (and rewritten), never as an error.
"""
from __future__ import annotations

import json
import os
import statistics
import tempfile

DEFAULT_CACHE = os.environ.get(
    "CDCT_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "cdct", "autotune.json"))

# (stages, ctas_per_sm): 0 = the kernel's default / as many CTAs as fit
CANDIDATES = ((0, 0), (1, 0), (2, 0), (3, 0), (0, 2), (0, 3))
DEFAULT = (0, 0)
ROUNDS = 3
MARGIN = 0.01


def choose(samples: dict, margin: float = MARGIN):
    """(stages, ctas_per_sm, median ms) from {(stages, ctas_per_sm): [ms, ...]}:
    the fastest median, unless the default schedule is within `margin` of it.
    Equal medians go to the smaller (stages, ctas_per_sm)."""
    med = {k: statistics.median(v) for k, v in samples.items() if v}
    best = min(med, key=lambda k: (med[k], k))
    if DEFAULT in med and med[DEFAULT] <= med[best] * (1.0 + margin):
        best = DEFAULT
    return best[0], best[1], med[best]


def cache_key(gpu: str, n: int, variant: str, conv: str, dtype: str, r: int) -> str:
    return f"{gpu}|N{n}|{variant}|{conv}|{dtype}|r{r}"


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    if not isinstance(data, dict):
        return {}
    good = {}
    for k, v in data.items():
        if (isinstance(k, str) and isinstance(v, dict) and isinstance(v.get("stages"), int)
                and isinstance(v.get("ctas_per_sm"), int) and v["stages"] in (0, 1, 2, 3)
                and 0 <= v["ctas_per_sm"] <= 32):
            good[k] = v
    return good


def save_cache(cache: dict, path: str = DEFAULT_CACHE) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(os.path.abspath(path)), suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_config(plan, img, r, stages, ctas, reps=5, warmup=2):
    import torch
    from . import binding
    plan.set_tuning(stages, ctas)
    ws = plan.workspace(img)
    out = torch.empty(img.shape, dtype=torch.float32, device=img.device)
    ps = torch.empty(img.shape[0] if img.dim() == 3 else 1, dtype=torch.float64, device=img.device)
    for _ in range(warmup):
        plan.fwd_zonal_inv(img, r, out=out, workspace=ws, psnr_out=ps)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        plan.fwd_zonal_inv(img, r, out=out, workspace=ws, psnr_out=ps)
    e.record()
    torch.cuda.synchronize()
    binding.check_device()
    return s.elapsed_time(e) / reps


def tune(plan, img, r, path: str = DEFAULT_CACHE, candidates=CANDIDATES, force=False):
    """Pick the fastest schedule for (plan, img's type, r); cached per GPU."""
    import torch
    dtype = "u8" if img.dtype == torch.uint8 else "i16"
    key = cache_key(torch.cuda.get_device_name(img.device), plan.n, plan.variant, plan.conv, dtype, r)
    cache = load_cache(path)
    if not force and key in cache:
        best = cache[key]
        plan.set_tuning(best["stages"], best["ctas_per_sm"])
        return best
    samples = {tuple(c): [] for c in candidates}
    for _ in range(ROUNDS):                 # interleaved, so that drift hits every candidate alike
        for st, ct in candidates:
            samples[(st, ct)].append(time_config(plan, img, r, st, ct))
    st, ct, ms = choose(samples)
    best = {"stages": st, "ctas_per_sm": ct, "ms": ms,
            "tried": [{"stages": a, "ctas_per_sm": b, "ms": statistics.median(t)} for (a, b), t in samples.items()]}
    plan.set_tuning(st, ct)
    cache[key] = best
    save_cache(cache, path)
    return best
