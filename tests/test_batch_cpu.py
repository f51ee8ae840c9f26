"""Descriptor-table batches and the autotune cache, without a GPU.

Batch creation validates the host descriptor list before anything touches
the device: each invalid descriptor is refused with CDCT_EINVAL naming the
image.  The pointers below are never dereferenced.
"""
import ctypes
import json

import pytest

from paper_2207_11638_gb300 import autotune
from paper_2207_11638_gb300 import binding as b

FAKE = 0x10000000


def descs(items):
    arr = (b.CdctBatchImage * len(items))()
    for i, (d, o, w, h, p, rp) in enumerate(items):
        arr[i] = b.CdctBatchImage(d, o, w, h, p, rp)
    return arr


def create(plan, items, dtype=0):
    h = ctypes.c_void_p()
    st = b.lib().cdct_batch_create(plan.handle, descs(items), len(items), dtype, ctypes.byref(h))
    return st, h


def test_valid_batch_sizes():
    plan = b.Plan(8, "hat")
    items = [(FAKE, FAKE, 64, 40, 64, 64), (FAKE + 4096, FAKE + 8192, 1040, 9, 1040, 1040)]
    st, h = create(plan, items)
    assert st == b.CDCT_OK
    tb, wb, px = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int64()
    assert b.lib().cdct_batch_sizes(h, ctypes.byref(tb), ctypes.byref(wb), ctypes.byref(px)) == 0
    # units: image 0 is 8 blocks wide (at most half of a 128-block unit), so its
    # 5 block rows pack into one unit of up to 128 / 8 = 16 rows; image 1:
    # 2 block rows x ceil(130 / 128) = 4 units
    assert wb.value == (1 + 4) * 4 * 8
    assert px.value == 64 * 40 + 1040 * 9
    # table: 2 descriptors (80 B), 3 prefix sums (24 B) padded to 112 B, then
    # one 64-byte record per work unit
    assert ctypes.sizeof(b.CdctBatchImage) == 40
    assert tb.value == 112 + (1 + 4) * 64
    assert b.lib().cdct_batch_destroy(h) == 0


@pytest.mark.parametrize("bad,msg", [
    ((0, FAKE, 64, 8, 64, 64), b"null pointer"),
    ((FAKE, 0, 64, 8, 64, 64), b"null pointer"),
    ((FAKE, FAKE, 0, 8, 64, 64), b"width and height"),
    ((FAKE, FAKE, 64, 8, 32, 64), b"pitch < width"),
    ((FAKE + 8, FAKE, 64, 8, 64, 64), b"16-byte aligned"),
    ((FAKE, FAKE, 40, 8, 40, 40), b"16-byte aligned"),     # u8 width not a multiple of 16
    ((FAKE, FAKE, 64, 8, 64, 66), b"16-byte aligned"),     # recon pitch not a multiple of 4 floats
])
def test_invalid_descriptor_rejected(bad, msg):
    plan = b.Plan(16, "tilde")
    good = (FAKE, FAKE, 64, 8, 64, 64)
    st, h = create(plan, [good, good, bad])
    assert st == b.CDCT_EINVAL and h.value is None
    err = b.lib().cdct_last_error()
    assert b"batch image 2" in err and msg in err


def test_batch_argument_checks():
    lib = b.lib()
    h = ctypes.c_void_p()
    assert lib.cdct_batch_create(b.Plan(8, "exact").handle, descs([(FAKE, FAKE, 64, 8, 64, 64)]), 1, 0,
                                 ctypes.byref(h)) == b.CDCT_EUNSUPPORTED
    assert lib.cdct_batch_create(b.Plan(8, "hat").handle, descs([(FAKE, FAKE, 64, 8, 64, 64)]), 0, 0,
                                 ctypes.byref(h)) == b.CDCT_EINVAL
    plan = b.Plan(8, "hat")
    assert lib.cdct_plan_set_tuning(plan.handle, 5, 0) == b.CDCT_EINVAL
    assert lib.cdct_plan_set_tuning(plan.handle, 3, -1) == b.CDCT_EINVAL
    assert lib.cdct_plan_set_tuning(plan.handle, 3, 2) == b.CDCT_OK
    st, hb = create(plan, [(FAKE, FAKE, 64, 8, 64, 64)])
    assert st == 0
    # r out of range and missing workspace are refused before any launch
    assert lib.cdct_batch_fzi(hb, ctypes.c_void_p(FAKE), 0, None, None, 0, None) == b.CDCT_EINVAL
    assert lib.cdct_batch_fzi(hb, ctypes.c_void_p(FAKE), 6, ctypes.c_void_p(FAKE), None, 0, None) == b.CDCT_EINVAL
    lib.cdct_batch_destroy(hb)


def test_autotune_cache_roundtrip_and_corruption(tmp_path):
    path = str(tmp_path / "tune.json")
    assert autotune.load_cache(path) == {}                      # missing
    open(path, "w").write("{ not json")
    assert autotune.load_cache(path) == {}                      # corrupt
    open(path, "w").write(json.dumps([1, 2, 3]))
    assert autotune.load_cache(path) == {}                      # wrong shape
    key = autotune.cache_key("GPU", 16, "hat", "paper", "i16", 64)
    bad = autotune.cache_key("GPU", 8, "hat", "paper", "i16", 16)
    open(path, "w").write(json.dumps({key: {"stages": 3, "ctas_per_sm": 2, "ms": 1.0},
                                      bad: {"stages": 7, "ctas_per_sm": 2}}))
    cache = autotune.load_cache(path)
    assert list(cache) == [key]                                  # invalid entries dropped
    cache[bad] = {"stages": 2, "ctas_per_sm": 0, "ms": 2.0}
    autotune.save_cache(cache, path)
    assert autotune.load_cache(path) == cache


def batch_unit(h, u):
    out = (ctypes.c_int32 * 4)()
    st = b.lib().cdct_batch_unit(h, u, out)
    return st, tuple(out)


@pytest.mark.parametrize("n", (8, 16, 32))
def test_unit_records_follow_the_packing_rule(n):
    """The host expands a batch into one record per work unit: an image at
    most half a unit wide (nbx <= S / 2, S = 128 / P blocks) packs S / nbx
    whole block rows per unit (the last unit keeps the remainder); any other
    image has one unit per block row and segment of S blocks, row-major."""
    plan = b.Plan(n, "hat")
    S = {8: 128, 16: 32, 32: 8}[n]
    dims = [(64, 40), (1040, 9), (16, 200), (2048, 33), (n * S // 2, 70), (n * S // 2 + 16, 3), (512, 512)]
    items = [(FAKE + 65536 * i, FAKE + 65536 * i, w, h, w, w) for i, (w, h) in enumerate(dims)]
    st, h = create(plan, items)
    assert st == b.CDCT_OK
    want = []
    for i, (w, hh) in enumerate(dims):
        nbx, nby = -(-w // n), -(-hh // n)
        if nbx <= S // 2:
            k = S // nbx
            want += [(i, by, 0, min(k, nby - by)) for by in range(0, nby, k)]
        else:
            want += [(i, by, seg, 1) for by in range(nby) for seg in range(-(-nbx // S))]
    tb, wb, px = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int64()
    assert b.lib().cdct_batch_sizes(h, ctypes.byref(tb), ctypes.byref(wb), ctypes.byref(px)) == 0
    assert wb.value == len(want) * 4 * 8
    got = []
    for u in range(len(want)):
        st, rec = batch_unit(h, u)
        assert st == b.CDCT_OK
        got.append(rec)
    assert got == want
    assert batch_unit(h, len(want))[0] == b.CDCT_EINVAL
    assert batch_unit(h, -1)[0] == b.CDCT_EINVAL
    assert b.lib().cdct_batch_destroy(h) == 0


def test_autotune_choice_keeps_the_default_within_the_noise():
    near = {(0, 0): [1.00, 1.006, 1.005], (2, 0): [0.998, 1.0, 0.997], (0, 3): [1.3, 1.2, 1.25]}
    assert autotune.choose(near)[:2] == (0, 0)          # 0.998 vs 1.005: within 1 %
    clear = {(0, 0): [1.035, 1.04, 1.03], (2, 0): [1.0, 0.99, 1.01], (1, 0): [1.02, 1.0, 1.03]}
    st, ct, ms = autotune.choose(clear)
    assert (st, ct) == (2, 0) and ms == 1.0              # median, not the best single sample
    tie = {(3, 0): [1.0], (2, 0): [1.0]}
    assert autotune.choose(tie)[:2] == (2, 0)            # no default among them: the smaller key
