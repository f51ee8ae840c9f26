"""Host side of the rate-distortion search: the library's tables against the
oracle's exact values, and argument checks that fail before any launch."""
import ctypes

import pytest

from oracle import rd
from paper_2207_11638_gb300 import binding as b


@pytest.mark.parametrize("variant", ("tilde", "hat"))
def test_rd_tables_equal_oracle(variant):
    d, c = b.RdSearch(variant).tables()
    for n in rd.SIZES:
        assert d[n] == rd.row_norms2(variant, n)
        assert c[n] == rd.dequant_scale(variant, n)


def _img(width=64, height=64, batch=1):
    return b.CdctImage(0x200000, 1, width, height, width, batch, width * height)


def test_rd_argument_checks_reject_before_launch():
    lib = b.lib()
    h = ctypes.c_void_p()
    assert lib.cdct_rd_create(0, ctypes.byref(h)) == b.CDCT_EINVAL          # exact DCT: no search
    assert lib.cdct_rd_create(2, None) == b.CDCT_EINVAL
    s = b.RdSearch("hat")
    d = _img()
    n = ctypes.c_int64()
    assert lib.cdct_rd_region_count(ctypes.byref(d), ctypes.byref(n)) == 0 and n.value == 4
    d2 = _img(65, 33, 3)
    assert lib.cdct_rd_region_count(ctypes.byref(d2), ctypes.byref(n)) == 0 and n.value == 3 * 3 * 2
    q = (ctypes.c_int32 * 5)(8, 16, 32, 64, 128)
    lab = ctypes.c_void_p(0x300000)
    call = lambda **k: lib.cdct_rd_search(k.get("h", s._h), ctypes.byref(k.get("d", d)), k.get("q", q),
                                          k.get("nq", 3), k.get("kn", 1), k.get("kd", 2), k.get("lab", lab),
                                          None, None)
    assert call(nq=0) == b.CDCT_EINVAL
    assert call(nq=5) == b.CDCT_EINVAL
    assert call(q=(ctypes.c_int32 * 1)(0), nq=1) == b.CDCT_EINVAL
    assert call(q=(ctypes.c_int32 * 1)(4097), nq=1) == b.CDCT_EINVAL
    assert call(kn=-1) == b.CDCT_EINVAL
    assert call(kn=1025) == b.CDCT_EINVAL
    assert call(kd=45) == b.CDCT_EINVAL
    assert call(lab=None) == b.CDCT_EINVAL
    assert call(h=None) == b.CDCT_EINVAL
    bad = _img()
    bad.dtype = 7
    assert call(d=bad) == b.CDCT_EINVAL
    assert b"dtype" in lib.cdct_last_error()
