"""The C-ABI library without a GPU: it loads, exports every declared symbol,
its host-side matrices (the kernels' own butterflies run on unit vectors)
equal the oracle's, and invalid arguments are rejected before any launch."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import matrices as mx
from oracle import pipeline as pl
from paper_2207_11638_gb300 import binding as b

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"\b(cdct_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    lib = b.lib()
    declared = declared_functions()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert set(b.EXPORTS) == declared
    assert b"sm_103a" in lib.cdct_version()


@pytest.mark.parametrize("variant", ("tilde", "hat"))
@pytest.mark.parametrize("n", (8, 16, 32))
def test_host_matrices_equal_oracle(variant, n):
    p = b.Plan(n, variant)
    np.testing.assert_array_equal(p.matrix(b.MATRIX_T), mx.T_N(variant, n))
    np.testing.assert_array_equal(p.matrix(b.MATRIX_U), mx.U_N(variant, n))
    np.testing.assert_allclose(p.matrix(b.MATRIX_S), mx.scale_S(mx.T_N(variant, n)), rtol=1e-15)
    zz = p.matrix(b.MATRIX_ZIGZAG)
    for k, (i, j) in enumerate(pl.zigzag_order(n)):
        assert zz[i, j] == k


def test_host_matrices_exact():
    p = b.Plan(8, "exact")
    c = mx.dct2_matrix(8)
    np.testing.assert_allclose(p.matrix(b.MATRIX_T), 2 * c, atol=2e-6)
    np.testing.assert_allclose(p.matrix(b.MATRIX_U), 4 * c.T, atol=4e-6)
    np.testing.assert_allclose(p.matrix(b.MATRIX_S), np.full(8, 0.5), atol=1e-6)


def test_plan_argument_checks():
    lib = b.lib()
    h = ctypes.c_void_p()
    assert lib.cdct_plan_create(7, 2, 0, ctypes.byref(h)) == b.CDCT_EINVAL
    assert b"8, 16 or 32" in lib.cdct_last_error()
    assert lib.cdct_plan_create(8, 9, 0, ctypes.byref(h)) == b.CDCT_EINVAL
    assert lib.cdct_plan_create(8, 2, 4, ctypes.byref(h)) == b.CDCT_EINVAL
    assert lib.cdct_plan_create(16, 0, 0, ctypes.byref(h)) == b.CDCT_EUNSUPPORTED
    assert lib.cdct_plan_create(8, 2, 0, None) == b.CDCT_EINVAL
    with pytest.raises(b.CdctError):
        b.Plan(12, "hat")


def _desc(w=64, h=64, pitch=64, batch=1, bstride=0, dtype=0, ptr=0x100000):
    return b.CdctImage(ptr, dtype, w, h, pitch, batch, bstride)


def test_call_argument_checks_reject_before_launch():
    """Invalid calls return CDCT_EINVAL; the pointers here are never touched."""
    lib = b.lib()
    p = b.Plan(8, "hat")
    fake = ctypes.c_void_p(0x200000)
    d = _desc()
    # r out of range
    for r in (0, 65):
        assert lib.cdct_fwd_zonal_inv(p.handle, ctypes.byref(d), r, fake, 64, 0, None, None, None, 0, None) == b.CDCT_EINVAL
    # null image, null data, bad sizes, bad dtype
    assert lib.cdct_fwd_zonal_inv(p.handle, None, 6, fake, 64, 0, None, None, None, 0, None) == b.CDCT_EINVAL
    for bad in (_desc(ptr=0), _desc(w=0), _desc(pitch=10), _desc(dtype=5), _desc(batch=2, bstride=100),
                _desc(batch=0)):
        assert lib.cdct_fwd_zonal_inv(p.handle, ctypes.byref(bad), 6, fake, 64, 0, None, None, None, 0,
                                      None) == b.CDCT_EINVAL
    # recon pitch too small, PSNR without workspace, misaligned coefficient buffers
    assert lib.cdct_fwd_zonal_inv(p.handle, ctypes.byref(d), 6, fake, 10, 0, None, None, None, 0, None) == b.CDCT_EINVAL
    assert lib.cdct_fwd_zonal_inv(p.handle, ctypes.byref(d), 6, fake, 64, 0, None, fake, None, 0, None) == b.CDCT_EINVAL
    assert lib.cdct_forward(p.handle, ctypes.byref(d), ctypes.c_void_p(0x200004), None) == b.CDCT_EINVAL
    assert lib.cdct_inverse(p.handle, ctypes.c_void_p(0x200004), 64, 64, 1, fake, 64, 0, None) == b.CDCT_EINVAL
    assert lib.cdct_zonal(p.handle, 0, fake, 10, None, None, None) == b.CDCT_EINVAL
    assert lib.cdct_psnr(ctypes.byref(d), fake, 64, 0, fake, None, 0, None) == b.CDCT_EINVAL
    assert lib.cdct_matrix(p.handle, 9, (ctypes.c_double * 64)()) == b.CDCT_EINVAL


def test_block_count_and_workspace():
    lib = b.lib()
    for n, w, h, batch in ((8, 1920, 1080, 3), (16, 960, 540, 2), (32, 1920, 1080, 1), (8, 13, 7, 1)):
        p = b.Plan(n, "hat")
        d = _desc(w=w, h=h, pitch=w, batch=batch, bstride=w * h)
        nb = ctypes.c_int64()
        assert lib.cdct_block_count(p.handle, ctypes.byref(d), ctypes.byref(nb)) == 0
        assert nb.value == batch * (-(-w // n)) * (-(-h // n))
        ws = ctypes.c_size_t()
        assert lib.cdct_workspace_size(p.handle, ctypes.byref(d), ctypes.byref(ws)) == 0
        assert ws.value >= 8 * batch and ws.value % 8 == 0


def test_fault_injection_hook_argument_checks():
    """The failure-detection test hook validates its arguments on the host."""
    for mode, limit in ((4, 1 << 21), (-1, 1 << 21), (1, 10), (1, 1 << 40)):
        with pytest.raises(b.CdctError):
            b.set_fault_injection(mode, limit)
    b.set_fault_injection(1, 1 << 21)
    b.set_fault_injection(0)
