"""The fused call without a workspace, for callers that cannot allocate.

cdct_fwd_zonal_inv_noalloc keeps its error partials in a fixed static
scratch inside the library instead of a caller-provided workspace, so a
caller that owns only its input and output buffers (fixed memory budget,
no device allocator of its own) can still get reconstructions and PSNRs.
This file checks it against cdct_fwd_zonal_inv, through the C ABI, on two
calls in a row (the scratch keeps the previous call's contents), on both
the pipelined and the fallback kernel, and checks the size limit.  It is
collected last so that a stop at the first failure has run everything else.
"""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2207_11638_gb300 import binding as b

pytestmark = pytest.mark.gpu

PSNR_TOL_DB = 1e-4
RECON_TOL = 1e-3
SCRATCH_BYTES = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _case(dtype, shape, seed):
    rng = np.random.default_rng(seed)
    if dtype == "u8":
        a = rng.integers(0, 256, size=shape).astype(np.uint8)
    else:
        a = rng.integers(-255, 256, size=shape).astype(np.int16)
    return torch.from_numpy(a).cuda()


def _same(got, want):
    rec, _, ps = got
    rec_w, _, ps_w = want
    assert float((rec - rec_w).abs().max()) <= RECON_TOL
    for g, w in zip(ps.cpu().tolist(), ps_w.cpu().tolist()):
        if math.isinf(w):
            assert math.isinf(g)
        else:
            assert abs(g - w) <= PSNR_TOL_DB


@pytest.mark.parametrize("n,variant,dtype,shape,r", [
    (16, "hat", "i16", (3, 96, 128), 64),      # aligned rows: pipelined kernel
    (8, "tilde", "u8", (2, 37, 45), 6),        # unaligned rows: fallback kernel
    (32, "hat", "i16", (2, 70, 200), 256),
])
def test_noalloc_matches_workspace_call_twice(n, variant, dtype, shape, r):
    plan = b.Plan(n, variant)
    img = _case(dtype, shape, seed=n + r)
    other = _case(dtype, (1, 64, 64), seed=99)
    want = plan.fwd_zonal_inv(img, r)
    want_other = plan.fwd_zonal_inv(other, r)
    for _ in range(2):                      # the scratch keeps the last call's contents
        got = b.fwd_zonal_inv_noalloc(plan, img, r)
        torch.cuda.synchronize()
        _same(got, want)
        # a smaller call in between, which finds the larger call's partials in the scratch
        got_other = b.fwd_zonal_inv_noalloc(plan, other, r)
        torch.cuda.synchronize()
        _same(got_other, want_other)
    b.check_device()


def test_noalloc_without_psnr_and_limit():
    plan = b.Plan(8, "hat")
    img = _case("i16", (2, 64, 96), seed=5)
    rec, _, ps = b.fwd_zonal_inv_noalloc(plan, img, 10, psnr=False)
    want, _, _ = plan.fwd_zonal_inv(img, 10, psnr=False)
    torch.cuda.synchronize()
    assert ps is None and float((rec - want).abs().max()) <= RECON_TOL
    # a call whose partials exceed the fixed scratch is refused before any launch
    d = b.image_desc(img)
    d.batch, d.batch_stride = 8192, d.pitch * d.height
    ws = ctypes.c_size_t()
    assert b.lib().cdct_workspace_size(plan.handle, ctypes.byref(d), ctypes.byref(ws)) == 0
    assert ws.value > SCRATCH_BYTES
    out = torch.empty(1, device="cuda")
    st = b.lib().cdct_fwd_zonal_inv_noalloc(plan.handle, ctypes.byref(d), 10, out.data_ptr(), d.width,
                                           d.width * d.height, None, out.data_ptr(), None)
    assert st == b.CDCT_EINVAL
    assert b"scratch" in b.lib().cdct_last_error()
