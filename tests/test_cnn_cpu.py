"""CNN selector entry points without a GPU: the flat parameter layout agrees
between the header, the seeded initialiser and the oracle, and invalid calls
are rejected before any launch."""
import ctypes

import numpy as np
import pytest

from oracle import cnn
from paper_2207_11638_gb300 import binding as b
from paper_2207_11638_gb300 import synth
from tests.cnn_util import from_oracle, to_oracle


def test_layouts_agree():
    assert b.CNN_PARAMS == cnn.param_count() == sum(n for _, n, _ in synth.CNN_LAYOUT)
    assert [n for _, n, _ in synth.CNN_LAYOUT] == [int(np.prod(s)) for _, s in cnn.PARAM_SHAPES]
    flat = synth.cnn_init_params(3, bias_std=0.1)
    assert np.array_equal(from_oracle(to_oracle(flat)), flat.astype(np.float64))
    # He-normal spread per weight tensor
    p = to_oracle(synth.cnn_init_params(0))
    assert abs(np.std(p["fc1_w"]) - np.sqrt(2 / 512)) < 0.01 * np.sqrt(2 / 512) * 10
    assert not np.any(p["conv2_b"])


def test_packed_size_and_workspace():
    lib = b.lib()
    assert lib.cdct_cnn_packed_bytes() % 256 == 0 and lib.cdct_cnn_packed_bytes() >= 2 * 48241 // 2
    n = ctypes.c_size_t()
    assert lib.cdct_cnn_workspace_size(64, ctypes.byref(n)) == 0
    small = n.value
    assert lib.cdct_cnn_workspace_size(256, ctypes.byref(n)) == 0
    assert n.value > 3 * small and n.value % 256 == 0
    for bad in (0, 32, 100, -64):
        assert lib.cdct_cnn_workspace_size(bad, ctypes.byref(n)) == b.CDCT_EINVAL


def test_cnn_argument_checks_reject_before_launch():
    lib = b.lib()
    fake = ctypes.c_void_p(0x200000)
    d = b.CdctImage(0x100000, 1, 64, 64, 64, 1, 0)
    slots = (ctypes.c_int32 * 3)(0, 1, 2)
    bad_slots = (ctypes.c_int32 * 2)(0, 4)
    assert lib.cdct_cnn_pack(None, fake, None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_pack(fake, ctypes.c_void_p(0x200004), None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_infer(fake, ctypes.byref(d), slots, 0, fake, None, None, None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_infer(fake, ctypes.byref(d), slots, 5, fake, None, None, None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_infer(fake, ctypes.byref(d), bad_slots, 2, fake, None, None, None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_infer(fake, ctypes.byref(d), slots, 3, None, None, None, None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_infer(None, ctypes.byref(d), slots, 3, fake, None, None, None) == b.CDCT_EINVAL
    bad_img = b.CdctImage(0x100000, 7, 64, 64, 64, 1, 0)
    assert lib.cdct_cnn_infer(fake, ctypes.byref(bad_img), slots, 3, fake, None, None, None) == b.CDCT_EINVAL
    ws = ctypes.c_void_p(0x300000)
    for batch in (0, 63, 100):
        assert lib.cdct_cnn_grad(fake, fake, batch, slots, 3, fake, None, 0.0, fake, fake, ws, 1 << 30,
                                 None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_grad(fake, fake, 64, slots, 3, fake, None, -1.0, fake, fake, ws, 1 << 30, None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_grad(fake, fake, 64, slots, 3, fake, None, 0.0, fake, fake, ws, 16, None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_grad(fake, fake, 64, slots, 3, fake, None, 0.0, fake, fake, ctypes.c_void_p(0x300010),
                             1 << 30, None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_grad(fake, None, 64, slots, 3, fake, None, 0.0, fake, fake, ws, 1 << 30, None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_adam(fake, fake, fake, fake, 0, 1e-3, 0.9, 0.999, 1e-8, None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_adam(fake, fake, fake, fake, 1, 0.0, 0.9, 0.999, 1e-8, None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_adam(fake, fake, fake, fake, 1, 1e-3, 1.0, 0.999, 1e-8, None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_adam(fake, None, fake, fake, 1, 1e-3, 0.9, 0.999, 1e-8, None) == b.CDCT_EINVAL


def test_fallback_and_evaluate_argument_checks():
    lib = b.lib()
    fake = ctypes.c_void_p(0x200000)
    d = b.CdctImage(0x100000, 1, 64, 64, 64, 1, 0)      # 4 regions
    q = (ctypes.c_int32 * 3)(8, 16, 32)
    rd = b.RdSearch("hat")
    h = rd._h
    assert lib.cdct_rd_search_subset(h, ctypes.byref(d), q, 3, 1, 2, None, fake, 4, fake, None, None) == b.CDCT_EINVAL
    assert lib.cdct_rd_search_subset(h, ctypes.byref(d), q, 3, 1, 2, fake, None, 4, fake, None, None) == b.CDCT_EINVAL
    assert lib.cdct_rd_search_subset(h, ctypes.byref(d), q, 3, 1, 2, fake, fake, 5, fake, None, None) == b.CDCT_EINVAL
    assert lib.cdct_rd_search_subset(h, ctypes.byref(d), q, 0, 1, 2, fake, fake, 4, fake, None, None) == b.CDCT_EINVAL
    assert lib.cdct_rd_search_subset(None, ctypes.byref(d), q, 3, 1, 2, fake, fake, 4, fake, None, None) == b.CDCT_EINVAL
    # max_count 0: nothing to do, nothing launched
    assert lib.cdct_rd_search_subset(h, ctypes.byref(d), q, 3, 1, 2, fake, fake, 0, fake, None, None) == b.CDCT_OK
    assert lib.cdct_rd_evaluate(h, ctypes.byref(d), q, 3, 1, 2, fake, None, None, None, None) == b.CDCT_EINVAL
    assert lib.cdct_rd_evaluate(h, ctypes.byref(d), q, 3, 1, 2, None, fake, None, None, None) == b.CDCT_EINVAL
    assert lib.cdct_rd_evaluate(h, ctypes.byref(d), q, 3, 2000, 2, fake, fake, None, None, None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_select(fake, 10, 0, 0.5, fake, fake, None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_select(fake, 10, 5, 0.5, fake, fake, None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_select(None, 10, 3, 0.5, fake, fake, None) == b.CDCT_EINVAL
    assert lib.cdct_cnn_select(fake, 10, 3, float("nan"), fake, fake, None) == b.CDCT_EINVAL


def test_ssim_argument_checks():
    lib = b.lib()
    fake = ctypes.c_void_p(0x200000)
    n = ctypes.c_size_t()
    d = b.CdctImage(0x100000, 0, 64, 48, 64, 2, 64 * 48)
    assert lib.cdct_ssim_workspace_size(ctypes.byref(d), ctypes.byref(n)) == b.CDCT_OK
    assert n.value == 2 * 2 * 2 * 8          # 2 images x (54/32 -> 2) x (38/32 -> 2) tiles x 8 bytes
    small = b.CdctImage(0x100000, 0, 10, 48, 64, 1, 0)
    assert lib.cdct_ssim_workspace_size(ctypes.byref(small), ctypes.byref(n)) == b.CDCT_EINVAL
    assert lib.cdct_ssim(ctypes.byref(d), fake, 64, 64 * 48, None, fake, 1 << 20, None) == b.CDCT_EINVAL
    assert lib.cdct_ssim(ctypes.byref(d), fake, 64, 64 * 48, fake, fake, 8, None) == b.CDCT_EINVAL
    assert lib.cdct_ssim(ctypes.byref(d), fake, 10, 64 * 48, fake, fake, 1 << 20, None) == b.CDCT_EINVAL
    assert lib.cdct_ssim(ctypes.byref(d), None, 64, 64 * 48, fake, fake, 1 << 20, None) == b.CDCT_EINVAL


def test_checkpoint_roundtrip_and_rejections(tmp_path):
    rng = np.random.default_rng(2)
    params = synth.cnn_init_params(4)
    m = rng.standard_normal(params.size).astype(np.float32)
    v = rng.random(params.size).astype(np.float32)
    path = str(tmp_path / "sel.ckpt")
    b.write_checkpoint(path, params, m, v, 1234, {"data_seed": 40, "epoch": 3})
    p2, m2, v2, step, extra = b.read_checkpoint(path)
    assert np.array_equal(p2, params) and np.array_equal(m2, m) and np.array_equal(v2, v)
    assert step == 1234 and extra == {"data_seed": 40, "epoch": 3}
    raw = open(path, "rb").read()
    for bad, why in ((raw[:-10], "truncated"), (raw[:100] + bytes([raw[100] ^ 1]) + raw[101:], "checksum"),
                     (b"XXXXXXXX" + raw[8:], "magic")):
        open(path, "wb").write(bad)
        with pytest.raises(b.CheckpointError):
            b.read_checkpoint(path)
    with pytest.raises(b.CheckpointError):
        b.write_checkpoint(path, params[:10], m, v, 1, {})
