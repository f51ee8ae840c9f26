"""Thin ctypes binding of libcdct.so (include/cdct.h).

Argument marshalling only: every step of the transform runs in the CUDA
library.  PyTorch provides device memory and the current stream.  There is
no CPU fallback: if the library is missing or fails to load, importing the
binding raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcdct.so")

CDCT_OK, CDCT_EINVAL, CDCT_ENOMEM, CDCT_ECUDA, CDCT_EUNSUPPORTED, CDCT_ETIMEOUT = range(6)
VARIANTS = {"exact": 0, "tilde": 1, "hat": 2}
CONVS = {"paper": 0, "transpose": 1}
DTYPES = {"u8": 0, "i16": 1}
MATRIX_T, MATRIX_U, MATRIX_S, MATRIX_ZIGZAG = range(4)

# every symbol include/cdct.h declares
EXPORTS = (
    "cdct_plan_create", "cdct_plan_destroy", "cdct_block_count", "cdct_workspace_size",
    "cdct_forward", "cdct_zonal", "cdct_inverse", "cdct_psnr", "cdct_fwd_zonal_inv",
    "cdct_matrix", "cdct_last_error", "cdct_version", "cdct_check_device",
    "cdct_fwd_zonal_inv_noalloc", "cdct_plan_set_tuning", "cdct_batch_create", "cdct_batch_destroy",
    "cdct_batch_sizes", "cdct_batch_upload", "cdct_batch_unit", "cdct_batch_fzi",
    "cdct_rd_create", "cdct_rd_destroy", "cdct_rd_tables", "cdct_rd_region_count", "cdct_rd_search",
    "cdct_cnn_packed_bytes", "cdct_cnn_pack", "cdct_cnn_infer", "cdct_cnn_workspace_size", "cdct_cnn_grad",
    "cdct_cnn_adam", "cdct_rd_search_subset", "cdct_rd_evaluate", "cdct_cnn_select",
    "cdct_ssim_workspace_size", "cdct_ssim", "cdct_set_fault_injection",
)
CNN_PARAMS, CNN_LABELS, CNN_SLOTS = 48241, 17, 4


class CdctImage(ctypes.Structure):
    _fields_ = [
        ("data", ctypes.c_void_p),
        ("dtype", ctypes.c_int32),
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("pitch", ctypes.c_int64),
        ("batch", ctypes.c_int32),
        ("batch_stride", ctypes.c_int64),
    ]


class CdctBatchImage(ctypes.Structure):
    _fields_ = [
        ("data", ctypes.c_void_p),
        ("recon", ctypes.c_void_p),
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("pitch", ctypes.c_int64),
        ("recon_pitch", ctypes.c_int64),
    ]


class CdctError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"cdct status {status}: {msg}")
        self.status = status


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2207_11638_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    img_p = ctypes.POINTER(CdctImage)
    sig = {
        "cdct_plan_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(vp)]),
        "cdct_plan_destroy": (ctypes.c_int, [vp]),
        "cdct_block_count": (ctypes.c_int, [vp, img_p, ctypes.POINTER(i64)]),
        "cdct_workspace_size": (ctypes.c_int, [vp, img_p, ctypes.POINTER(sz)]),
        "cdct_forward": (ctypes.c_int, [vp, img_p, vp, vp]),
        "cdct_zonal": (ctypes.c_int, [vp, ctypes.c_int, vp, i64, vp, vp, vp]),
        "cdct_inverse": (ctypes.c_int, [vp, vp, i32, i32, i32, vp, i64, i64, vp]),
        "cdct_psnr": (ctypes.c_int, [img_p, vp, i64, i64, vp, vp, sz, vp]),
        "cdct_fwd_zonal_inv": (ctypes.c_int, [vp, img_p, ctypes.c_int, vp, i64, i64, vp, vp, vp, sz, vp]),
        "cdct_matrix": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
        "cdct_last_error": (ctypes.c_char_p, []),
        "cdct_version": (ctypes.c_char_p, []),
        "cdct_check_device": (ctypes.c_int, [vp]),
        "cdct_set_fault_injection": (ctypes.c_int, [ctypes.c_int, i64]),
        "cdct_fwd_zonal_inv_noalloc": (ctypes.c_int, [vp, img_p, ctypes.c_int, vp, i64, i64, vp, vp, vp]),
        "cdct_plan_set_tuning": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
        "cdct_batch_create": (ctypes.c_int, [vp, ctypes.POINTER(CdctBatchImage), ctypes.c_int, ctypes.c_int,
                                             ctypes.POINTER(vp)]),
        "cdct_batch_destroy": (ctypes.c_int, [vp]),
        "cdct_batch_sizes": (ctypes.c_int, [vp, ctypes.POINTER(sz), ctypes.POINTER(sz), ctypes.POINTER(i64)]),
        "cdct_batch_upload": (ctypes.c_int, [vp, vp, vp]),
        "cdct_batch_unit": (ctypes.c_int, [vp, i64, ctypes.POINTER(i32)]),
        "cdct_batch_fzi": (ctypes.c_int, [vp, vp, ctypes.c_int, vp, vp, sz, vp]),
        "cdct_rd_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(vp)]),
        "cdct_rd_destroy": (ctypes.c_int, [vp]),
        "cdct_rd_tables": (ctypes.c_int, [vp, ctypes.POINTER(i32)]),
        "cdct_rd_region_count": (ctypes.c_int, [img_p, ctypes.POINTER(i64)]),
        "cdct_rd_search": (ctypes.c_int, [vp, img_p, ctypes.POINTER(i32), i32, i32, i32, vp, vp, vp]),
        "cdct_rd_search_subset": (ctypes.c_int, [vp, img_p, ctypes.POINTER(i32), i32, i32, i32, vp, vp, i64, vp,
                                                 vp, vp]),
        "cdct_rd_evaluate": (ctypes.c_int, [vp, img_p, ctypes.POINTER(i32), i32, i32, i32, vp, vp, vp, vp, vp]),
        "cdct_cnn_select": (ctypes.c_int, [vp, i64, i32, ctypes.c_float, vp, vp, vp]),
        "cdct_ssim_workspace_size": (ctypes.c_int, [img_p, ctypes.POINTER(sz)]),
        "cdct_ssim": (ctypes.c_int, [img_p, vp, i64, i64, vp, vp, sz, vp]),
        "cdct_cnn_packed_bytes": (sz, []),
        "cdct_cnn_pack": (ctypes.c_int, [vp, vp, vp]),
        "cdct_cnn_infer": (ctypes.c_int, [vp, img_p, ctypes.POINTER(i32), i32, vp, vp, vp, vp]),
        "cdct_cnn_workspace_size": (ctypes.c_int, [i32, ctypes.POINTER(sz)]),
        "cdct_cnn_grad": (ctypes.c_int, [vp, vp, i32, ctypes.POINTER(i32), i32, vp, vp, ctypes.c_float, vp, vp, vp,
                                         sz, vp]),
        "cdct_cnn_adam": (ctypes.c_int, [vp, vp, vp, vp, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                         ctypes.c_float, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_LIB = None


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


def check_device(stream=None) -> None:
    """Synchronise the stream; raise if a kernel gave up a bounded wait."""
    check(lib().cdct_check_device(stream_handle(stream)))


def device_status(stream=None) -> int:
    """cdct_check_device's status code (CDCT_OK, or CDCT_ETIMEOUT once after a wait gave up)."""
    return int(lib().cdct_check_device(stream_handle(stream)))


def set_fault_injection(mode: int, wait_limit_cycles: int = 0) -> None:
    """cdct_set_fault_injection: failure-detection test hook (0 turns it off)."""
    check(lib().cdct_set_fault_injection(mode, wait_limit_cycles))


def check(status: int) -> None:
    if status != CDCT_OK:
        raise CdctError(status, lib().cdct_last_error().decode())


# ---------------------------------------------------------------------------
# torch-facing helpers (torch is imported lazily: the C ABI needs none of it)
# ---------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def stream_handle(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def image_desc(t) -> CdctImage:
    """Descriptor of a CUDA tensor [H, W] or [B, H, W] (uint8 or int16, unit column stride)."""
    torch = _torch()
    if not t.is_cuda:
        raise ValueError("image must be a CUDA tensor")
    if t.dtype == torch.uint8:
        dt = 0
    elif t.dtype == torch.int16:
        dt = 1
    else:
        raise ValueError("image dtype must be uint8 or int16")
    if t.dim() == 2:
        t3 = t.unsqueeze(0)
    elif t.dim() == 3:
        t3 = t
    else:
        raise ValueError("image must be [H, W] or [B, H, W]")
    if t3.stride(2) != 1:
        raise ValueError("image rows must be contiguous")
    b, h, w = t3.shape
    return CdctImage(t3.data_ptr(), dt, w, h, t3.stride(1), b, t3.stride(0) if b > 1 else h * t3.stride(1))


class Plan:
    """A transform plan: block size N, variant and 2-D convention (Sec. 5.1)."""

    def __init__(self, n: int, variant: str = "hat", conv: str = "paper"):
        self.n, self.variant, self.conv = n, variant, conv
        h = ctypes.c_void_p()
        check(lib().cdct_plan_create(n, VARIANTS[variant], CONVS[conv], ctypes.byref(h)))
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _LIB is not None:
            _LIB.cdct_plan_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def set_tuning(self, stages: int = 0, ctas_per_sm: int = 0):
        """Staging depth (0, 2, 3) and resident CTAs per SM (0 = all that fit)."""
        check(lib().cdct_plan_set_tuning(self._h, stages, ctas_per_sm))
        self.tuning = (stages, ctas_per_sm)

    # -- host tables ---------------------------------------------------------
    def matrix(self, which: int):
        import numpy as np
        n = self.n
        size = n if which == MATRIX_S else n * n
        buf = (ctypes.c_double * size)()
        check(lib().cdct_matrix(self._h, which, buf))
        arr = np.frombuffer(buf, dtype=np.float64).copy()
        return arr if which == MATRIX_S else arr.reshape(n, n)

    def block_count(self, img) -> int:
        d = image_desc(img)
        out = ctypes.c_int64()
        check(lib().cdct_block_count(self._h, ctypes.byref(d), ctypes.byref(out)))
        return out.value

    def workspace_size(self, img) -> int:
        d = image_desc(img)
        out = ctypes.c_size_t()
        check(lib().cdct_workspace_size(self._h, ctypes.byref(d), ctypes.byref(out)))
        return out.value

    def workspace(self, img):
        torch = _torch()
        nbytes = self.workspace_size(img)
        return torch.empty(max(1, nbytes // 8), dtype=torch.float64, device=img.device)

    # -- pipeline calls --------------------------------------------------------
    def _coeff_dtype(self):
        torch = _torch()
        return torch.float32 if self.variant == "exact" else torch.int32

    def forward(self, img, stream=None):
        """Block-major coefficients [B, nby, nbx, N, N] (int32; float32 for exact)."""
        torch = _torch()
        d = image_desc(img)
        n = self.n
        nby, nbx = -(-d.height // n), -(-d.width // n)
        coeff = torch.empty((d.batch, nby, nbx, n, n), dtype=self._coeff_dtype(), device=img.device)
        check(lib().cdct_forward(self._h, ctypes.byref(d), coeff.data_ptr(), stream_handle(stream)))
        return coeff

    def zonal(self, coeff, r: int, scaled: bool = False, kept: bool = False, stream=None):
        """Mask coeff in place; optionally return scaled B and the kept coefficients."""
        torch = _torch()
        n = self.n
        nblocks = coeff.numel() // (n * n)
        sc = torch.empty(coeff.shape, dtype=torch.float32, device=coeff.device) if scaled else None
        kp = torch.empty((*coeff.shape[:-2], r), dtype=coeff.dtype, device=coeff.device) if kept else None
        check(lib().cdct_zonal(self._h, r, coeff.data_ptr(), nblocks,
                               sc.data_ptr() if sc is not None else None,
                               kp.data_ptr() if kp is not None else None, stream_handle(stream)))
        return coeff, sc, kp

    def inverse(self, coeff, width: int, height: int, out=None, stream=None):
        """Reconstruction [B, H, W] float32 from block-major coefficients."""
        torch = _torch()
        b = coeff.shape[0]
        if out is None:
            out = torch.empty((b, height, width), dtype=torch.float32, device=coeff.device)
        check(lib().cdct_inverse(self._h, coeff.data_ptr(), width, height, b, out.data_ptr(),
                                 out.stride(1), out.stride(0) if b > 1 else height * out.stride(1),
                                 stream_handle(stream)))
        return out

    def fwd_zonal_inv(self, img, r: int, out=None, kept: bool = False, psnr: bool = True,
                      workspace=None, psnr_out=None, kept_out=None, stream=None):
        """Fused forward -> zonal(r) -> inverse (+ per-image PSNR on the device).

        Returns (recon [B, H, W] float32, kept [B, nby, nbx, r] or None,
        psnr [B] float64 on the device or None).
        """
        torch = _torch()
        d = image_desc(img)
        n = self.n
        if out is None:
            out = torch.empty((d.batch, d.height, d.width), dtype=torch.float32, device=img.device)
        o3 = out if out.dim() == 3 else out.unsqueeze(0)
        kp = kept_out
        if kept and kp is None:
            nby, nbx = -(-d.height // n), -(-d.width // n)
            kp = torch.empty((d.batch, nby, nbx, r), dtype=self._coeff_dtype(), device=img.device)
        ps = psnr_out
        if psnr and ps is None:
            ps = torch.empty(d.batch, dtype=torch.float64, device=img.device)
        ws = workspace
        if psnr and ws is None:
            ws = self.workspace(img)
        check(lib().cdct_fwd_zonal_inv(
            self._h, ctypes.byref(d), r, o3.data_ptr(), o3.stride(1),
            o3.stride(0) if d.batch > 1 else d.height * o3.stride(1),
            kp.data_ptr() if kp is not None else None,
            ps.data_ptr() if ps is not None else None,
            ws.data_ptr() if ws is not None else None,
            ws.numel() * ws.element_size() if ws is not None else 0,
            stream_handle(stream)))
        return out, kp, ps


def fwd_zonal_inv_noalloc(plan, img, r, out=None, kept=False, psnr=True, stream=None):
    """cdct_fwd_zonal_inv_noalloc: the fused call without a workspace (the
    library's fixed static scratch holds the error partials)."""
    torch = _torch()
    d = image_desc(img)
    n = plan.n
    if out is None:
        out = torch.empty((d.batch, d.height, d.width), dtype=torch.float32, device=img.device)
    o3 = out if out.dim() == 3 else out.unsqueeze(0)
    kp = None
    if kept:
        nby, nbx = -(-d.height // n), -(-d.width // n)
        kp = torch.empty((d.batch, nby, nbx, r), dtype=plan._coeff_dtype(), device=img.device)
    ps = torch.empty(d.batch, dtype=torch.float64, device=img.device) if psnr else None
    check(lib().cdct_fwd_zonal_inv_noalloc(
        plan.handle, ctypes.byref(d), r, o3.data_ptr(), o3.stride(1),
        o3.stride(0) if d.batch > 1 else d.height * o3.stride(1),
        kp.data_ptr() if kp is not None else None,
        ps.data_ptr() if ps is not None else None, stream_handle(stream)))
    return out, kp, ps


class Batch:
    """Images of uneven sizes run by one persistent launch (cdct_batch_*).

    ``images``: CUDA tensors [H, W] (uint8 or int16, same dtype, rows
    contiguous and 16-byte aligned).  Reconstructions are float32 tensors
    [H, W] allocated here unless given.
    """

    def __init__(self, plan: Plan, images, recons=None):
        torch = _torch()
        self.plan, self.images = plan, list(images)
        dt = self.images[0].dtype
        if any(t.dtype != dt for t in self.images):
            raise ValueError("all images of a batch share one dtype")
        self.dtype = DTYPES["u8" if dt == torch.uint8 else "i16"]
        if recons is None:
            recons = [torch.empty(t.shape, dtype=torch.float32, device=t.device) for t in self.images]
        self.recons = list(recons)
        n = len(self.images)
        descs = (CdctBatchImage * n)()
        for i, (t, o) in enumerate(zip(self.images, self.recons)):
            if t.dim() != 2 or t.stride(1) != 1 or o.stride(1) != 1:
                raise ValueError("batch images must be [H, W] with contiguous rows")
            descs[i] = CdctBatchImage(t.data_ptr(), o.data_ptr(), t.shape[1], t.shape[0], t.stride(0), o.stride(0))
        h = ctypes.c_void_p()
        check(lib().cdct_batch_create(plan.handle, descs, n, self.dtype, ctypes.byref(h)))
        self._h = h
        tb, wb, px = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int64()
        check(lib().cdct_batch_sizes(h, ctypes.byref(tb), ctypes.byref(wb), ctypes.byref(px)))
        dev = self.images[0].device
        self.pixels = px.value
        self.table = torch.empty(max(16, tb.value), dtype=torch.uint8, device=dev)
        self.workspace = torch.empty(max(1, wb.value // 8), dtype=torch.float64, device=dev)
        self.psnr = torch.empty(n, dtype=torch.float64, device=dev)
        check(lib().cdct_batch_upload(h, self.table.data_ptr(), stream_handle()))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _LIB is not None:
            _LIB.cdct_batch_destroy(h)
            self._h = None

    def run(self, r: int, psnr: bool = True, stream=None):
        """Fused forward -> zonal(r) -> inverse over every image; returns the
        per-image PSNR tensor (device) or None."""
        check(lib().cdct_batch_fzi(self._h, self.table.data_ptr(), r,
                                   self.psnr.data_ptr() if psnr else None,
                                   self.workspace.data_ptr() if psnr else None,
                                   self.workspace.numel() * 8 if psnr else 0, stream_handle(stream)))
        return self.psnr if psnr else None


_PSNR_PLAN = None


def _psnr_plan():
    # cdct_workspace_size() of any plan covers the standalone PSNR reduction
    global _PSNR_PLAN
    if _PSNR_PLAN is None:
        _PSNR_PLAN = Plan(8, "hat")
    return _PSNR_PLAN


def psnr(ref, recon, workspace=None, stream=None):
    """Per-image PSNR [B] (float64, device) of a float32 reconstruction against ref."""
    torch = _torch()
    d = image_desc(ref)
    r3 = recon if recon.dim() == 3 else recon.unsqueeze(0)
    out = torch.empty(d.batch, dtype=torch.float64, device=ref.device)
    if workspace is None:
        workspace = _psnr_plan().workspace(ref)
    check(lib().cdct_psnr(ctypes.byref(d), r3.data_ptr(), r3.stride(1),
                          r3.stride(0) if d.batch > 1 else d.height * r3.stride(1),
                          out.data_ptr(), workspace.data_ptr(),
                          workspace.numel() * workspace.element_size(), stream_handle(stream)))
    return out


# ---------------------------------------------------------------------------
# Rate-distortion quadtree search (cdct_rd_*)
# ---------------------------------------------------------------------------

RD_PARTITIONS = 17
RD_COST_SCALE = float(2 ** 24 * 32 ** 4)     # J' / RD_COST_SCALE = SSE + kappa q^2 R


class RdSearch:
    """Exhaustive RD quadtree search over the 32 x 32 regions of images.

    ``variant``: "tilde" or "hat".  ``kappa`` = kappa_num / 2**kappa_log2_den
    (lambda = kappa q^2; default 1/4)."""

    def __init__(self, variant: str = "hat", kappa_num: int = 1, kappa_log2_den: int = 2):
        self.variant, self.kappa_num, self.kappa_log2_den = variant, kappa_num, kappa_log2_den
        h = ctypes.c_void_p()
        check(lib().cdct_rd_create(VARIANTS[variant], ctypes.byref(h)))
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _LIB is not None:
            _LIB.cdct_rd_destroy(h)
            self._h = None

    def tables(self):
        """(d {32, 16, 8: [N]}, c {32, 16, 8: [N][N]}) host tables, as lists."""
        buf = (ctypes.c_int32 * 1440)()
        check(lib().cdct_rd_tables(self._h, buf))
        v = list(buf)
        d = {n: v[k * 32:k * 32 + n] for k, n in enumerate((32, 16, 8))}
        c, off = {}, 96
        for n in (32, 16, 8):
            c[n] = [v[off + i * n:off + (i + 1) * n] for i in range(n)]
            off += n * n
        return d, c

    @staticmethod
    def region_count(img) -> int:
        d = image_desc(img)
        n = ctypes.c_int64()
        check(lib().cdct_rd_region_count(ctypes.byref(d), ctypes.byref(n)))
        return n.value

    def search(self, img, qs, costs: bool = False, stream=None):
        """labels [len(qs), R] uint8 (device) and, with ``costs``, the 17 partition costs
        [len(qs), R, 17] as (low, high) int64 word pairs [len(qs), R, 17, 2] (device)."""
        torch = _torch()
        d = image_desc(img)
        n = self.region_count(img)
        qs = [int(q) for q in qs]
        qa = (ctypes.c_int32 * len(qs))(*qs)
        labels = torch.empty((len(qs), n), dtype=torch.uint8, device=img.device)
        pc = torch.empty((len(qs), n, RD_PARTITIONS, 2), dtype=torch.int64, device=img.device) if costs else None
        check(lib().cdct_rd_search(self._h, ctypes.byref(d), qa, len(qs), self.kappa_num, self.kappa_log2_den,
                                   labels.data_ptr(), pc.data_ptr() if costs else None, stream_handle(stream)))
        return (labels, pc) if costs else labels

    def search_subset(self, img, qs, region_index, count, labels, costs=None, stream=None):
        """Re-decide the regions listed in region_index (device int64; *count of them,
        a device int64) into ``labels`` [len(qs), R] in place (and ``costs`` if given)."""
        d = image_desc(img)
        n = self.region_count(img)
        qs = [int(q) for q in qs]
        qa = (ctypes.c_int32 * len(qs))(*qs)
        check(lib().cdct_rd_search_subset(self._h, ctypes.byref(d), qa, len(qs), self.kappa_num, self.kappa_log2_den,
                                          region_index.data_ptr(), count.data_ptr(), min(n, region_index.numel()),
                                          labels.data_ptr(),
                                          costs.data_ptr() if costs is not None else None, stream_handle(stream)))
        return labels

    def evaluate(self, img, qs, labels, stream=None):
        """(cost [len(qs), R, 2], dist [len(qs), R, 2] as (low, high) int64 words, bits
        [len(qs), R] int32) of coding every region with the labelled quadtree (device)."""
        torch = _torch()
        d = image_desc(img)
        n = self.region_count(img)
        qs = [int(q) for q in qs]
        qa = (ctypes.c_int32 * len(qs))(*qs)
        cost = torch.empty((len(qs), n, 2), dtype=torch.int64, device=img.device)
        dist = torch.empty((len(qs), n, 2), dtype=torch.int64, device=img.device)
        bits = torch.empty((len(qs), n), dtype=torch.int32, device=img.device)
        check(lib().cdct_rd_evaluate(self._h, ctypes.byref(d), qa, len(qs), self.kappa_num, self.kappa_log2_den,
                                     labels.contiguous().data_ptr(), cost.data_ptr(), dist.data_ptr(),
                                     bits.data_ptr(), stream_handle(stream)))
        return cost, dist, bits


def ssim(ref, recon, out=None, workspace=None, stream=None):
    """Mean SSIM per image of recon (float32 [B, H, W] or [H, W]) against ref (uint8 / int16),
    as a device float64 tensor [B]."""
    torch = _torch()
    d = image_desc(ref)
    r3 = recon if recon.dim() == 3 else recon.unsqueeze(0)
    if r3.dtype != torch.float32 or r3.stride(2) != 1:
        raise ValueError("recon must be float32 with contiguous rows")
    n = ctypes.c_size_t()
    check(lib().cdct_ssim_workspace_size(ctypes.byref(d), ctypes.byref(n)))
    if workspace is None:
        workspace = torch.empty(max(n.value // 8, 1), dtype=torch.float64, device=ref.device)
    if out is None:
        out = torch.empty(d.batch, dtype=torch.float64, device=ref.device)
    check(lib().cdct_ssim(ctypes.byref(d), r3.data_ptr(), r3.stride(1),
                          r3.stride(0) if d.batch > 1 else d.height * r3.stride(1), out.data_ptr(),
                          workspace.data_ptr(), workspace.numel() * workspace.element_size(), stream_handle(stream)))
    return out


def cnn_select(margin, threshold: float, stream=None):
    """(region_index [R] int64, count [1] int64) device tensors: the regions whose smallest
    margin over the slots (margin [n_slots, R]) is below ``threshold``."""
    torch = _torch()
    ns, n = margin.shape
    idx = torch.empty(max(n, 1), dtype=torch.int64, device=margin.device)
    cnt = torch.empty(1, dtype=torch.int64, device=margin.device)
    check(lib().cdct_cnn_select(margin.contiguous().data_ptr(), n, ns, float(threshold), idx.data_ptr(),
                                cnt.data_ptr(), stream_handle(stream)))
    return idx, cnt


def rd_cost_ints(pc_host) -> list:
    """(low, high) uint64 word pairs (as int64) -> Python ints."""
    import numpy as np
    a = np.asarray(pc_host).astype(np.uint64)
    lo, hi = a[..., 0], a[..., 1]
    return [[[int(h) << 64 | int(l) for l, h in zip(lr, hr)] for lr, hr in zip(lq, hq)] for lq, hq in zip(lo, hi)]


class Cnn:
    """Learned quadtree selector (include/cdct.h, cdct_cnn_*).

    ``params``: device float32 tensor of CNN_PARAMS master weights, owned by
    this object (updated in place by ``adam``); Adam state and the packed
    inference weights live beside it.  ``slots`` index the quantiser steps the
    network was trained for (0..3)."""

    def __init__(self, params):
        torch = _torch()
        if params.dtype != torch.float32 or params.numel() != CNN_PARAMS or not params.is_cuda:
            raise ValueError("params must be a CUDA float32 tensor of CNN_PARAMS values")
        self.params = params.contiguous()
        dev = self.params.device
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self.packed = torch.empty(lib().cdct_cnn_packed_bytes(), dtype=torch.uint8, device=dev)
        self._ws = None
        self.grad_buf = torch.empty_like(self.params)
        self.loss_buf = torch.empty(1, dtype=torch.float32, device=dev)

    def pack(self, stream=None):
        check(lib().cdct_cnn_pack(self.params.data_ptr(), self.packed.data_ptr(), stream_handle(stream)))

    def infer(self, img, slots, logits: bool = False, margin: bool = False, stream=None):
        """labels [len(slots), R] uint8 (device); with ``logits`` / ``margin`` also
        [len(slots), R, 17] and [len(slots), R] float32.  Uses the last ``pack``."""
        torch = _torch()
        d = image_desc(img)
        n = RdSearch.region_count(img)
        slots = [int(k) for k in slots]
        sa = (ctypes.c_int32 * len(slots))(*slots)
        lab = torch.empty((len(slots), n), dtype=torch.uint8, device=img.device)
        lg = torch.empty((len(slots), n, CNN_LABELS), dtype=torch.float32, device=img.device) if logits else None
        mg = torch.empty((len(slots), n), dtype=torch.float32, device=img.device) if margin else None
        check(lib().cdct_cnn_infer(self.packed.data_ptr(), ctypes.byref(d), sa, len(slots), lab.data_ptr(),
                                   lg.data_ptr() if logits else None, mg.data_ptr() if margin else None,
                                   stream_handle(stream)))
        out = [lab] + ([lg] if logits else []) + ([mg] if margin else [])
        return out[0] if len(out) == 1 else tuple(out)

    def workspace(self, batch: int):
        torch = _torch()
        n = ctypes.c_size_t()
        check(lib().cdct_cnn_workspace_size(int(batch), ctypes.byref(n)))
        if self._ws is None or self._ws.numel() < n.value:
            self._ws = torch.empty(n.value, dtype=torch.uint8, device=self.params.device)
        return self._ws

    def grad(self, regions, slots, labels, costs=None, mu: float = 0.0, stream=None):
        """(grad [CNN_PARAMS], loss [1]) device tensors for int16 regions [B, 32, 32]
        (B a multiple of 64), labels [len(slots), B] uint8 and, for the regret term,
        the search's partition costs [len(slots), B, 17, 2] (int64 words)."""
        torch = _torch()
        if regions.dtype != torch.int16 or regions.dim() != 3 or tuple(regions.shape[1:]) != (32, 32):
            raise ValueError("regions must be int16 [B, 32, 32]")
        regions = regions.contiguous()
        labels = labels.contiguous()
        B = regions.shape[0]
        slots = [int(k) for k in slots]
        sa = (ctypes.c_int32 * len(slots))(*slots)
        ws = self.workspace(B)
        if costs is not None:
            costs = costs.contiguous()
        check(lib().cdct_cnn_grad(self.params.data_ptr(), regions.data_ptr(), B, sa, len(slots), labels.data_ptr(),
                                  costs.data_ptr() if costs is not None else None, float(mu),
                                  self.grad_buf.data_ptr(), self.loss_buf.data_ptr(), ws.data_ptr(), ws.numel(),
                                  stream_handle(stream)))
        return self.grad_buf, self.loss_buf

    def adam(self, grad, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None):
        self.step += 1
        check(lib().cdct_cnn_adam(self.params.data_ptr(), grad.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                                  self.step, float(lr), float(beta1), float(beta2), float(eps), stream_handle(stream)))

    def train_step(self, regions, slots, labels, lr: float, costs=None, mu: float = 0.0, stream=None):
        """Gradient + Adam update; returns the (device) loss of the batch before the update."""
        g, loss = self.grad(regions, slots, labels, costs, mu, stream)
        self.adam(g, lr, stream=stream)
        return loss

    def save(self, path: str, extra: dict | None = None) -> None:
        """Write the training state (master weights, Adam m and v, step, and an optional
        JSON-able ``extra`` such as the data order's seed) to a checkpoint file."""
        torch = _torch()
        torch.cuda.synchronize(self.params.device)
        write_checkpoint(path, self.params.cpu().numpy(), self.m.cpu().numpy(), self.v.cpu().numpy(), self.step,
                         extra or {})

    @classmethod
    def load(cls, path: str, device="cuda"):
        """(Cnn, extra) restored from a checkpoint written by ``save``; training resumes
        exactly where it stopped (the kernels are deterministic)."""
        torch = _torch()
        params, m, v, step, extra = read_checkpoint(path)
        net = cls(torch.from_numpy(params).to(device))
        net.m.copy_(torch.from_numpy(m))
        net.v.copy_(torch.from_numpy(v))
        net.step = step
        return net, extra


# ---- checkpoint files of the selector's training state ----------------------
# Layout (little-endian): magic b"CDCTCNN1", uint32 version, uint32 parameter
# count, int64 Adam step, uint32 length of a UTF-8 JSON "extra" block, then
# the JSON, then params, m, v as float32 arrays, then a CRC-32 (zlib) of every
# preceding byte.  A file with another magic, version or parameter count, a
# wrong length or a wrong checksum is rejected.
CKPT_MAGIC, CKPT_VERSION = b"CDCTCNN1", 1


class CheckpointError(ValueError):
    pass


def write_checkpoint(path: str, params, m, v, step: int, extra: dict) -> None:
    import json
    import struct
    import zlib

    import numpy as np
    blob = json.dumps(extra, sort_keys=True).encode()
    arrays = [np.ascontiguousarray(a, dtype="<f4") for a in (params, m, v)]
    if any(a.size != CNN_PARAMS for a in arrays):
        raise CheckpointError("every array must hold CNN_PARAMS values")
    body = (CKPT_MAGIC + struct.pack("<IIqI", CKPT_VERSION, CNN_PARAMS, int(step), len(blob)) + blob +
            b"".join(a.tobytes() for a in arrays))
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        f.write(body + struct.pack("<I", zlib.crc32(body) & 0xFFFFFFFF))
    os.replace(tmp, path)


def read_checkpoint(path: str):
    """(params, m, v, step, extra) of a checkpoint file; raises CheckpointError if it is invalid."""
    import json
    import struct
    import zlib

    import numpy as np
    with open(path, "rb") as f:
        data = f.read()
    head = len(CKPT_MAGIC) + struct.calcsize("<IIqI")
    if len(data) < head + 4 or data[:len(CKPT_MAGIC)] != CKPT_MAGIC:
        raise CheckpointError("not a selector checkpoint (magic)")
    version, count, step, nblob = struct.unpack_from("<IIqI", data, len(CKPT_MAGIC))
    if version != CKPT_VERSION or count != CNN_PARAMS:
        raise CheckpointError(f"unsupported checkpoint version {version} or parameter count {count}")
    if len(data) != head + nblob + 3 * 4 * count + 4:
        raise CheckpointError("truncated or oversized checkpoint")
    (crc,) = struct.unpack_from("<I", data, len(data) - 4)
    if zlib.crc32(data[:-4]) & 0xFFFFFFFF != crc:
        raise CheckpointError("checkpoint checksum mismatch")
    extra = json.loads(data[head:head + nblob].decode())
    off = head + nblob
    arrs = [np.frombuffer(data, dtype="<f4", count=count, offset=off + k * 4 * count).astype(np.float32)
            for k in range(3)]
    return arrs[0], arrs[1], arrs[2], int(step), extra
