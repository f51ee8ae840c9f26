"""The video-frame workload: 64 frames of 1920x1080 4:2:0 int16 residuals.

One step is one pass of the whole hot path over the batch for every
transform the workload names: N in {8, 16, 32} x {T~, T^}, each a fused
forward -> zonal(r = N^2/4) -> inverse -> per-plane PSNR launch over the
luma planes and one over the chroma planes.  Inputs are generated on the
host by ``synth`` and copied to the device once; outputs are overwritten each
pass (the reconstructions of the last pass remain), the PSNRs of every pass
are kept.
"""
from __future__ import annotations

import numpy as np

from . import binding as b
from . import synth

FRAMES, HEIGHT, WIDTH = 64, 1080, 1920
PASSES = tuple((n, v) for n in (8, 16, 32) for v in ("tilde", "hat"))


def zonal_r(n: int) -> int:
    return n * n // 4


def host_batch(frames: int = FRAMES, height: int = HEIGHT, width: int = WIDTH, seed: int = 2):
    """(luma [F, H, W], chroma [2F, H/2, W/2]) int16 residuals in [-255, 255]."""
    return synth.residual_frames_420(frames, height, width, seed)


def pixels(luma: np.ndarray, chroma: np.ndarray) -> int:
    return int(luma.size + chroma.size)


class FrameStep:
    """Device buffers, plans and launches of one step over a resident batch."""

    def __init__(self, luma_dev, chroma_dev, passes=PASSES, conv: str = "paper", per_pass_outputs: bool = False):
        """``per_pass_outputs``: every pass writes its own reconstruction buffers
        (``recon_y_of[p]``, ``recon_c_of[p]``) instead of overwriting one pair."""
        import torch
        self.torch = torch
        self.luma, self.chroma = luma_dev, chroma_dev
        self.passes = passes
        self.plans = {p: b.Plan(p[0], p[1], conv) for p in passes}
        dev = luma_dev.device
        self.recon_y = torch.empty(luma_dev.shape, dtype=torch.float32, device=dev)
        self.recon_c = torch.empty(chroma_dev.shape, dtype=torch.float32, device=dev)
        self.recon_y_of = {p: self.recon_y for p in passes}
        self.recon_c_of = {p: self.recon_c for p in passes}
        if per_pass_outputs:
            for p in passes[1:]:
                self.recon_y_of[p] = torch.empty_like(self.recon_y)
                self.recon_c_of[p] = torch.empty_like(self.recon_c)
        self.psnr_y = {p: torch.empty(luma_dev.shape[0], dtype=torch.float64, device=dev) for p in passes}
        self.psnr_c = {p: torch.empty(chroma_dev.shape[0], dtype=torch.float64, device=dev) for p in passes}
        ws = max(max(self.plans[p].workspace_size(luma_dev), self.plans[p].workspace_size(chroma_dev))
                 for p in passes)
        self.ws = torch.empty(ws // 8 + 1, dtype=torch.float64, device=dev)
        self.npix = int(luma_dev.numel() + chroma_dev.numel())

    def launch_pass(self, p, stream=None):
        plan = self.plans[p]
        r = zonal_r(p[0])
        plan.fwd_zonal_inv(self.luma, r, out=self.recon_y_of[p], psnr_out=self.psnr_y[p], workspace=self.ws,
                           stream=stream)
        plan.fwd_zonal_inv(self.chroma, r, out=self.recon_c_of[p], psnr_out=self.psnr_c[p], workspace=self.ws,
                           stream=stream)

    def run(self, stream=None, events=None, after_pass=None):
        """One step.  ``events``: optional list receiving (start, end, npix) per fused pass.
        ``after_pass(p)``: optional callback after each pass is enqueued."""
        for p in self.passes:
            if events is not None:
                s = self.torch.cuda.Event(enable_timing=True)
                e = self.torch.cuda.Event(enable_timing=True)
                s.record(stream)
                self.launch_pass(p, stream)
                e.record(stream)
                events.append((s, e, p))
            else:
                self.launch_pass(p, stream)
            if after_pass is not None:
                after_pass(p)

    # launches per step of the library's own kernels: fused + finalize, two planes, per pass
    @property
    def launches_per_step(self) -> int:
        return 4 * len(self.passes)

    def psnr_host(self):
        """{pass: (luma PSNRs, chroma PSNRs)} as numpy arrays (synchronises)."""
        return {p: (self.psnr_y[p].cpu().numpy(), self.psnr_c[p].cpu().numpy()) for p in self.passes}
