"""Python binding of the differentiable soft layer (dp_pix_soft_*): y = w * P~_{b0}(x) + (1 - w) * P~_{b1}(x)
as a torch.autograd.Function whose forward and backward are the library's CUDA kernels.  The noise is a
constant of the layer (the backward sees the forward's draws)."""
from __future__ import annotations

import ctypes as ct
from typing import Optional, Sequence

import torch

from . import _lib as L

__all__ = ["SoftSpec", "soft_forward", "soft_backward", "SoftPixelize", "soft_pixelize"]


class SoftSpec:
    """Parameters of the layer (everything except the tensors)."""

    def __init__(self, grids: Sequence[int] = (8, 16), eps: Sequence[float] = (0.5, 1.0), R: float = 1.0,
                 m: float = 16.0, pad_mode: int = L.PAD_REFLECT, noise_free: bool = False, stream_id: int = 0,
                 seed: int = 0, frame0: int = 0):
        self.grids, self.eps = tuple(int(b) for b in grids), tuple(float(e) for e in eps)
        if len(self.grids) != 2 or len(self.eps) != 2:
            raise ValueError("the soft layer mixes exactly two grids")
        self.R, self.m, self.pad_mode = float(R), float(m), int(pad_mode)
        self.noise_free, self.stream_id = bool(noise_free), int(stream_id)
        self.seed, self.frame0 = int(seed) & (2**64 - 1), int(frame0) & (2**64 - 1)

    def desc(self, x: torch.Tensor) -> L.SoftDesc:
        if x.dim() != 4:
            raise ValueError("x must be [B, C, H, W]")
        d = L.SoftDesc()
        d.B, d.C, d.H, d.W = (int(v) for v in x.shape)
        d.grid[0], d.grid[1] = self.grids
        d.eps[0], d.eps[1] = self.eps
        d.value_range, d.m, d.pad_mode, d.noise_free = self.R, self.m, self.pad_mode, int(self.noise_free)
        d.stream_id, d.seed, d.frame0 = self.stream_id, self.seed, self.frame0
        return d


def _p(t: Optional[torch.Tensor]):
    return None if t is None else ct.c_void_p(t.data_ptr())


def _check_f32(*ts):
    for t in ts:
        if t.device.type != "cuda" or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError("soft layer tensors must be contiguous float32 CUDA tensors")


def _pre_numel(d: L.SoftDesc) -> int:
    nb = ct.c_uint64(0)
    L.check(L.lib().dp_pix_soft_sizes(ct.byref(d), ct.byref(nb)), "dp_pix_soft_sizes")
    return int(nb.value) // 4


def soft_forward(x: torch.Tensor, w: torch.Tensor, spec: SoftSpec, stream=None):
    """Returns (y [B, C, H, W], pre: the unclipped noisy cell means the backward needs)."""
    _check_f32(x, w)
    if w.shape != (x.shape[0], 1, x.shape[2], x.shape[3]):
        raise ValueError("w must be [B, 1, H, W]")
    d = spec.desc(x)
    pre = torch.empty(_pre_numel(d), dtype=torch.float32, device=x.device)
    y = torch.empty_like(x)
    s = ct.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    L.check(L.lib().dp_pix_soft_forward(ct.byref(d), _p(x), _p(w), _p(y), _p(pre), s), "dp_pix_soft_forward")
    return y, pre


def soft_backward(w: torch.Tensor, gy: torch.Tensor, pre: torch.Tensor, spec: SoftSpec, stream=None):
    """Returns (dx [B, C, H, W], dw [B, 1, H, W]) for dL/dy = gy."""
    _check_f32(w, gy, pre)
    d = spec.desc(gy)
    dx = torch.empty_like(gy)
    dw = torch.empty_like(w)
    ws = torch.empty(_pre_numel(d), dtype=torch.float32, device=gy.device)
    s = ct.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    L.check(L.lib().dp_pix_soft_backward(ct.byref(d), _p(w), _p(gy), _p(pre), _p(dx), _p(dw), _p(ws), s),
            "dp_pix_soft_backward")
    return dx, dw


class SoftPixelize(torch.autograd.Function):
    """autograd wrapper: forward and backward run in the library's kernels."""

    @staticmethod
    def forward(ctx, x, w, spec: SoftSpec):
        x, w = x.contiguous(), w.contiguous()
        y, pre = soft_forward(x, w, spec)
        ctx.save_for_backward(w, pre)
        ctx.spec = spec
        return y

    @staticmethod
    def backward(ctx, gy):
        w, pre = ctx.saved_tensors
        dx, dw = soft_backward(w, gy.contiguous(), pre, ctx.spec)
        return dx, dw, None


def soft_pixelize(x: torch.Tensor, w: torch.Tensor, spec: Optional[SoftSpec] = None, **kw) -> torch.Tensor:
    """y = w * P~_{b0}(x) + (1 - w) * P~_{b1}(x), differentiable in x and w (noise held constant)."""
    return SoftPixelize.apply(x, w, spec if spec is not None else SoftSpec(**kw))
