"""Binding of the utility metrics and the edge mask (dp_pix_utility, dp_pix_sobel_mask): argument
marshalling only; the work runs in the library's kernels."""
from __future__ import annotations

import ctypes as ct
from typing import Optional

import torch

from . import _lib as L
from .api import _ptr, _stream_handle


def _frames(t: torch.Tensor) -> torch.Tensor:
    """[n,] M x N [x C] u8 CUDA tensor -> 4-D view [n, M, N, C] with unit element and channel strides."""
    if t.dtype != torch.uint8 or not t.is_cuda:
        raise ValueError("frames must be a uint8 CUDA tensor")
    if t.dim() == 2:
        t = t[None, :, :, None]
    elif t.dim() == 3:
        t = t[None]
    if t.dim() != 4 or t.stride(3) != 1 or t.stride(2) != t.shape[3]:
        raise ValueError("frames must be [n,] M x N [x C] with contiguous pixels")
    return t


def dp_pix_sobel_mask(frames: torch.Tensor, tau: int, pad_mode: int = L.PAD_REFLECT,
                      out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """u8 masks [n, M, N]: 1 where the squared Sobel gradient of the channel-sum intensity is < tau."""
    f = _frames(frames)
    n, M, N, C = f.shape
    if out is None:
        out = torch.empty((n, M, N), dtype=torch.uint8, device=f.device)
    L.check(L.lib().dp_pix_sobel_mask(_ptr(f), M, N, C, f.stride(1), f.stride(0), n, int(pad_mode), int(tau),
                                      _ptr(out), out.stride(-2), out.stride(0) if out.dim() == 3 else M * out.stride(-2),
                                      _stream_handle(stream)), "dp_pix_sobel_mask")
    return out


def dp_pix_utility(x: torch.Tensor, y: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Per-frame (sse, windows, ssim_sum, mse, ssim) of release y against original x, as a device buffer of
    dp_pix_utility_t records (use utility_values() to read them)."""
    a, b = _frames(x), _frames(y)
    if a.shape != b.shape:
        raise ValueError("x and y differ in shape")
    n, M, N, C = a.shape
    if out is None:
        out = torch.empty((n, ct.sizeof(L.Utility)), dtype=torch.uint8, device=a.device)
    L.check(L.lib().dp_pix_utility(_ptr(a), _ptr(b), M, N, C, a.stride(1), b.stride(1), a.stride(0), b.stride(0), n,
                                   _ptr(out), _stream_handle(stream)), "dp_pix_utility")
    return out


def utility_values(buf: torch.Tensor) -> list:
    """Host copy of dp_pix_utility's records as dicts."""
    raw = buf.cpu().contiguous().numpy().tobytes()
    size = ct.sizeof(L.Utility)
    res = []
    for i in range(len(raw) // size):
        u = L.Utility.from_buffer_copy(raw[i * size:(i + 1) * size])
        res.append({"sse": u.sse, "windows": u.windows, "ssim_sum": u.ssim_sum, "mse": u.mse, "ssim": u.ssim})
    return res
