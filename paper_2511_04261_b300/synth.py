"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs; it holds none of the pixelization arithmetic and imports neither the
CUDA path nor the oracle, so both can be fed from it.  The datasets the paper measures on (PETS09-S2L1
768x576, Venice-2 1920x1080, PPM-100 portraits with alpha mattes, CelebA) are not available; these
generators copy their shapes, value ranges and region structure instead.

All draws come from numpy's PCG64 (`default_rng(seed)`), in a fixed order, so a seed fixes the input.
Values are rounded half to even and clipped to [0, 255] before the uint8 cast.
"""
from __future__ import annotations

import numpy as np
from scipy.special import ndtr

__all__ = [
    "gradient_background", "rect_frame", "moving_rect_clip", "portrait", "portrait_batch_shapes",
    "soft_batch", "camera_pool", "random_frame", "portrait_device",
]


def _to_u8(a: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(a), 0, 255).astype(np.uint8)


def gradient_background(rng: np.random.Generator, M: int, N: int, C: int = 3) -> np.ndarray:
    """Smooth linear gradient per channel: a_c + g_c * x/(N-1) + h_c * y/(M-1), a in U[30,120],
    g, h in U[-60, 90].  Returns float32 [M, N, C] (noise is added by the callers)."""
    a = rng.uniform(30, 120, size=C)
    g = rng.uniform(-60, 90, size=C)
    h = rng.uniform(-60, 90, size=C)
    xs = np.arange(N, dtype=np.float64) / max(N - 1, 1)
    ys = np.arange(M, dtype=np.float64) / max(M - 1, 1)
    bg = a[None, None, :] + g[None, None, :] * xs[None, :, None] + h[None, None, :] * ys[:, None, None]
    return bg.astype(np.float32)


def _draw_rects(rng, M, N, count, C):
    rects = []
    for _ in range(count):
        w = int(rng.integers(40, 121))
        h = int(rng.integers(100, 301))
        w, h = min(w, N), min(h, M)
        x0 = int(rng.integers(0, N - w + 1))
        y0 = int(rng.integers(0, M - h + 1))
        tex = rng.integers(0, 256, size=(h, w, C), dtype=np.uint8)
        rects.append([y0, x0, h, w, tex])
    return rects


def rect_frame(seed: int = 1001, M: int = 576, N: int = 768, C: int = 3, n_rects: int = 6):
    """One frame: gradient background + N(0, 6^2) noise, with `n_rects` rectangles (40-120 px wide,
    100-300 px tall, uniformly placed inside the frame) of i.i.d. uniform 0..255 texture; a later rectangle
    wins on overlap.  Returns (image u8 [M, N, C], simple-region mask u8 [M, N] with 1 = background)."""
    rng = np.random.default_rng(seed)
    bg = gradient_background(rng, M, N, C)
    img = bg + rng.normal(0.0, 6.0, size=(M, N, C)).astype(np.float32)
    img = _to_u8(img)
    fg = np.zeros((M, N), dtype=bool)
    for y0, x0, h, w, tex in _draw_rects(rng, M, N, n_rects, C):
        img[y0:y0 + h, x0:x0 + w] = tex
        fg[y0:y0 + h, x0:x0 + w] = True
    return img, (~fg).astype(np.uint8)


def moving_rect_clip(seed: int = 1002, frames: int = 64, M: int = 1080, N: int = 1920, C: int = 3,
                     out: np.ndarray | None = None) -> np.ndarray:
    """A clip: fixed gradient background with fresh N(0, 6^2) noise per frame, and 10-30 rectangles
    (drawn once, fixed texture) that move by a seeded random walk of dx, dy in U{-8..8} per frame,
    clamped inside the frame.  Returns u8 [frames, M, N, C] (written into `out` if given)."""
    rng = np.random.default_rng(seed)
    bg = gradient_background(rng, M, N, C)
    n_rects = int(rng.integers(10, 31))
    rects = _draw_rects(rng, M, N, n_rects, C)
    if out is None:
        out = np.empty((frames, M, N, C), dtype=np.uint8)
    for f in range(frames):
        noise = rng.standard_normal(size=(M, N, C), dtype=np.float32) * np.float32(6.0)
        fr = _to_u8(bg + noise)
        for r in rects:
            y0, x0, h, w, tex = r
            fr[y0:y0 + h, x0:x0 + w] = tex
        out[f] = fr
        for r in rects:  # random walk for the next frame
            dy, dx = rng.integers(-8, 9, size=2)
            r[0] = int(np.clip(r[0] + dy, 0, M - r[2]))
            r[1] = int(np.clip(r[1] + dx, 0, N - r[3]))
    return out


def portrait(rng: np.random.Generator, H: int, W: int, C: int = 3):
    """Portrait-like image: gradient background (+ N(0, 6^2)), an elliptical subject (center within +-10%
    of the image center, semi-axes U[0.2, 0.35] * H and * W) of mean-128 texture with N(0, 40^2), and a
    soft alpha matte in [0, 1]: the ellipse indicator blurred by a Gaussian of std 0.01 * min(H, W) px,
    taken in the closed form Phi(d / s) of a blurred edge at signed distance d (first-order distance to
    the ellipse).  Composite = alpha * subject + (1 - alpha) * background.
    Returns (image u8 [H, W, C], alpha f32 [H, W])."""
    bg = gradient_background(rng, H, W, C)
    cy = H / 2 * (1 + rng.uniform(-0.1, 0.1))
    cx = W / 2 * (1 + rng.uniform(-0.1, 0.1))
    ay = rng.uniform(0.2, 0.35) * H
    ax = rng.uniform(0.2, 0.35) * W
    s = 0.01 * min(H, W)
    ys = (np.arange(H, dtype=np.float64) + 0.5 - cy)[:, None]
    xs = (np.arange(W, dtype=np.float64) + 0.5 - cx)[None, :]
    rho = np.sqrt((ys / ay) ** 2 + (xs / ax) ** 2)
    grad = np.sqrt((ys / ay**2) ** 2 + (xs / ax**2) ** 2) / np.maximum(rho, 1e-12)
    dist = (1.0 - rho) / np.maximum(grad, 1e-12)  # > 0 inside
    alpha = ndtr(dist / s).astype(np.float32)
    subject = 128.0 + rng.normal(0.0, 40.0, size=(H, W, C)).astype(np.float32)
    noise = rng.normal(0.0, 6.0, size=(H, W, C)).astype(np.float32)
    a3 = alpha[:, :, None]
    img = a3 * subject + (1.0 - a3) * (bg + noise)
    return _to_u8(img), alpha


def portrait_batch_shapes(seed: int = 1003, n: int = 256, lo: int = 512, hi: int = 4096):
    """Image sides of the ragged batch: H, W independently uniform in {lo..hi}."""
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(lo, hi + 1)), int(rng.integers(lo, hi + 1))) for _ in range(n)]


def soft_batch(seed: int = 1004, B: int = 32, H: int = 1024, W: int = 1024, C: int = 3, grad_seed: int = 1005):
    """Differentiable-layer inputs: x = portrait image / 255 as f32 [B, C, H, W] in [0, 1], soft weights
    w = the portrait's alpha matte f32 [B, 1, H, W], and an upstream gradient g ~ N(0, 1) [B, C, H, W]."""
    rng = np.random.default_rng(seed)
    x = np.empty((B, C, H, W), dtype=np.float32)
    w = np.empty((B, 1, H, W), dtype=np.float32)
    for i in range(B):
        img, alpha = portrait(rng, H, W, C)
        x[i] = np.transpose(img, (2, 0, 1)).astype(np.float32) / np.float32(255.0)
        w[i, 0] = alpha
    g = np.random.default_rng(grad_seed).standard_normal(size=(B, C, H, W), dtype=np.float32)
    return x, w, g


def camera_pool(seed: int, M: int, N: int, pool: int = 32, C: int = 3) -> np.ndarray:
    """Pre-generated frames of one simulated camera (moving-rectangle clip), cycled by the server."""
    return moving_rect_clip(seed=seed, frames=pool, M=M, N=N, C=C)


def random_frame(seed: int, M: int, N: int, C: int = 3, pitch: int | None = None) -> np.ndarray:
    """Uniform random u8 frame for parity tests; with `pitch` the rows are padded (extra bytes random)."""
    rng = np.random.default_rng(seed)
    if pitch is None:
        return rng.integers(0, 256, size=(M, N, C), dtype=np.uint8)
    buf = rng.integers(0, 256, size=(M, pitch), dtype=np.uint8)
    return buf


def portrait_device(seed: int, H: int, W: int, C: int = 3, device="cuda"):
    """The portrait generator's distribution drawn on the GPU with torch (for the 256-image ragged batch,
    whose 1.36 Gpx would take minutes in numpy): same background, subject, noise and matte recipe as
    `portrait`, from torch's Philox generator seeded with `seed` (values differ from `portrait`'s).
    Returns (image u8 [H, W, C], alpha f32 [H, W]) on `device`."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))

    def u(lo, hi, n=1):
        return lo + (hi - lo) * torch.rand(n, generator=gen, device=device, dtype=torch.float64)

    a, g, h = u(30, 120, C), u(-60, 90, C), u(-60, 90, C)
    xs = torch.arange(W, device=device, dtype=torch.float64) / max(W - 1, 1)
    ys = torch.arange(H, device=device, dtype=torch.float64) / max(H - 1, 1)
    bg = (a[None, None, :] + g[None, None, :] * xs[None, :, None] + h[None, None, :] * ys[:, None, None]).float()
    cy = H / 2 * (1 + float(u(-0.1, 0.1)))
    cx = W / 2 * (1 + float(u(-0.1, 0.1)))
    ay = float(u(0.2, 0.35)) * H
    ax = float(u(0.2, 0.35)) * W
    s = 0.01 * min(H, W)
    yy = (torch.arange(H, device=device, dtype=torch.float64) + 0.5 - cy)[:, None]
    xx = (torch.arange(W, device=device, dtype=torch.float64) + 0.5 - cx)[None, :]
    rho = torch.sqrt((yy / ay) ** 2 + (xx / ax) ** 2)
    grad = torch.sqrt((yy / ay**2) ** 2 + (xx / ax**2) ** 2) / torch.clamp(rho, min=1e-12)
    dist = (1.0 - rho) / torch.clamp(grad, min=1e-12)
    alpha = torch.special.ndtr(dist / s).float()
    subject = 128.0 + 40.0 * torch.randn((H, W, C), generator=gen, device=device, dtype=torch.float32)
    noise = 6.0 * torch.randn((H, W, C), generator=gen, device=device, dtype=torch.float32)
    a3 = alpha[:, :, None]
    img = a3 * subject + (1.0 - a3) * (bg + noise)
    return torch.clamp(torch.round(img), 0, 255).to(torch.uint8), alpha
