"""Utility metrics and edge-based region masks, written plainly in numpy (fp64 / exact integers).

TEST INFRASTRUCTURE ONLY: used by tests/ and the benchmark's CPU-baseline leg, never by the product path.

- MSE and SSIM are the two utility measures of the paper's experiments (Sec. VII-A and VII-B: image
  fidelity of the released frames against the originals).  SSIM is Wang et al.'s structural similarity
  (IEEE TIP 2004) evaluated as the paper's toolkit does by default: local statistics over every 7 x 7
  window that lies inside the image (uniform weights, sample variances and covariance with the 1/(n-1)
  normalisation), constants C1 = (0.01 L)^2 and C2 = (0.03 L)^2 with L = 255, the mean over the windows;
  for several channels the mean over channels.
- The edge mask follows the paper's pointer to the Sobel operator for finding complex regions (Sec. VI-A):
  the intensity is the channel sum, the two 3 x 3 Sobel responses are taken with the frame mirrored at
  its borders, and a pixel is complex when Gx^2 + Gy^2 >= tau.  The mask holds 1 for simple pixels and 0
  for complex ones (the release's simple-mask convention).
"""
import numpy as np

REFLECT, SYMMETRIC = 0, 1


def _pad_mode(pad_mode):
    return "reflect" if pad_mode == REFLECT else "symmetric"


def sobel_responses(frame, pad_mode=REFLECT):
    """Gx, Gy (int64) of the channel-sum intensity of an M x N x C u8 frame, borders mirrored.

    Gx is the horizontal derivative (right column minus left column, rows weighted 1, 2, 1); Gy the vertical
    one (bottom row minus top row, columns weighted 1, 2, 1)."""
    f = np.asarray(frame)
    if f.ndim == 2:
        f = f[:, :, None]
    inten = f.astype(np.int64).sum(axis=2)
    p = np.pad(inten, 1, mode=_pad_mode(pad_mode))
    M, N = inten.shape
    gx = np.zeros((M, N), np.int64)
    gy = np.zeros((M, N), np.int64)
    # the 3 x 3 kernels written out tap by tap: weight w at offset (dy, dx)
    for dy, wy in ((-1, 1), (0, 2), (1, 1)):
        gx += wy * (p[1 + dy:1 + dy + M, 2:2 + N] - p[1 + dy:1 + dy + M, 0:N])
    for dx, wx in ((-1, 1), (0, 2), (1, 1)):
        gy += wx * (p[2:2 + M, 1 + dx:1 + dx + N] - p[0:M, 1 + dx:1 + dx + N])
    return gx, gy


def sobel_mask(frame, tau, pad_mode=REFLECT):
    """u8 M x N mask: 1 where Gx^2 + Gy^2 < tau (simple), 0 where it is >= tau (complex)."""
    gx, gy = sobel_responses(frame, pad_mode)
    return ((gx * gx + gy * gy) < int(tau)).astype(np.uint8)


def sse(x, y):
    """Exact sum of squared sample differences of two u8 images of the same shape (Python int)."""
    d = np.asarray(x).astype(np.int64) - np.asarray(y).astype(np.int64)
    return int((d * d).sum())


def mse(x, y):
    """Mean squared error over all samples."""
    return sse(x, y) / float(np.asarray(x).size)


def ssim_channel(x, y, L=255.0, win=7):
    """Mean SSIM of one channel (2-D arrays) over all win x win windows inside the image (fp64)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    M, N = x.shape
    if M < win or N < win:
        raise ValueError("image smaller than the window")
    C1 = (0.01 * L) ** 2
    C2 = (0.03 * L) ** 2
    n = win * win
    total = 0.0
    count = 0
    for i in range(M - win + 1):
        for j in range(N - win + 1):
            a = x[i:i + win, j:j + win]
            b = y[i:i + win, j:j + win]
            mx, my = a.mean(), b.mean()
            vx = ((a - mx) ** 2).sum() / (n - 1)
            vy = ((b - my) ** 2).sum() / (n - 1)
            cxy = ((a - mx) * (b - my)).sum() / (n - 1)
            total += ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))
            count += 1
    return total / count, count


def ssim(x, y, L=255.0, win=7):
    """Mean SSIM of two M x N (x C) images: the mean over channels of each channel's window mean."""
    x = np.asarray(x)
    y = np.asarray(y)
    if x.ndim == 2:
        return ssim_channel(x, y, L, win)[0]
    vals = [ssim_channel(x[:, :, c], y[:, :, c], L, win)[0] for c in range(x.shape[2])]
    return float(np.mean(vals))
