"""Pins of the oracle's utility metrics and edge mask (oracle/utility.py) against library routines,
closed forms and invariants (CPU only)."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import utility as U

SCIPY_MODE = {U.REFLECT: "mirror", U.SYMMETRIC: "reflect"}  # scipy's names for numpy's reflect / symmetric


@pytest.mark.parametrize("C", [1, 3])
@pytest.mark.parametrize("mode", [U.REFLECT, U.SYMMETRIC])
def test_sobel_responses_match_scipy(C, mode):
    rng = np.random.default_rng(11 + C + 7 * mode)
    f = rng.integers(0, 256, size=(23, 37, C), dtype=np.uint8)
    gx, gy = U.sobel_responses(f, mode)
    inten = f.astype(np.int64).sum(axis=2)
    np.testing.assert_array_equal(gx, ndimage.sobel(inten, axis=1, mode=SCIPY_MODE[mode]))
    np.testing.assert_array_equal(gy, ndimage.sobel(inten, axis=0, mode=SCIPY_MODE[mode]))


def test_sobel_step_edge_closed_form():
    # a vertical step from 0 to 255 between columns 9 and 10: |Gx| = (1 + 2 + 1) * 255 on both sides of it,
    # 0 elsewhere in the interior; Gy = 0 everywhere
    f = np.zeros((12, 20, 1), np.uint8)
    f[:, 10:] = 255
    gx, gy = U.sobel_responses(f)
    assert (gy == 0).all()
    assert (gx[:, 9] == 1020).all() and (gx[:, 10] == 1020).all()
    assert (gx[:, 1:9] == 0).all() and (gx[:, 11:19] == 0).all()
    m = U.sobel_mask(f, 1020 * 1020)
    assert (m[:, 9:11] == 0).all() and (m[:, :9] == 1).all() and (m[:, 11:] == 1).all()
    assert (U.sobel_mask(f, 1020 * 1020 + 1) == 1).all()


def test_sobel_mask_threshold_extremes():
    rng = np.random.default_rng(3)
    f = rng.integers(0, 256, size=(9, 14, 3), dtype=np.uint8)
    assert (U.sobel_mask(f, 0) == 0).all()                  # every squared gradient is >= 0
    assert (U.sobel_mask(f, 2**40) == 1).all()
    flat = np.full((9, 14, 3), 77, np.uint8)
    assert (U.sobel_mask(flat, 1) == 1).all()               # no gradient anywhere


def test_mse_closed_forms():
    rng = np.random.default_rng(5)
    x = rng.integers(0, 200, size=(17, 19, 3), dtype=np.uint8)
    assert U.mse(x, x) == 0.0
    assert U.mse(x, x + np.uint8(13)) == 169.0
    y = x.copy()
    y[3, 4, 1] += 10
    assert U.sse(x, y) == 100 and U.mse(x, y) == 100.0 / x.size


def test_ssim_identity_and_symmetry():
    rng = np.random.default_rng(9)
    x = rng.integers(0, 256, size=(15, 18), dtype=np.uint8)
    y = rng.integers(0, 256, size=(15, 18), dtype=np.uint8)
    assert U.ssim(x, x) == pytest.approx(1.0, abs=1e-12)
    assert U.ssim(x, y) == pytest.approx(U.ssim(y, x), abs=1e-12)
    assert U.ssim(x, y) < 0.5


def test_ssim_constant_images_closed_form():
    # both images constant: variances and covariance vanish, each window is (2ab + C1) / (a^2 + b^2 + C1)
    a, b = 120.0, 150.0
    C1 = (0.01 * 255) ** 2
    x = np.full((10, 12), a, np.uint8)
    y = np.full((10, 12), b, np.uint8)
    assert U.ssim(x, y) == pytest.approx((2 * a * b + C1) / (a * a + b * b + C1), rel=1e-12)
    val, count = U.ssim_channel(x, y)
    assert count == (10 - 6) * (12 - 6)


def _ssim_by_filters(x, y, L=255.0, win=7):
    """The same statistic by a different route: uniform filters for the local moments (scipy), scaled to
    sample statistics, cropped to the windows inside the image."""
    x = x.astype(np.float64)
    y = y.astype(np.float64)
    C1, C2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    n = win * win
    ux, uy = ndimage.uniform_filter(x, win), ndimage.uniform_filter(y, win)
    uxx, uyy, uxy = (ndimage.uniform_filter(v, win) for v in (x * x, y * y, x * y))
    vx, vy, vxy = (n / (n - 1)) * (uxx - ux * ux), (n / (n - 1)) * (uyy - uy * uy), (n / (n - 1)) * (uxy - ux * uy)
    s = ((2 * ux * uy + C1) * (2 * vxy + C2)) / ((ux * ux + uy * uy + C1) * (vx + vy + C2))
    p = win // 2
    return s[p:-p, p:-p].mean()


@pytest.mark.parametrize("shape", [(7, 7), (12, 9), (21, 30)])
def test_ssim_matches_filter_route(shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.integers(0, 256, size=shape, dtype=np.uint8)
    noise = rng.integers(-40, 41, size=shape)
    y = np.clip(x.astype(np.int64) + noise, 0, 255).astype(np.uint8)
    assert U.ssim(x, y) == pytest.approx(_ssim_by_filters(x, y), abs=1e-10)


def test_ssim_channels_are_averaged():
    rng = np.random.default_rng(21)
    x = rng.integers(0, 256, size=(11, 13, 3), dtype=np.uint8)
    y = rng.integers(0, 256, size=(11, 13, 3), dtype=np.uint8)
    per = [U.ssim(x[:, :, c], y[:, :, c]) for c in range(3)]
    assert U.ssim(x, y) == pytest.approx(np.mean(per), abs=1e-12)
