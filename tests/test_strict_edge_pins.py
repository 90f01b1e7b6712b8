"""Pins of the oracle's privacy-strict edge mode (pad mode 2: no padding; a cell on the frame's edge uses
only its h x w samples inside the frame, mean over them, noise scale R m / (h w eps) -- Alg. 1's partial
cells).  CPU only."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O


def _valid_block_stats(img, b):
    """Per-cell sums and counts of a uniform b-grid over the unpadded image (numpy reduceat)."""
    M, N, C = img.shape
    ys, xs = np.arange(0, M, b), np.arange(0, N, b)
    sums = np.add.reduceat(np.add.reduceat(img.astype(np.int64), ys, axis=0), xs, axis=1)
    h = np.minimum(b, M - ys)[:, None]
    w = np.minimum(b, N - xs)[None, :]
    return sums, h * w


@pytest.mark.parametrize("M,N,b", [(37, 53, 8), (16, 16, 8), (5, 7, 8), (61, 77, 6)])
def test_sums_and_means_over_valid_samples(M, N, b):
    rng = np.random.default_rng(M * N + b)
    img = rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8)
    lab = np.zeros((-(-M // b), -(-N // b)), np.uint8)
    kw = dict(grids=[b], eps=[1.0], source=O.SRC_TILE_LABELS, pad_mode=O.PAD_NONE)
    rec, means, sums, eta = O.release(img, lab, dtype=O.DT_SUM, **kw)
    exp_sums, n = _valid_block_stats(img, b)
    np.testing.assert_array_equal(sums.reshape(exp_sums.shape), exp_sums)
    rec, means, sums, eta = O.release(img, lab, dtype=O.DT_F32, noise_free=True, **kw)
    np.testing.assert_allclose(means.reshape(exp_sums.shape), exp_sums / n[:, :, None], rtol=0, atol=1e-12)
    # the reconstruction paints each cell's mean over its own pixels only
    got = O.reconstruct(rec, out_type=2)
    exp_img = np.repeat(np.repeat(exp_sums / n[:, :, None], b, axis=0), b, axis=1)[:M, :N]
    np.testing.assert_allclose(got, exp_img, rtol=0, atol=255 * 2**-24)


def test_edge_noise_scale_follows_valid_count():
    # residuals of edge cells, divided by R m / (h w eps), are standard Laplace draws; a b^2 divisor would
    # make them n / b^2 times too small
    M, N, b, eps, m = 1003, 1005, 8, 0.5, 16.0
    img = np.full((M, N, 1), 100, np.uint8)
    lab = np.zeros((-(-M // b), -(-N // b)), np.uint8)
    rec, means, sums, eta = O.release(img, lab, grids=[b], eps=[eps], m=m, C=1, source=O.SRC_TILE_LABELS,
                                      pad_mode=O.PAD_NONE, seed=9)
    _, n = _valid_block_stats(img, b)
    n = n.reshape(-1).astype(np.float64)
    z = eta / (255.0 * m / (n * eps))
    edge = n < b * b
    assert edge.sum() > 200
    assert stats.kstest(z[edge], stats.laplace.cdf).pvalue > 0.01
    assert stats.kstest(z[~edge], stats.laplace.cdf).pvalue > 0.01
    assert abs(np.mean(np.abs(z[edge])) - 1.0) < 0.1


def test_mask_tiles_classified_on_valid_pixels():
    rng = np.random.default_rng(4)
    M, N, T = 50, 70, 24
    mask = (rng.random((M, N)) < 0.5).astype(np.uint8)
    img = rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8)
    rec, *_ = O.release(img, mask, grids=[24, 8], eps=[1, 1], source=O.SRC_MASK, pad_mode=O.PAD_NONE)
    got = O.record_map(rec).reshape(-(-M // T), -(-N // T))
    for ty in range(got.shape[0]):
        for tx in range(got.shape[1]):
            part = mask[ty * T:(ty + 1) * T, tx * T:(tx + 1) * T]
            assert got[ty, tx] == (0 if 2 * int(part.sum()) > part.size else 1)


def test_no_padding_limit_and_variance_rejected():
    # padding beyond the frame's own extent is fine without mirroring (reflect needs P <= M - 1: 5 > 2 here)
    img = np.zeros((3, 7, 3), np.uint8)
    O.release(img, np.zeros((1, 1), np.uint8), grids=[8], eps=[1], source=O.SRC_TILE_LABELS, pad_mode=O.PAD_NONE)
    assert O.geometry_rc(M=3, N=7, C=3, grids=[8], eps=[1], pad_mode=O.PAD_REFLECT) != 0
    assert O.geometry_rc(M=64, N=64, C=3, grids=[8, 16], eps=[1, 1], source=O.SRC_VARIANCE, pad_mode=O.PAD_NONE) != 0


def test_interior_cells_match_mirror_mode():
    # cells wholly inside the frame do not see the padding: same sums, noise and values in every mode
    rng = np.random.default_rng(8)
    M, N, b = 40, 44, 8
    img = rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8)
    lab = np.zeros((5, 6), np.uint8)
    a = O.release(img, lab, grids=[b], eps=[0.7], source=O.SRC_TILE_LABELS, pad_mode=O.PAD_NONE, seed=3)
    r = O.release(img, lab, grids=[b], eps=[0.7], source=O.SRC_TILE_LABELS, pad_mode=O.PAD_REFLECT, seed=3)
    cells = np.arange(5 * 6)
    inner = (cells % 6) < 5  # the last cell column (x 40..47) crosses the right edge
    for arr_a, arr_r in zip(a[1:], r[1:]):
        np.testing.assert_array_equal(arr_a.reshape(30, 3)[inner], arr_r.reshape(30, 3)[inner])
