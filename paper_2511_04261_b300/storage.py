"""Host-side storage of released records (Sec. V-D Table III, Sec. VI-F Table IV; the storage study of
Sec. VII-A and VII-B).

The record written by the release is already the compact form the paper stores: the tile map plus the
noisy means (u8 when the plan's record dtype is DP_PIX_REC_U8).  The paper keeps it in a ZIP container
(NPZ); here the record bytes are deflated with zlib, the same compression.  For comparison with storing the
pixelized frame as an image (the paper uses PNG), png_like_bytes applies PNG's "up" row filter and deflate
to the frame, without the container's few dozen bytes of chunk headers.  Host code only: the record is
copied out with dp_pix_store first.
"""
from __future__ import annotations

import zlib

import numpy as np


def deflate_record(record: bytes, level: int = 6) -> bytes:
    """zlib stream of a record's bytes (what dp_pix_store wrote)."""
    return zlib.compress(bytes(record), level)


def inflate_record(blob: bytes) -> bytes:
    return zlib.decompress(blob)


def up_filter(img: np.ndarray) -> np.ndarray:
    """PNG filter type 2 ("up") of an M x N x C u8 image, one filter-type byte in front of each row."""
    a = np.ascontiguousarray(img, dtype=np.uint8).reshape(img.shape[0], -1)
    f = a.copy()
    f[1:] = a[1:] - a[:-1]  # u8 arithmetic wraps modulo 256, as PNG specifies
    return np.concatenate([np.full((a.shape[0], 1), 2, np.uint8), f], axis=1)


def up_unfilter(filtered: np.ndarray, shape) -> np.ndarray:
    """Inverse of up_filter."""
    f = np.asarray(filtered, np.uint8)[:, 1:]
    return np.cumsum(f, axis=0, dtype=np.uint64).astype(np.uint8).reshape(shape)


def png_like_bytes(img: np.ndarray, level: int = 6) -> int:
    """Size of the deflated, up-filtered image data (a PNG's IDAT payload for this filter choice)."""
    return len(zlib.compress(up_filter(img).tobytes(), level))
