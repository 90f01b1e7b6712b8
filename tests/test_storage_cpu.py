"""Host-side storage helpers (CPU): the PNG row filter against its definition, deflate round trips."""
import numpy as np

from paper_2511_04261_b300 import storage as S


def test_up_filter_inverts_and_matches_definition():
    rng = np.random.default_rng(1)
    img = rng.integers(0, 256, size=(9, 7, 3), dtype=np.uint8)
    f = S.up_filter(img)
    assert f.shape == (9, 1 + 21) and (f[:, 0] == 2).all()
    rows = img.reshape(9, 21).astype(np.int64)
    np.testing.assert_array_equal(f[0, 1:], rows[0])
    np.testing.assert_array_equal(f[1:, 1:], (rows[1:] - rows[:-1]) % 256)
    np.testing.assert_array_equal(S.up_unfilter(f, img.shape), img)


def test_deflate_round_trip_and_flat_image_compresses():
    blob = bytes(range(256)) * 10
    assert S.inflate_record(S.deflate_record(blob)) == blob
    flat = np.full((64, 64, 3), 100, np.uint8)
    assert S.png_like_bytes(flat) < 200  # one constant row, then zero differences
