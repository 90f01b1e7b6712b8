"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element on seeded inputs."""
import math

import numpy as np
import pytest
import torch
from scipy import stats

import oracle as O
import paper_2511_04261_b300 as P
from paper_2511_04261_b300 import synth
from tests.gpu_util import REL_TOL, compare_records, gpu_release

pytestmark = pytest.mark.gpu


def _labels(rng, M, N, grids):
    T = math.lcm(*grids)
    return rng.integers(0, len(grids), size=(-(-M // T), -(-N // T)), dtype=np.uint8)


# ------------------------------------------------------------------------------------------------------
# Noise: Philox words bit-exact, Laplace draws within tolerance, KS
# ------------------------------------------------------------------------------------------------------
def test_philox_words_bit_exact_and_laplace():
    rng = np.random.default_rng(1)
    n = 16384
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64)
    ctr[:4] = [[0, 0, 0, 0], [2**32 - 1] * 4, [1, 0, 0, 0], [0, 0, 0, 1]]
    seed = 0x1234567890ABCDEF
    sigma = 127.5
    words, eta = P.dp_pix_debug_noise(seed, torch.from_numpy(ctr.astype(np.int64)).cuda(), sigma)
    words = words.cpu().numpy()
    eta = eta.cpu().numpy().astype(np.float64)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(n):
        exp = O.philox4x32_10(ctr[i].astype(np.uint32), key)
        assert np.array_equal(words[i].astype(np.uint32), exp), i
        for j in range(4):
            e = O.laplace_from_word(int(exp[j]), sigma)
            assert abs(eta[i, j] - e) <= 1e-6 * abs(e) + 1e-7 * sigma


def test_gpu_laplace_ks():
    n = 50000
    ctr = torch.zeros((n, 4), dtype=torch.int64, device="cuda")
    ctr[:, 0] = torch.arange(n, device="cuda")
    ctr[:, 1] = 5
    _, eta = P.dp_pix_debug_noise(99, ctr, 1.0)
    e = eta.cpu().numpy().reshape(-1).astype(np.float64)
    assert stats.kstest(e, "laplace").pvalue > 0.01
    assert np.mean(np.abs(e)) == pytest.approx(1.0, rel=0.02)


# ------------------------------------------------------------------------------------------------------
# Release parity across sources, grids, channels, paddings and record types
# ------------------------------------------------------------------------------------------------------
CASES_LABELS = [
    (100, 130, 3, [24, 8], 0), (61, 67, 1, [6, 20], 0), (37, 53, 4, [4, 8, 16], 1), (70, 90, 3, [5], 0),
    (33, 47, 3, [12, 6, 4], 0), (64, 64, 3, [32, 16, 8, 4], 1), (150, 97, 3, [2, 3], 0), (45, 200, 3, [1, 4], 0),
]


@pytest.mark.parametrize("M,N,C,grids,pad", CASES_LABELS)
@pytest.mark.parametrize("dtype", [O.DT_F32, O.DT_U8, O.DT_SUM])
def test_release_tile_labels(M, N, C, grids, pad, dtype):
    rng = np.random.default_rng(M * 1000 + N + dtype)
    img = rng.integers(0, 256, size=(M, N, C), dtype=np.uint8)
    lab = _labels(rng, M, N, grids)
    kw = dict(M=M, N=N, C=C, grids=grids, eps=[0.5 + 0.25 * i for i in range(len(grids))], pad_mode=pad,
              source=O.SRC_TILE_LABELS, dtype=dtype, seed=12345, m=16)
    _, _, recs = gpu_release(img, lab, **kw)
    rec, means, sums, etas = O.release(img, lab, frame_idx=0, stream_id=0, **kw)
    compare_records(recs[0], rec, means, sums, etas, dtype)


@pytest.mark.parametrize("M,N,pad", [(200, 260, 0), (576, 768, 0), (131, 157, 1)])
def test_release_mask(M, N, pad):
    img, mask = synth.rect_frame(seed=1001 + M, M=M, N=N)
    kw = dict(M=M, N=N, C=3, grids=[24, 8], eps=[1.0, 0.5], pad_mode=pad, source=O.SRC_MASK, dtype=O.DT_F32,
              seed=1, m=16)
    _, _, recs = gpu_release(img, mask, **kw)
    rec, means, sums, etas = O.release(img, mask, **kw)
    compare_records(recs[0], rec, means, sums, etas, O.DT_F32)


@pytest.mark.parametrize("M,N", [(180, 250), (333, 421)])
def test_release_matte(M, N):
    img, alpha = synth.portrait(np.random.default_rng(M), M, N)
    kw = dict(M=M, N=N, C=3, grids=[20, 6], eps=[1.5, 0.5], source=O.SRC_MATTE, dtype=O.DT_F32, seed=3, m=32,
              matte_thr=0.5)
    _, _, recs = gpu_release(img, alpha, **kw)
    rec, means, sums, etas = O.release(img, alpha, **kw)
    compare_records(recs[0], rec, means, sums, etas, O.DT_F32)


@pytest.mark.parametrize("M,N,grids,eps", [
    (200, 330, [32, 16, 8, 4], [2, 1, .5, .25]),     # g = 4: g-cell sums, one read of the image
    (130, 250, [16, 8], [1, .5]),                     # g = 8
    (121, 245, [6, 20], [.5, 1.5]),                   # g = 2: statistics pass, then a second read
    (64, 96, [32, 32], [1, 1]),                       # g = 32 > 16: two passes
])
@pytest.mark.parametrize("dtype", [O.DT_F32, O.DT_SUM])
def test_release_variance(M, N, grids, eps, dtype):
    img = synth.moving_rect_clip(seed=7 + M, frames=1, M=M, N=N)[0]
    kw = dict(M=M, N=N, C=3, grids=grids, eps=eps, source=O.SRC_VARIANCE, dtype=dtype, seed=2, m=16)
    _, _, recs = gpu_release(img, None, **kw)
    rec, means, sums, etas = O.release(img, None, **kw)
    compare_records(recs[0], rec, means, sums, etas, dtype)


@pytest.mark.parametrize("M,N,C,grids,eps", [
    (96, 256, 3, [32, 16, 8, 4], [2, 1, .5, .25]),   # no padding
    (100, 256, 3, [32, 16, 8, 4], [2, 1, .5, .25]),  # mirrored rows
    (130, 128, 1, [16, 8], [1, .5]),                  # g = 8, one 16-byte chunk per tile
    (70, 64, 4, [8, 4], [1, .5]),                     # C = 4
    (64, 192, 3, [16], [1]),                          # g = 16, K = 1 (Alg. 2)
])
@pytest.mark.parametrize("dtype", [O.DT_F32, O.DT_SUM])
def test_release_variance_aligned_frames(M, N, C, grids, eps, dtype):
    """Frames without column padding and with 16-byte rows: the statistics pass reads them directly."""
    rng = np.random.default_rng(M + N + C)
    F = 3
    imgs = rng.integers(0, 256, size=(F, M, N, C), dtype=np.uint8)
    imgs[:, : M // 2] //= 4  # give the tiles different spreads
    kw = dict(M=M, N=N, C=C, grids=grids, eps=eps, source=O.SRC_VARIANCE, dtype=dtype, seed=8, m=16)
    _, _, recs = gpu_release(imgs, None, frame_idx0=3, **kw)
    for i in range(F):
        rec, means, sums, etas = O.release(imgs[i], None, frame_idx=3 + i, **kw)
        compare_records(recs[i], rec, means, sums, etas, dtype)


def test_release_batch_frames_stream_and_frame_index():
    rng = np.random.default_rng(3)
    F, M, N = 5, 75, 110
    imgs = rng.integers(0, 256, size=(F, M, N, 3), dtype=np.uint8)
    kw = dict(M=M, N=N, C=3, grids=[32, 16, 8, 4], eps=[2, 1, .5, .25], source=O.SRC_VARIANCE, dtype=O.DT_F32,
              seed=77, m=16)
    _, _, recs = gpu_release(imgs, None, frame_idx0=7, stream_id=3, **kw)
    for i in range(F):
        rec, means, sums, etas = O.release(imgs[i], None, frame_idx=7 + i, stream_id=3, **kw)
        h = compare_records(recs[i], rec, means, sums, etas, O.DT_F32)
        assert h["frame_idx"] == 7 + i and h["stream_id"] == 3


@pytest.mark.parametrize("pitch_extra,offset", [(13, 0), (16 * 5 - 0, 0), (3, 3)])
def test_release_row_pitch_and_alignment(pitch_extra, offset):
    rng = np.random.default_rng(pitch_extra + offset)
    M, N, C = 90, 125, 3
    pitch = N * C + pitch_extra
    buf = rng.integers(0, 256, size=(M * pitch + offset + 64,), dtype=np.uint8)
    img2d = buf[offset:offset + M * pitch].reshape(M, pitch)
    lab = _labels(rng, M, N, [24, 8])
    kw = dict(M=M, N=N, C=C, grids=[24, 8], eps=[1, .5], source=O.SRC_TILE_LABELS, dtype=O.DT_SUM, seed=4, m=16)
    plan = P.Plan(pitch=pitch, **kw)
    tb = torch.from_numpy(buf).cuda()
    t = tb[offset:offset + M * pitch].view(M, pitch)
    recs = plan.release(t, torch.from_numpy(lab).cuda())
    got = P.dp_pix_store(recs[0])
    rec, means, sums, etas = O.release(img2d, lab, pitch=pitch, **kw)
    compare_records(got, rec, means, sums, etas, O.DT_SUM)


def test_noise_free_release_is_block_mean():
    rng = np.random.default_rng(8)
    M, N = 97, 131
    img = rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8)
    lab = _labels(rng, M, N, [24, 8])
    kw = dict(M=M, N=N, C=3, grids=[24, 8], eps=[1, 1], source=O.SRC_TILE_LABELS, dtype=O.DT_F32, noise_free=True)
    plan, recs_d, recs = gpu_release(img, lab, **kw)
    rec, means, sums, etas = O.release(img, lab, **kw)
    compare_records(recs[0], rec, means, sums, etas, O.DT_F32)
    out = P.dp_pix_reconstruct(recs_d, M, N, 3, P.OUT_F32).cpu().numpy()[0]
    assert np.allclose(out, O.reconstruct(rec, 2), rtol=0, atol=255 * 2**-23)


# ------------------------------------------------------------------------------------------------------
# Reconstruction: bit-exact against the oracle's reconstruction of the same (GPU) record
# ------------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("M,N,C,grids,src", [
    (100, 130, 3, [24, 8], O.SRC_TILE_LABELS), (61, 67, 1, [6, 20], O.SRC_TILE_LABELS),
    (200, 330, 3, [32, 16, 8, 4], O.SRC_VARIANCE), (37, 53, 4, [4, 8, 16], O.SRC_TILE_LABELS),
    (45, 200, 3, [1, 4], O.SRC_TILE_LABELS),
])
@pytest.mark.parametrize("dtype", [O.DT_F32, O.DT_U8, O.DT_SUM])
def test_reconstruct_bit_exact(M, N, C, grids, src, dtype):
    rng = np.random.default_rng(M + N + C)
    F = 3
    imgs = rng.integers(0, 256, size=(F, M, N, C), dtype=np.uint8)
    lab = np.stack([_labels(rng, M, N, grids) for _ in range(F)]) if src == O.SRC_TILE_LABELS else None
    kw = dict(M=M, N=N, C=C, grids=grids, eps=[0.5] * len(grids), source=src, dtype=dtype, seed=5, m=16)
    plan, recs_d, recs = gpu_release(imgs, lab, **kw)
    for ot, npdt in [(P.OUT_U8, np.uint8), (P.OUT_F32, np.float32)]:
        out = P.dp_pix_reconstruct(recs_d, M, N, C, ot).cpu().numpy()
        for i in range(F):
            exp = O.reconstruct(np.frombuffer(recs[i], np.uint8), 0 if ot == P.OUT_U8 else 1)
            assert np.array_equal(out[i], exp), (i, ot)
    assert P.dp_pix_status() == 0


@pytest.mark.parametrize("M,N,C,grids,src", [
    (100, 130, 3, [24, 8], O.SRC_TILE_LABELS), (61, 67, 1, [6, 20], O.SRC_TILE_LABELS),
    (200, 330, 3, [32, 16, 8, 4], O.SRC_VARIANCE), (37, 53, 4, [4, 8, 16], O.SRC_TILE_LABELS),
    (45, 200, 3, [1, 4], O.SRC_TILE_LABELS), (96, 256, 3, [32, 16, 8, 4], O.SRC_VARIANCE),
    (70, 90, 3, [5], O.SRC_TILE_LABELS), (64, 80, 3, [2, 8], O.SRC_TILE_LABELS),
    (50, 2100, 3, [32, 16, 8, 4], O.SRC_TILE_LABELS),
])
@pytest.mark.parametrize("dtype", [O.DT_F32, O.DT_U8, O.DT_SUM])
def test_reconstruct_aligned_rows_bit_exact(M, N, C, grids, src, dtype):
    """Output rows 16-byte aligned (a padded pitch), the layout the vectorised reconstruction serves."""
    rng = np.random.default_rng(M * 7 + N + C)
    F = 2
    imgs = rng.integers(0, 256, size=(F, M, N, C), dtype=np.uint8)
    lab = np.stack([_labels(rng, M, N, grids) for _ in range(F)]) if src == O.SRC_TILE_LABELS else None
    kw = dict(M=M, N=N, C=C, grids=grids, eps=[0.5] * len(grids), source=src, dtype=dtype, seed=6, m=16)
    plan, recs_d, recs = gpu_release(imgs, lab, **kw)
    for ot, oes in [(P.OUT_U8, 1), (P.OUT_F32, 4)]:
        dt = torch.uint8 if ot == P.OUT_U8 else torch.float32
        Np = N
        while (Np * C * oes) % 16:
            Np += 1
        Np += 16 // math.gcd(16, C * oes)  # always leave a margin past the row
        big = torch.full((F, M, Np, C), 7, dtype=dt, device="cuda")
        view = big[:, :, :N, :]
        P.dp_pix_reconstruct(recs_d, M, N, C, ot, out=view)
        got = big.cpu().numpy()
        for i in range(F):
            exp = O.reconstruct(np.frombuffer(recs[i], np.uint8), 0 if ot == P.OUT_U8 else 1)
            assert np.array_equal(got[i, :, :N], exp), (i, ot)
            assert np.all(got[i, :, N:] == 7)  # nothing written past the row
    assert P.dp_pix_status() == 0


def test_reconstruct_strided_output():
    rng = np.random.default_rng(11)
    M, N = 50, 70
    img = rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8)
    lab = _labels(rng, M, N, [8, 4])
    plan, recs_d, recs = gpu_release(img, lab, M=M, N=N, C=3, grids=[8, 4], eps=[1, 1], seed=1)
    big = torch.zeros((M, N + 7, 3), dtype=torch.uint8, device="cuda")
    view = big[:, 3:3 + N, :]
    P.dp_pix_reconstruct(recs_d[0], M, N, 3, P.OUT_U8, out=view)
    exp = O.reconstruct(np.frombuffer(recs[0], np.uint8), 0)
    got = big.cpu().numpy()
    assert np.array_equal(got[:, 3:3 + N], exp)
    assert not got[:, :3].any() and not got[:, 3 + N:].any()


# ------------------------------------------------------------------------------------------------------
# Edge cases
# ------------------------------------------------------------------------------------------------------
def test_edge_one_pixel_and_exact_tile():
    for (M, N, grids) in [(1, 1, [1]), (24, 24, [24, 8]), (8, 8, [8]), (2, 3, [2])]:
        pad = 0
        rng = np.random.default_rng(M * N)
        img = rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8)
        lab = _labels(rng, M, N, grids)
        kw = dict(M=M, N=N, C=3, grids=grids, eps=[1] * len(grids), source=O.SRC_TILE_LABELS, dtype=O.DT_F32,
                  seed=9, pad_mode=pad)
        plan, recs_d, recs = gpu_release(img, lab, **kw)
        rec, means, sums, etas = O.release(img, lab, **kw)
        compare_records(recs[0], rec, means, sums, etas, O.DT_F32)
        out = P.dp_pix_reconstruct(recs_d, M, N, 3).cpu().numpy()[0]
        assert np.array_equal(out, O.reconstruct(np.frombuffer(recs[0], np.uint8), 0))


def test_zero_frames_is_noop_and_bad_labels_flag_status():
    plan = P.Plan(M=32, N=32, C=3, grids=[16], eps=[1])
    img = torch.zeros((0, 32, 32, 3), dtype=torch.uint8, device="cuda")
    recs = plan.release(img, torch.zeros((0, 2, 2), dtype=torch.uint8, device="cuda"))
    assert recs.shape[0] == 0
    img = torch.zeros((32, 32, 3), dtype=torch.uint8, device="cuda")
    bad = torch.full((2, 2), 5, dtype=torch.uint8, device="cuda")  # label >= K
    plan.release(img, bad)
    with pytest.raises(P.DppixError) as e:
        P.dp_pix_status()
    assert e.value.code == -8
    assert P.dp_pix_status() == 0  # cleared


def test_reconstruct_rejects_malformed_record():
    rec = torch.zeros((1, 4096), dtype=torch.uint8, device="cuda")
    out = torch.zeros((1, 8, 8, 3), dtype=torch.uint8, device="cuda")
    P.dp_pix_reconstruct(rec, 8, 8, 3, out=out)
    with pytest.raises(P.DppixError):
        P.dp_pix_status()
    assert not out.any()


@pytest.mark.parametrize("M,N,grids", [
    (32, 32, [32, 16, 8, 4]),      # one tile, four classes: three boundaries lie beyond the last rank
    (32, 96, [32, 16, 8, 4]),      # three tiles
    (200, 330, [32, 16, 8, 4]),    # 77 tiles
    (720, 1280, [16, 8]),          # 3600 tiles
    (1080, 1920, [16, 8]),         # 8160 tiles
    (720, 1280, [8, 4]),           # 14400 tiles
    (2160, 3840, [32, 16, 8, 4]),  # 4K frames: 8160 tiles of 32 x 32
])
def test_variance_classes_every_rank_path(M, N, grids):
    """The tile -> class map (variance quantile classes: tiles ranked by (key, tile index), class
    floor(K rank / n)) equals the oracle's.  Frames: the moving-rectangle clip; the same, flat in its upper
    half (hundreds of tiles share the key 0); one random tile repeated over the frame (equal keys away from
    the mirrored edges, so a boundary's histogram bin is full and the kernel sorts); uniform noise (keys
    within a few per cent of each other)."""
    T = math.lcm(*grids)
    clip = np.concatenate([synth.moving_rect_clip(seed=M + N, frames=2, M=M, N=N)] * 2)
    clip[1, : M // 2] = 17
    rng = np.random.default_rng(M * N)
    tile = rng.integers(0, 256, size=(T, T, 3), dtype=np.uint8)
    clip[2] = np.tile(tile, (-(-M // T), -(-N // T), 1))[:M, :N]
    clip[3] = rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8)
    kw = dict(M=M, N=N, C=3, grids=grids, eps=[1.0] * len(grids), source=O.SRC_VARIANCE, dtype=O.DT_F32, seed=3,
              m=16)
    plan = P.Plan(**kw)
    recs_d = plan.release(torch.from_numpy(clip).cuda(), None)
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    for i in range(len(clip)):
        got = O.record_map(np.frombuffer(P.dp_pix_store(recs_d[i]), np.uint8))
        exp = O.classify(clip[i], None, **kw)
        assert np.array_equal(got, exp), (i, int((got != exp).sum()))
        K, n = len(grids), exp.size  # class q holds the ranks r with floor(K r / n) = q
        assert np.array_equal(np.bincount(exp.reshape(-1), minlength=K), np.bincount(K * np.arange(n) // n, minlength=K))


@pytest.mark.parametrize("b", list(range(2, 21)))
def test_uniform_grayscale_every_grid(b):
    """Alg. 2 (one region, uniform grid b) on grayscale frames of 70 x 101 pixels, every b of the paper's
    timing sweep (Sec. VII, 2..20): records and reconstructions equal the oracle's (ragged edges mirrored)."""
    F, M, N = 2, 70, 101
    clip = synth.moving_rect_clip(seed=40 + b, frames=F, M=M, N=N, C=1)
    lab = np.zeros((F, -(-M // b), -(-N // b)), dtype=np.uint8)
    kw = dict(M=M, N=N, C=1, grids=[b], eps=[0.5], m=16, source=O.SRC_TILE_LABELS, dtype=O.DT_F32, seed=11)
    plan, recs_d, recs = gpu_release(clip, lab, **kw)
    outs = P.dp_pix_reconstruct(recs_d, M, N, 1).cpu().numpy()
    for i in range(F):
        rec, means, sums, etas = O.release(clip[i], lab[i], frame_idx=i, **kw)
        compare_records(recs[i], rec, means, sums, etas, O.DT_F32)
        assert np.array_equal(outs[i], O.reconstruct(np.frombuffer(recs[i], np.uint8), 0))


@pytest.mark.parametrize("b", [10, 14, 16])
def test_uniform_grayscale_768x576(b):
    """The paper's PETS shape (768 x 576 grayscale, eps 0.5, m 16) at b = 16 and at the two grids that leave
    a padded edge (10, 14): one release + reconstruction call, every record element and pixel checked."""
    F, M, N = 3, 576, 768
    clip = synth.moving_rect_clip(seed=700 + b, frames=F, M=M, N=N, C=1)
    lab = np.zeros((F, -(-M // b), -(-N // b)), dtype=np.uint8)
    kw = dict(M=M, N=N, C=1, grids=[b], eps=[0.5], m=16, source=O.SRC_TILE_LABELS, dtype=O.DT_F32, seed=12)
    plan = P.Plan(**kw)
    recs_d, outs = plan.release_reconstruct(torch.from_numpy(clip).cuda(), torch.from_numpy(lab).cuda())
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    outs = outs.cpu().numpy()
    for i in range(F):
        got = P.dp_pix_store(recs_d[i])
        rec, means, sums, etas = O.release(clip[i], lab[i], frame_idx=i, **kw)
        compare_records(got, rec, means, sums, etas, O.DT_F32)
        assert np.array_equal(outs[i], O.reconstruct(np.frombuffer(got, np.uint8), 0))


@pytest.mark.parametrize("b", [1, 2, 3])
def test_uniform_grayscale_1080p_small_grids(b):
    """The paper's Venice shape (1920 x 1080 grayscale, eps 0.5, m 16) at the smallest grids of its sweep:
    518,400 tiles at b = 2 and 2,073,600 at b = 1, more than a shared-memory map holds, so the record is
    laid out from the map in global memory.  Every record element and pixel checked against the oracle."""
    F, M, N = 2, 1080, 1920
    clip = synth.moving_rect_clip(seed=800 + b, frames=F, M=M, N=N, C=1)
    lab = np.zeros((F, -(-M // b), -(-N // b)), dtype=np.uint8)
    kw = dict(M=M, N=N, C=1, grids=[b], eps=[0.5], m=16, source=O.SRC_TILE_LABELS, dtype=O.DT_F32, seed=13)
    plan = P.Plan(**kw)
    recs_d, outs = plan.release_reconstruct(torch.from_numpy(clip).cuda(), torch.from_numpy(lab).cuda())
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    outs = outs.cpu().numpy()
    for i in range(F):
        got = P.dp_pix_store(recs_d[i])
        rec, means, sums, etas = O.release(clip[i], lab[i], frame_idx=i, **kw)
        compare_records(got, rec, means, sums, etas, O.DT_F32)
        assert np.array_equal(outs[i], O.reconstruct(np.frombuffer(got, np.uint8), 0))


# ------------------------------------------------------------------------------------------------------
# Full-size workloads at the benchmark's launch configuration, sampled against the oracle
# ------------------------------------------------------------------------------------------------------
def test_config1_full_frame():
    """768 x 576 RGB, 6 rectangles, fg b=8 eps=.5, bg b=24 eps=1, m=16, seed 1: complete record + image."""
    img, mask = synth.rect_frame(seed=1001)
    kw = dict(M=576, N=768, C=3, grids=[24, 8], eps=[1.0, 0.5], source=O.SRC_MASK, dtype=O.DT_F32, seed=1, m=16)
    plan, recs_d, recs = gpu_release(img, mask, **kw)
    rec, means, sums, etas = O.release(img, mask, **kw)
    compare_records(recs[0], rec, means, sums, etas, O.DT_F32)
    out = P.dp_pix_reconstruct(recs_d, 576, 768, 3).cpu().numpy()[0]
    assert np.array_equal(out, O.reconstruct(np.frombuffer(recs[0], np.uint8), 0))


def test_config2_full_clip_sampled():
    """64 frames 1920 x 1080, 4 variance classes (b 32/16/8/4, eps 2/1/.5/.25), one launch sequence as in the
    benchmark; frames 0, 31 and 63 compared completely with the oracle, invariants on all frames."""
    F, M, N = 64, 1080, 1920
    clip = synth.moving_rect_clip(seed=1002, frames=F, M=M, N=N)
    kw = dict(M=M, N=N, C=3, grids=[32, 16, 8, 4], eps=[2, 1, .5, .25], source=O.SRC_VARIANCE, dtype=O.DT_F32,
              seed=2, m=16)
    plan = P.Plan(**kw)
    frames = torch.from_numpy(clip).cuda()
    recs_d = plan.release(frames, None)
    outs = P.dp_pix_reconstruct(recs_d, M, N, 3)
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    for i in [0, 31, 63]:
        got = P.dp_pix_store(recs_d[i])
        rec, means, sums, etas = O.release(clip[i], None, frame_idx=i, **kw)
        compare_records(got, rec, means, sums, etas, O.DT_F32)
        assert np.array_equal(outs[i].cpu().numpy(), O.reconstruct(np.frombuffer(got, np.uint8), 0))
    # every frame: 2040 tiles in four equal classes of 510, record size by the C4 formula
    a16 = lambda x: (x + 15) // 16 * 16
    for i in range(F):
        h = P.record_header(P.dp_pix_store(recs_d[i]))
        assert h["count"] == [510, 510, 510, 510]
        exp = 512 + a16(34 * 4 * 4) + a16(2040) + sum(a16(510 * (32 // b) ** 2 * 12) for b in [32, 16, 8, 4])
        assert h["total_bytes"] == exp


# ------------------------------------------------------------------------------------------------------
# Release and reconstruction in one call (Alg. 3 with the restoring steps of Sec. VI-F)
# ------------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("M,N,C,grids,src,padded", [
    (96, 256, 3, [32, 16, 8, 4], O.SRC_VARIANCE, False),    # fused kernel, g = 4
    (100, 256, 3, [32, 16, 8, 4], O.SRC_VARIANCE, True),    # fused kernel, mirrored rows, padded pitch
    (130, 128, 1, [16, 8], O.SRC_VARIANCE, True),           # fused kernel, g = 8, C = 1
    (70, 64, 4, [8, 4], O.SRC_VARIANCE, False),             # fused kernel, C = 4
    (64, 192, 3, [16], O.SRC_VARIANCE, True),               # fused kernel, g = 16, K = 1
    (200, 330, 3, [32, 16, 8, 4], O.SRC_VARIANCE, True),    # fused kernel, mirrored columns (staged statistics)
    (200, 330, 3, [32, 16, 8, 4], O.SRC_VARIANCE, False),   # rows not 16-byte aligned: release, then reconstruct
    (121, 245, 3, [6, 20], O.SRC_VARIANCE, True),           # g = 2: release, then reconstruct
    (100, 130, 3, [24, 8], O.SRC_TILE_LABELS, True),        # labels: release, then reconstruct
])
@pytest.mark.parametrize("dtype", [O.DT_F32, O.DT_U8, O.DT_SUM])
@pytest.mark.parametrize("ot", [P.OUT_U8, P.OUT_F32])
def test_release_reconstruct_matches_two_calls(M, N, C, grids, src, padded, dtype, ot):
    """The fused call writes the records dp_pix_release writes and the images dp_pix_reconstruct makes from
    them, bit for bit; the images also equal the oracle's reconstruction of the oracle-checked records."""
    rng = np.random.default_rng(M * 3 + N + C + dtype)
    F = 3
    imgs = rng.integers(0, 256, size=(F, M, N, C), dtype=np.uint8)
    imgs[:, : M // 3] //= 8
    lab = np.stack([_labels(rng, M, N, grids) for _ in range(F)]) if src == O.SRC_TILE_LABELS else None
    kw = dict(M=M, N=N, C=C, grids=grids, eps=[0.5 + 0.25 * i for i in range(len(grids))], source=src, dtype=dtype,
              seed=12, m=16)
    plan, recs_d, recs = gpu_release(imgs, lab, frame_idx0=5, **kw)
    oes = 1 if ot == P.OUT_U8 else 4
    dt = torch.uint8 if ot == P.OUT_U8 else torch.float32
    Np = N
    if padded:
        while (Np * C * oes) % 16:
            Np += 1
        Np += 16 // math.gcd(16, C * oes)
    big = torch.full((F, M, Np, C), 7, dtype=dt, device="cuda")
    view = big[:, :, :N, :]
    t = torch.from_numpy(imgs).cuda()
    s = torch.from_numpy(lab).cuda() if lab is not None else None
    recs2 = torch.full_like(recs_d, 0xAB)
    plan.release_reconstruct(t, s, frame_idx0=5, out_type=ot, records=recs2, out=view)
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    ref = P.dp_pix_reconstruct(recs_d, M, N, C, ot)
    got = big.cpu().numpy()
    assert np.array_equal(got[:, :, :N], ref.cpu().numpy())
    if Np > N:
        assert np.all(got[:, :, N:] == 7)
    for i in range(F):
        assert P.dp_pix_store(recs2[i]) == recs[i]
        exp = O.reconstruct(np.frombuffer(recs[i], np.uint8), 0 if ot == P.OUT_U8 else 1)
        assert np.array_equal(got[i, :, :N], exp), i
    rec, means, sums, etas = O.release(imgs[0], lab[0] if lab is not None else None, frame_idx=5, **kw)
    compare_records(recs[0], rec, means, sums, etas, dtype)


def test_release_reconstruct_config2_sampled():
    """A 1080p clip through the fused call: records equal to dp_pix_release's, images equal to
    dp_pix_reconstruct's, and sampled frames checked against the oracle."""
    F, M, N = 6, 1080, 1920
    clip = synth.moving_rect_clip(seed=21, frames=F, M=M, N=N)
    kw = dict(M=M, N=N, C=3, grids=[32, 16, 8, 4], eps=[2, 1, .5, .25], source=O.SRC_VARIANCE, dtype=O.DT_F32,
              seed=4, m=16)
    plan, recs_d, recs = gpu_release(clip, None, **kw)
    t = torch.from_numpy(clip).cuda()
    r2, img = plan.release_reconstruct(t)
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    assert torch.equal(r2, recs_d) or all(P.dp_pix_store(r2[i]) == recs[i] for i in range(F))
    assert torch.equal(img, P.dp_pix_reconstruct(recs_d, M, N, 3, P.OUT_U8))
    for i in (0, F - 1):
        rec, means, sums, etas = O.release(clip[i], None, frame_idx=i, **kw)
        compare_records(recs[i], rec, means, sums, etas, O.DT_F32)


@pytest.mark.parametrize("ot", [P.OUT_U8, P.OUT_F32])
def test_release_reconstruct_launch_shapes_do_not_change_results(ot):
    """Every fused launch shape (pixel columns per item, threads per block, frame chunks pipelined between the
    caller's stream and a side stream, blocks per SM of the fused kernel) gives the same bytes."""
    F, M, N = 8, 200, 352
    rng = np.random.default_rng(17)
    imgs = rng.integers(0, 256, size=(F, M, N, 3), dtype=np.uint8)
    imgs[:, :, : N // 2] //= 16
    kw = dict(M=M, N=N, C=3, grids=[32, 16, 8, 4], eps=[2, 1, .5, .25], source=O.SRC_VARIANCE, dtype=O.DT_F32,
              seed=23, m=16)
    t = torch.from_numpy(imgs).cuda()
    base = None
    for px, thr, split, cap in [(64, 128, 1, 0), (96, 256, 2, 1), (512, 128, 4, 2), (512, 256, 1, 0),
                                (1024, 128, 3, 0), (2048, 256, 4, 3), (2048, 128, 1, 0), (960, 192, 1, 0),
                                (640, 96, 2, 4), (1024, 128, 8, 1)]:
        if True:
            plan = (P.Plan(**kw).tune(P.TUNE_FUSED_PX, px).tune(P.TUNE_FUSED_THREADS, thr).tune(P.TUNE_SPLIT, split)
                    .tune(P.TUNE_FUSED_CAP, cap))
            recs, img = plan.release_reconstruct(t, out_type=ot)
            torch.cuda.synchronize()
            assert P.dp_pix_status() == 0
            got = ([P.dp_pix_store(recs[i]) for i in range(F)], img.cpu().numpy())
            if base is None:
                base = got
                for i in range(F):
                    exp = O.reconstruct(np.frombuffer(got[0][i], np.uint8), 0 if ot == P.OUT_U8 else 1)
                    assert np.array_equal(got[1][i], exp)
            else:
                assert got[0] == base[0], (px, thr, split, cap)
                assert np.array_equal(got[1], base[1]), (px, thr, split, cap)
