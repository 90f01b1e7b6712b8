"""Parity of the privacy-strict edge mode (DP_PIX_PAD_NONE: Alg. 1's partial cells, mean and noise scale
from the h x w samples inside the frame) with the oracle, for every region source it serves, single frames
and ragged batches, and the reconstruction of such records."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2511_04261_b300 as P
from paper_2511_04261_b300 import synth
from tests.gpu_util import compare_records, gpu_release

pytestmark = pytest.mark.gpu


def _labels(rng, M, N, grids):
    import math
    T = math.lcm(*grids)
    return rng.integers(0, len(grids), size=(-(-M // T), -(-N // T)), dtype=np.uint8)


@pytest.mark.parametrize("M,N,C,grids", [(37, 53, 3, [8]), (61, 77, 3, [6, 20]), (45, 200, 1, [4, 16]),
                                         (5, 7, 3, [8]), (100, 130, 2, [12, 6, 4]), (64, 64, 3, [16])])
@pytest.mark.parametrize("dtype", [O.DT_F32, O.DT_U8, O.DT_SUM])
def test_strict_release_tile_labels(M, N, C, grids, dtype):
    rng = np.random.default_rng(M * 1000 + N + dtype)
    img = rng.integers(0, 256, size=(M, N, C), dtype=np.uint8)
    lab = _labels(rng, M, N, grids)
    kw = dict(M=M, N=N, C=C, grids=grids, eps=[0.5 + 0.25 * i for i in range(len(grids))], pad_mode=O.PAD_NONE,
              source=O.SRC_TILE_LABELS, dtype=dtype, seed=77, m=16)
    plan, recs_t, recs = gpu_release(img, lab, **kw)
    rec, means, sums, etas = O.release(img, lab, **kw)
    compare_records(recs[0], rec, means, sums, etas, dtype)
    if dtype != O.DT_SUM:
        out = P.dp_pix_reconstruct(recs_t, M, N, C)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out[0].cpu().numpy(), O.reconstruct(np.frombuffer(recs[0], np.uint8), 0))


@pytest.mark.parametrize("M,N", [(131, 157), (200, 260)])
def test_strict_release_mask(M, N):
    img, mask = synth.rect_frame(seed=1001 + M, M=M, N=N)
    kw = dict(M=M, N=N, C=3, grids=[24, 8], eps=[1.0, 0.5], pad_mode=O.PAD_NONE, source=O.SRC_MASK,
              dtype=O.DT_F32, seed=1, m=16)
    _, _, recs = gpu_release(img, mask, **kw)
    rec, means, sums, etas = O.release(img, mask, **kw)
    compare_records(recs[0], rec, means, sums, etas, O.DT_F32)


@pytest.mark.parametrize("dtype", [O.DT_F32, O.DT_U8])
def test_strict_noise_free_is_valid_sample_block_mean(dtype):
    rng = np.random.default_rng(40 + dtype)
    M, N, grids = 45, 67, [8, 24]
    img = rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8)
    lab = _labels(rng, M, N, grids)
    kw = dict(M=M, N=N, C=3, grids=grids, eps=[1.0, 1.0], pad_mode=O.PAD_NONE, source=O.SRC_TILE_LABELS,
              dtype=dtype, seed=5, m=16, noise_free=True)
    _, recs_t, recs = gpu_release(img, lab, **kw)
    rec, means, sums, etas = O.release(img, lab, **kw)
    compare_records(recs[0], rec, means, sums, etas, dtype)


def test_strict_release_matte():
    img, alpha = synth.portrait(np.random.default_rng(5), 181, 251)
    kw = dict(M=181, N=251, C=3, grids=[20, 6], eps=[1.5, 0.5], pad_mode=O.PAD_NONE, source=O.SRC_MATTE,
              dtype=O.DT_F32, seed=3, m=32, matte_thr=0.5)
    _, _, recs = gpu_release(img, alpha, **kw)
    rec, means, sums, etas = O.release(img, alpha, **kw)
    compare_records(recs[0], rec, means, sums, etas, O.DT_F32)


@pytest.mark.parametrize("path", [-1, 0, 3])
def test_strict_ragged_batch_matches_oracle(path):
    """Alg. 1's partial edge cells in a ragged batch, on the default release path, the staged path and the
    whole-warps-per-tile path (DP_PIX_BATCH_PATH_STAGED / _TILES = 0 / 3)."""
    sizes = [(181, 251), (64, 60), (7, 130), (300, 119)]
    rng = np.random.default_rng(12)
    imgs, mattes = zip(*[synth.portrait(rng, M, N) for M, N in sizes])
    bp = P.BatchPlan(sizes, grids=(6, 20), eps=(0.5, 1.5), m=32.0, pad_mode=P.PAD_NONE, source=P.SRC_MATTE_F32,
                     dtype=P.REC_F32, seed=3)
    frames = [torch.from_numpy(np.ascontiguousarray(i)).cuda() for i in imgs]
    srcs = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in mattes]
    recs, ws = bp.alloc_records(), bp.alloc_workspace()
    outs = [torch.empty((M, N, 3), dtype=torch.uint8, device="cuda") for M, N in sizes]
    bp.set_path(path)
    bp.bind(frames, srcs, recs, ws, outs=outs, stream_ids=[2] * len(sizes), frame_idx=list(range(len(sizes))))
    bp.run(use_graph=False)
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    for i, (M, N) in enumerate(sizes):
        kw = dict(M=M, N=N, C=3, grids=[6, 20], eps=[0.5, 1.5], pad_mode=O.PAD_NONE, source=O.SRC_MATTE,
                  dtype=O.DT_F32, seed=3, m=32, matte_thr=0.5, stream_id=2, frame_idx=i)
        rec, means, sums, etas = O.release(imgs[i], mattes[i], **kw)
        got = P.dp_pix_store(recs[i])
        compare_records(got, rec, means, sums, etas, O.DT_F32)
        np.testing.assert_array_equal(outs[i].cpu().numpy(), O.reconstruct(np.frombuffer(got, np.uint8), 0))


def test_strict_mode_rejected_where_unsupported():
    with pytest.raises(P.DppixError):
        P.Plan(M=64, N=64, C=3, grids=[8, 16], eps=[1, 1], pad_mode=P.PAD_NONE, source=P.SRC_VARIANCE)
    with pytest.raises(P.DppixError):
        P.Plan(M=64, N=64, C=3, grids=[8], eps=[1], pad_mode=7)
