"""Ragged batches (dp_pix_batch_*): every image's record is byte-identical to what dp_pix_release writes for
that image alone (same kernels, same keyed noise) and agrees with the oracle; reconstructions equal the
oracle's; the CUDA-graph replay and every autotuned segment width give the same bytes."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_2511_04261_b300 as P
from paper_2511_04261_b300 import synth
from tests.gpu_util import compare_records, gpu_release

pytestmark = pytest.mark.gpu

KW = dict(C=3, grids=[6, 20], eps=[0.5, 1.5], R=255.0, m=32.0, seed=3)


def _portraits(sizes, seed):
    rng = np.random.default_rng(seed)
    imgs, mattes = [], []
    for (M, N) in sizes:
        img, alpha = synth.portrait(rng, M, N)
        imgs.append(img)
        mattes.append(alpha)
    return imgs, mattes


def _run_batch(sizes, imgs, srcs, source, dtype=O.DT_F32, outs=True, out_type=P.OUT_U8, use_graph=True,
               autotune=False, pitch_extra=0):
    bp = P.BatchPlan(sizes, source=source, dtype=dtype, **KW)
    frames = []
    for im in imgs:
        if pitch_extra:
            M, N, C = im.shape
            buf = torch.zeros((M, N * C + pitch_extra), dtype=torch.uint8, device="cuda")
            buf[:, : N * C] = torch.from_numpy(im.reshape(M, N * C)).cuda()
            frames.append(buf[:, : N * C])
        else:
            frames.append(torch.from_numpy(np.ascontiguousarray(im)).cuda())
    src_t = [torch.from_numpy(np.ascontiguousarray(s)).cuda() if s is not None else None for s in srcs]
    recs = bp.alloc_records()
    ws = bp.alloc_workspace()
    dt = torch.uint8 if out_type == P.OUT_U8 else torch.float32
    o = [torch.full((M, N, 3), 7, dtype=dt, device="cuda") for (M, N) in sizes] if outs else None
    bp.bind(frames, src_t, recs, ws, outs=o, out_type=out_type, stream_ids=[5 + i for i in range(len(sizes))],
            frame_idx=[100 + i for i in range(len(sizes))])
    if autotune:
        bp.autotune(reps=1)
    bp.run(use_graph=use_graph)
    if use_graph:
        bp.run(use_graph=True)  # a replay gives the same bytes
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    got = [P.dp_pix_store(r) for r in recs]
    return bp, got, [t.cpu().numpy() for t in o] if outs else None


def _check_against_single_and_oracle(sizes, imgs, srcs, source, got, outs, dtype=O.DT_F32, out_type=P.OUT_U8,
                                     oracle_every=1):
    for i, (M, N) in enumerate(sizes):
        kw = dict(M=M, N=N, source=source, dtype=dtype, stream_id=5 + i, **KW)
        _, _, single = gpu_release(imgs[i], srcs[i], frame_idx0=100 + i, **kw)
        assert got[i] == single[0], i
        if i % oracle_every == 0:
            rec, means, sums, etas = O.release(imgs[i], srcs[i], frame_idx=100 + i, **kw)
            compare_records(got[i], rec, means, sums, etas, dtype)
        if outs is not None:
            exp = O.reconstruct(np.frombuffer(got[i], np.uint8), 0 if out_type == P.OUT_U8 else 1)
            assert np.array_equal(outs[i], exp), i


@pytest.mark.parametrize("out_type", [P.OUT_U8, P.OUT_F32])
def test_batch_matte_matches_single_release_and_oracle(out_type):
    sizes = [(130, 250), (61, 61), (600, 413), (59, 700), (240, 120), (333, 333)]
    imgs, mattes = _portraits(sizes, 11)
    bp, got, outs = _run_batch(sizes, imgs, mattes, O.SRC_MATTE, out_type=out_type)
    _check_against_single_and_oracle(sizes, imgs, mattes, O.SRC_MATTE, got, outs, out_type=out_type)


@pytest.mark.parametrize("dtype", [O.DT_U8, O.DT_SUM])
def test_batch_mask_and_labels(dtype):
    sizes = [(200, 180), (64, 300), (121, 65)]
    rng = np.random.default_rng(5)
    imgs = [rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8) for (M, N) in sizes]
    masks = [(rng.random((M, N)) < 0.6).astype(np.uint8) for (M, N) in sizes]
    _, got, outs = _run_batch(sizes, imgs, masks, O.SRC_MASK, dtype=dtype)
    _check_against_single_and_oracle(sizes, imgs, masks, O.SRC_MASK, got, outs, dtype=dtype)
    labels = [rng.integers(0, 2, size=(-(-M // 60), -(-N // 60)), dtype=np.uint8) for (M, N) in sizes]
    _, got, outs = _run_batch(sizes, imgs, labels, O.SRC_TILE_LABELS, dtype=dtype, use_graph=False)
    _check_against_single_and_oracle(sizes, imgs, labels, O.SRC_TILE_LABELS, got, outs, dtype=dtype)


def test_batch_autotune_and_strided_frames_keep_the_bytes():
    sizes = [(300, 500), (90, 800), (61, 120), (180, 180)]
    imgs, mattes = _portraits(sizes, 12)
    _, base, base_out = _run_batch(sizes, imgs, mattes, O.SRC_MATTE, use_graph=False)
    bp, tuned, tuned_out = _run_batch(sizes, imgs, mattes, O.SRC_MATTE, autotune=True, pitch_extra=13)
    assert 1 <= bp.seg_tiles() <= 16
    assert tuned == base
    for a, b in zip(tuned_out, base_out):
        assert np.array_equal(a, b)


def test_batch_without_outputs_and_rebinding():
    sizes = [(120, 200), (64, 64)]
    imgs, mattes = _portraits(sizes, 13)
    _, got, _ = _run_batch(sizes, imgs, mattes, O.SRC_MATTE, outs=False)
    _check_against_single_and_oracle(sizes, imgs, mattes, O.SRC_MATTE, got, None)


def test_batch_rejects_bad_arguments():
    with pytest.raises(P.DppixError):
        P.BatchPlan([(100, 100)], source=P.SRC_VARIANCE, grids=[8, 16], eps=[1, 1])
    bp = P.BatchPlan([(100, 100)], source=P.SRC_MATTE_F32, **KW)
    fr = torch.zeros((100, 100, 3), dtype=torch.uint8, device="cuda")
    matte = torch.zeros((100, 100), dtype=torch.float32, device="cuda")
    recs = bp.alloc_records()
    with pytest.raises(P.DppixError):  # workspace too small
        bp.bind([fr], [matte], recs, torch.empty(16, dtype=torch.uint8, device="cuda"))
    with pytest.raises(P.DppixError):  # matte missing
        bp.bind([fr], [None], recs, bp.alloc_workspace())


def test_batch_config3_shapes_sampled():
    """Images drawn from the ragged-batch size distribution (sides 512..4096), released and rebuilt in one
    batch; every record equals its single-image release and a sample is checked against the oracle."""
    sizes = synth.portrait_batch_shapes(seed=1003, n=256)[:12]
    imgs, mattes = _portraits(sizes, 1003)
    _, got, outs = _run_batch(sizes, imgs, mattes, O.SRC_MATTE)
    _check_against_single_and_oracle(sizes, imgs, mattes, O.SRC_MATTE, got, outs, oracle_every=4)


@pytest.mark.parametrize("source", [O.SRC_MATTE, O.SRC_MASK])
def test_batch_release_paths_give_the_same_bytes(source):
    """The staged path, the whole-warps-per-tile path, the streaming path and the streaming path with the images
    written in the same launch (DP_PIX_BATCH_PATH_*) at several segment widths write byte-identical records and
    images."""
    sizes = [(517, 1003), (64, 75), (300, 241), (1200, 700)]
    imgs, mattes = _portraits(sizes, 77)
    srcs = mattes if source == O.SRC_MATTE else [(m < 0.5).astype(np.uint8) for m in mattes]
    bp = P.BatchPlan(sizes, source=source, dtype=O.DT_F32, **KW)
    frames = [torch.from_numpy(np.ascontiguousarray(im)).cuda() for im in imgs]
    src_t = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in srcs]
    recs = bp.alloc_records()
    outs = [torch.full((M, N, 3), 7, dtype=torch.uint8, device="cuda") for (M, N) in sizes]
    bp.bind(frames, src_t, recs, bp.alloc_workspace(), outs=outs, stream_ids=[5 + i for i in range(4)],
            frame_idx=[100 + i for i in range(4)])
    ref = None
    for path, seg in [(P.BATCH_PATH_STAGED, 2), (P.BATCH_PATH_STREAM, 0), (P.BATCH_PATH_STREAM_FUSED, 0),
                      (P.BATCH_PATH_STREAM, 5), (P.BATCH_PATH_STREAM_FUSED, 3), (P.BATCH_PATH_TILES, 0),
                      (P.BATCH_PATH_TILES, 1), (P.BATCH_PATH_TILES, 4), (P.BATCH_PATH_TILES, 8)]:
        for o in outs:
            o.fill_(7)
        bp.set_path(path, seg)
        assert bp.tuning()[1] == path
        bp.run(use_graph=False)
        torch.cuda.synchronize()
        assert P.dp_pix_status() == 0
        got = ([P.dp_pix_store(r) for r in recs], [o.cpu().numpy() for o in outs])
        if ref is None:
            ref = got
            _check_against_single_and_oracle(sizes, imgs, srcs, source, got[0], got[1], oracle_every=2)
        else:
            assert got[0] == ref[0], (path, seg)
            for a, b in zip(got[1], ref[1]):
                assert np.array_equal(a, b), (path, seg)


@pytest.mark.parametrize("C,grids", [(1, (64, 128)), (2, (2, 3)), (4, (5, 7)), (3, (1, 4)), (1, (3, 8))])
def test_batch_tiles_path_other_channels_and_tile_sizes(C, grids):
    """The whole-warps-per-tile release (the default) against the staged one and the oracle, for C = 1, 2, 4
    and tiles from T = 6 (cells of 2 and 3 px, many per tile) to T = 128 (one cell of 128 px: the cell split
    into row parts over whole warps) and T = 4 with b = 1 (cells of one pixel): exact u32 sums in the record."""
    T = math.lcm(*grids)
    sizes = [(2 * T + 3, 3 * T + 1), (T, T), (T + 1, 5 * T - 2), (T // 2 + 1, 2 * T + 5)]
    rng = np.random.default_rng(C * 1000 + T)
    imgs = [rng.integers(0, 256, size=(M, N, C), dtype=np.uint8) for (M, N) in sizes]
    labels = [rng.integers(0, 2, size=(-(-M // T), -(-N // T)), dtype=np.uint8) for (M, N) in sizes]
    kw = dict(C=C, grids=list(grids), eps=[0.5, 1.5], R=255.0, m=32.0, seed=3)
    bp = P.BatchPlan(sizes, source=O.SRC_TILE_LABELS, dtype=O.DT_SUM, **kw)
    frames = [torch.from_numpy(np.ascontiguousarray(im)).cuda() for im in imgs]
    src_t = [torch.from_numpy(lab).cuda() for lab in labels]
    recs = bp.alloc_records()
    outs = [torch.zeros((M, N, C), dtype=torch.uint8, device="cuda") for (M, N) in sizes]
    bp.bind(frames, src_t, recs, bp.alloc_workspace(), outs=outs, stream_ids=[9] * len(sizes),
            frame_idx=list(range(len(sizes))))
    ref = None
    # 8 tiles per item stage 2 T rows of 8 T C bytes: past the CTA's shared memory at T = 128
    for path, seg in [(P.BATCH_PATH_STAGED, 1), (P.BATCH_PATH_TILES, 1), (P.BATCH_PATH_TILES, 2),
                      (P.BATCH_PATH_TILES, 4 if T > 64 else 8)]:
        bp.set_path(path, seg)
        assert bp.tuning()[1] == path
        bp.run(use_graph=False)
        torch.cuda.synchronize()
        assert P.dp_pix_status() == 0
        got = [P.dp_pix_store(r) for r in recs]
        if ref is None:
            ref = got
            for i, (M, N) in enumerate(sizes):
                rec, means, sums, etas = O.release(imgs[i], labels[i], M=M, N=N, source=O.SRC_TILE_LABELS,
                                                   dtype=O.DT_SUM, stream_id=9, frame_idx=i, **kw)
                compare_records(got[i], rec, means, sums, etas, O.DT_SUM)
                assert np.array_equal(outs[i].cpu().numpy(), O.reconstruct(np.frombuffer(got[i], np.uint8), 0))
        else:
            assert got == ref, (path, seg)
