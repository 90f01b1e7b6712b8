"""dp_pix_release_noalloc: the release for callers that cannot allocate device memory (graph-capture
regions, plug-ins whose host framework owns all allocations, real-time loops).  It must give the same
records as dp_pix_release with a caller workspace, call after call, although its built-in scratch keeps
the previous call's contents; and it must refuse work that does not fit its fixed scratch.

This file is collected last on purpose, so that a failure here never hides the other tests' results."""
import ctypes as ct

import numpy as np
import pytest
import torch

import paper_2511_04261_b300 as P
from paper_2511_04261_b300 import _lib, synth

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 16 << 20


def _noalloc(plan, frames, records, frame_idx0, src=None, stream_id=0):
    """Call the entry point through the C ABI with the same arguments dp_pix_release takes, minus the
    workspace."""
    L = _lib.lib()
    s = torch.cuda.current_stream()
    sp = ct.c_void_p(src.data_ptr()) if src is not None else None
    src_pitch = src.stride(1) * src.element_size() if src is not None else 0
    src_stride = src.stride(0) * src.element_size() if src is not None else 0
    return L.dp_pix_release_noalloc(plan.handle, ct.c_void_p(frames.data_ptr()), frames.stride(0), sp, src_pitch,
                                    src_stride, frames.shape[0], stream_id, frame_idx0,
                                    ct.c_void_p(records.data_ptr()), records.stride(0), ct.c_void_p(s.cuda_stream))


def _same_records(a, b):
    """The two calls run the same kernels on the same inputs, only with another scratch address: every
    record byte must be identical."""
    a = a.cpu().numpy()
    b = b.cpu().numpy()
    for i in range(a.shape[0]):
        h = P.record_header(a[i].tobytes())
        assert h == P.record_header(b[i].tobytes())
        end = h["total_bytes"]
        assert np.array_equal(a[i, :end], b[i, :end]), i


def _check_call(plan, frames, src, frame_idx0):
    ref = plan.release(frames, src, frame_idx0=frame_idx0)  # caller workspace, allocated by torch
    got = torch.zeros_like(ref)
    rc = _noalloc(plan, frames, got, frame_idx0, src=src)
    assert rc == 0, _lib.lib().dp_pix_last_error()
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    _same_records(ref, got)


def test_noalloc_matches_workspace_release_two_calls_in_a_row():
    torch.cuda.set_device(0)
    F, M, N = 6, 540, 960
    plan = P.Plan(M=M, N=N, C=3, grids=[32, 16, 8, 4], eps=[2, 1, .5, .25], m=16, source=P.SRC_VARIANCE,
                  dtype=P.REC_F32, seed=21)
    assert F * plan.ws_per_frame <= SCRATCH_BYTES
    for call, seed in enumerate([1101, 1102]):
        frames = torch.from_numpy(synth.moving_rect_clip(seed=seed, frames=F, M=M, N=N)).cuda()
        _check_call(plan, frames, None, 100 * call)


def test_noalloc_other_region_sources_on_used_scratch():
    """Mask and tile-label plans use other scratch regions (tile offsets, tile list) than the variance
    path; run them right after a variance call has filled the scratch with other data."""
    torch.cuda.set_device(0)
    F, M, N = 4, 576, 768
    var = P.Plan(M=M, N=N, C=3, grids=[32, 16, 8, 4], eps=[2, 1, .5, .25], m=16, source=P.SRC_VARIANCE, seed=3)
    frames = torch.from_numpy(synth.moving_rect_clip(seed=1103, frames=F, M=M, N=N)).cuda()
    _check_call(var, frames, None, 7)
    imgs, masks = zip(*[synth.rect_frame(seed=1110 + i, M=M, N=N) for i in range(F)])
    frames = torch.from_numpy(np.stack(imgs)).cuda()
    mask = torch.from_numpy(np.stack(masks)).cuda()
    mplan = P.Plan(M=M, N=N, C=3, grids=[24, 8], eps=[1.0, 0.5], m=16, source=P.SRC_MASK_U8, seed=1)
    _check_call(mplan, frames, mask, 0)
    lplan = P.Plan(M=M, N=N, C=3, grids=[24, 12, 8], eps=[1.0, 0.75, 0.5], m=16, source=P.SRC_TILE_LABELS, seed=2)
    rng = np.random.default_rng(1120)
    labels = torch.from_numpy(rng.integers(0, 3, size=(F, M // 24, N // 24), dtype=np.uint8)).cuda()
    _check_call(lplan, frames, labels, 40)
    _check_call(var, frames, None, 8)


def test_noalloc_rejects_work_beyond_its_scratch():
    plan = P.Plan(M=1080, N=1920, C=3, grids=[32, 16, 8, 4], eps=[2, 1, .5, .25], m=16, source=P.SRC_VARIANCE)
    F = SCRATCH_BYTES // plan.ws_per_frame + 1
    frames = torch.zeros((F, 1080, 1920, 3), dtype=torch.uint8, device="cuda")
    records = torch.zeros((F, plan.record_stride()), dtype=torch.uint8, device="cuda")
    rc = _noalloc(plan, frames, records, 0)
    assert rc == _lib.E_BUFFER_TOO_SMALL
    assert b"scratch" in _lib.lib().dp_pix_last_error()
    torch.cuda.synchronize()
    assert not records.any()  # nothing was launched
    # an empty call succeeds and leaves no earlier message behind
    assert _noalloc(plan, frames[:0], records, 0) == 0
    assert _lib.lib().dp_pix_last_error() == b""
