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
from tests.gpu_util import REL_TOL

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 16 << 20


def _noalloc(plan, frames, records, frame_idx0, stream_id=0):
    """Call the entry point through the C ABI with the same arguments dp_pix_release takes, minus the
    workspace."""
    L = _lib.lib()
    s = torch.cuda.current_stream()
    return L.dp_pix_release_noalloc(plan.handle, ct.c_void_p(frames.data_ptr()), frames.stride(0), None, 0, 0,
                                    frames.shape[0], stream_id, frame_idx0, ct.c_void_p(records.data_ptr()),
                                    records.stride(0), ct.c_void_p(s.cuda_stream))


def _same_records(a, b, plan):
    a = a.cpu().numpy()
    b = b.cpu().numpy()
    for i in range(a.shape[0]):
        h = P.record_header(a[i].tobytes())
        assert h == P.record_header(b[i].tobytes())
        pay = h["payload_offset"]
        assert np.array_equal(a[i, :pay], b[i, :pay])  # header, tile-row index and map: bit-exact
        end = h["total_bytes"]
        va = a[i, pay:end].view("<f4").astype(np.float64)
        vb = b[i, pay:end].view("<f4").astype(np.float64)
        assert np.all(np.abs(va - vb) <= REL_TOL * np.maximum(np.abs(va), np.abs(vb)))


def test_noalloc_matches_workspace_release_two_calls_in_a_row():
    torch.cuda.set_device(0)
    F, M, N = 6, 540, 960
    plan = P.Plan(M=M, N=N, C=3, grids=[32, 16, 8, 4], eps=[2, 1, .5, .25], m=16, source=P.SRC_VARIANCE,
                  dtype=P.REC_F32, seed=21)
    assert F * plan.ws_per_frame <= SCRATCH_BYTES
    for call, seed in enumerate([1101, 1102]):
        frames = torch.from_numpy(synth.moving_rect_clip(seed=seed, frames=F, M=M, N=N)).cuda()
        ref = plan.release(frames, None, frame_idx0=100 * call)  # caller workspace, allocated by torch
        got = torch.zeros_like(ref)
        rc = _noalloc(plan, frames, got, 100 * call)
        assert rc == 0, _lib.lib().dp_pix_last_error()
        torch.cuda.synchronize()
        assert P.dp_pix_status() == 0
        _same_records(ref, got, plan)


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
