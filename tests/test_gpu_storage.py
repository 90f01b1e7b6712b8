"""Storage round trip on the GPU: a u8 record copied out, deflated, inflated and uploaded again rebuilds the
same pixelized frame (Sec. VII-A, VII-B: the stored metadata suffice to restore the image), and its size is
the oracle's."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2511_04261_b300 as P
from paper_2511_04261_b300 import storage as S
from paper_2511_04261_b300 import synth
from tests.gpu_util import compare_records

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("b", [2, 4, 16, 64])
def test_uniform_u8_record_round_trip(b):
    f, _ = synth.rect_frame(seed=1001)
    ft = torch.from_numpy(f).cuda()
    plan = P.Plan(M=576, N=768, C=3, grids=[b], eps=[0.5], m=16.0, seed=7, source=P.SRC_TILE_LABELS, dtype=P.REC_U8)
    lab = torch.zeros((1, -(-576 // b), -(-768 // b)), dtype=torch.uint8, device="cuda")
    recs, out = plan.release_reconstruct(ft[None], lab)
    host = P.dp_pix_store(recs[0])
    ora = O.release(f, np.zeros((-(-576 // b), -(-768 // b)), np.uint8), M=576, N=768, C=3, grids=[b], eps=[0.5], m=16.0,
                    seed=7, source=O.SRC_TILE_LABELS, dtype=O.DT_U8)[0]
    assert len(host) == len(ora)
    back = S.inflate_record(S.deflate_record(host))
    assert back == host
    dev = torch.zeros_like(recs[0])
    dev[:len(back)] = torch.frombuffer(bytearray(back), dtype=torch.uint8).cuda()
    again = P.dp_pix_reconstruct(dev[None], 576, 768, 3)
    torch.cuda.synchronize()
    assert torch.equal(again[0], out[0])


@pytest.mark.parametrize("n", [1, 4, 64])
def test_region_adaptive_u8_record_round_trip(n):
    rng = np.random.default_rng(70 + n)
    img, alpha = synth.portrait(rng, 512, 640)
    it = torch.from_numpy(img).cuda()
    at = torch.from_numpy(alpha).cuda()
    grids = [64, 64 // n]
    plan = P.Plan(M=512, N=640, C=3, grids=grids, eps=[0.5, 0.5], m=32.0, seed=7, source=P.SRC_MATTE_F32,
                  dtype=P.REC_U8)
    recs, out = plan.release_reconstruct(it[None], at[None])
    host = P.dp_pix_store(recs[0])
    back = S.inflate_record(S.deflate_record(host))
    dev = torch.zeros_like(recs[0])
    dev[:len(back)] = torch.frombuffer(bytearray(back), dtype=torch.uint8).cuda()
    again = P.dp_pix_reconstruct(dev[None], 512, 640, 3)
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    assert torch.equal(again[0], out[0])


@pytest.mark.parametrize("b", [1, 128])
def test_uniform_u8_record_extreme_grids_1080p(b):
    """The ends of the paper's grid sweep for storage (Sec. VII-A: b = 1 .. 128) on a 1920 x 1080 RGB frame:
    the u8 record equals the oracle's (map, layout and sizes bit-exact, values up to rint ties) and rebuilds
    the oracle's reconstruction of it."""
    M, N = 1080, 1920
    f = synth.moving_rect_clip(seed=900 + b, frames=1, M=M, N=N)[0]
    lab = np.zeros((-(-M // b), -(-N // b)), np.uint8)
    kw = dict(M=M, N=N, C=3, grids=[b], eps=[0.5], m=16.0, seed=8, source=O.SRC_TILE_LABELS, dtype=O.DT_U8)
    plan = P.Plan(**kw)
    recs, out = plan.release_reconstruct(torch.from_numpy(f).cuda()[None], torch.from_numpy(lab).cuda()[None])
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    host = P.dp_pix_store(recs[0])
    rec, means, sums, etas = O.release(f, lab, **kw)
    compare_records(host, rec, means, sums, etas, O.DT_U8)
    assert np.array_equal(out[0].cpu().numpy(), O.reconstruct(np.frombuffer(host, np.uint8), 0))


@pytest.mark.parametrize("n", [1, 2, 8, 32, 128])
def test_region_adaptive_u8_record_b128(n):
    """Alg. 3 at the paper's storage setting (Sec. VII-B: background b = 128, foreground b / n for n = 1 ..
    128) on a 1152 x 1536 portrait with its matte: u8 record against the oracle, reconstruction against the
    oracle's reconstruction of the same record."""
    M, N = 1152, 1536
    rng = np.random.default_rng(90 + n)
    img, alpha = synth.portrait(rng, M, N)
    grids = [128, 128 // n]
    kw = dict(M=M, N=N, C=3, grids=grids, eps=[0.5, 0.5], m=32.0, seed=9, source=O.SRC_MATTE, dtype=O.DT_U8)
    plan = P.Plan(**{**kw, "source": P.SRC_MATTE_F32})
    recs, out = plan.release_reconstruct(torch.from_numpy(img).cuda()[None], torch.from_numpy(alpha).cuda()[None])
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    host = P.dp_pix_store(recs[0])
    rec, means, sums, etas = O.release(img, alpha, **kw)
    compare_records(host, rec, means, sums, etas, O.DT_U8)
    assert np.array_equal(out[0].cpu().numpy(), O.reconstruct(np.frombuffer(host, np.uint8), 0))
