"""The bounds-checked build (libdppix_checked.so, loaded when DPPIX_CHECKED=1): the release, fused,
statistics, reconstruction and batch kernels test their global accesses against the extents of the buffers
they belong to.  In a child process with that library loaded: parity cases agree with the oracle with no check
firing, and a check made to fire on purpose -- the records' extent as the checks see it shrunk by a test knob,
while every access stays inside the real buffer -- skips the writes past it and reports DP_PIX_E_DEVICE with
detail 0x601 (a record write), after which the device still releases correctly."""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def _body():
    import torch

    import oracle as O
    import paper_2511_04261_b300 as P
    from paper_2511_04261_b300 import _lib, synth
    from tests.gpu_util import compare_records

    assert _lib.LIB_PATH.endswith("libdppix_checked.so")
    torch.cuda.set_device(0)
    rng = np.random.default_rng(31)
    # staged release, tile labels
    M, N = 200, 264
    img = rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8)
    lab = rng.integers(0, 2, size=(-(-M // 24), -(-N // 24)), dtype=np.uint8)
    kw = dict(M=M, N=N, C=3, grids=[24, 8], eps=[1.0, 0.5], m=16, source=O.SRC_TILE_LABELS, dtype=O.DT_F32, seed=5)
    plan = P.Plan(**kw)
    recs = plan.release(torch.from_numpy(img).cuda(), torch.from_numpy(lab).cuda())
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    rec, means, sums, etas = O.release(img, lab, **kw)
    compare_records(P.dp_pix_store(recs[0]), rec, means, sums, etas, O.DT_F32)
    # variance classes: statistics pass and fused emission + image
    F, M2, N2 = 3, 270, 480
    clip = synth.moving_rect_clip(seed=33, frames=F, M=M2, N=N2)
    kv = dict(M=M2, N=N2, C=3, grids=[32, 16, 8, 4], eps=[2, 1, .5, .25], m=16, source=O.SRC_VARIANCE,
              dtype=O.DT_F32, seed=6)
    vplan = P.Plan(**kv)
    vrecs, imgs = vplan.release_reconstruct(torch.from_numpy(clip).cuda())
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    imgs = imgs.cpu().numpy()
    for i in range(F):
        got = P.dp_pix_store(vrecs[i])
        rec, means, sums, etas = O.release(clip[i], None, frame_idx=i, **kv)
        compare_records(got, rec, means, sums, etas, O.DT_F32)
        assert np.array_equal(imgs[i], O.reconstruct(np.frombuffer(got, np.uint8), 0))
    # ragged batch, streaming path with the images
    sizes = [(301, 517), (130, 250)]
    pimgs, mattes = zip(*[synth.portrait(rng, a, b) for a, b in sizes])
    kb = dict(C=3, grids=[6, 20], eps=[0.5, 1.5], R=255.0, m=32.0, seed=3)
    for path in (P.BATCH_PATH_STAGED, P.BATCH_PATH_STREAM_FUSED, P.BATCH_PATH_TILES):
        bp = P.BatchPlan(sizes, source=P.SRC_MATTE_F32, dtype=P.REC_F32, **kb)
        brecs = bp.alloc_records()
        outs = [torch.zeros((a, b, 3), dtype=torch.uint8, device="cuda") for a, b in sizes]
        bp.set_path(path)
        bp.bind([torch.from_numpy(x).cuda() for x in pimgs], [torch.from_numpy(x).cuda() for x in mattes], brecs,
                bp.alloc_workspace(), outs=outs, stream_ids=[1, 2], frame_idx=[3, 4])
        bp.run(use_graph=False)
        torch.cuda.synchronize()
        assert P.dp_pix_status() == 0
        for i, (a, b) in enumerate(sizes):
            got = P.dp_pix_store(brecs[i])
            rec, means, sums, etas = O.release(pimgs[i], mattes[i], M=a, N=b, source=O.SRC_MATTE, dtype=O.DT_F32,
                                               stream_id=1 + i, frame_idx=3 + i, **kb)
            compare_records(got, rec, means, sums, etas, O.DT_F32)
            assert np.array_equal(outs[i].cpu().numpy(), O.reconstruct(np.frombuffer(got, np.uint8), 0))
    # a check made to fire: the record's last 16 written bytes lie outside the extent the checks see
    total = P.record_header(P.dp_pix_store(recs[0]))["total_bytes"]
    shrunk = P.Plan(**kw).tune(P.TUNE_TEST_SHRINK, plan.record_stride() - total + 16)
    shrunk.release(torch.from_numpy(img).cuda(), torch.from_numpy(lab).cuda())
    with pytest.raises(P.DppixError) as e:
        P.dp_pix_status()
    assert e.value.code == _lib.E_DEVICE and "0x601" in str(e.value), e.value
    recs = plan.release(torch.from_numpy(img).cuda(), torch.from_numpy(lab).cuda())
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    rec, means, sums, etas = O.release(img, lab, **kw)
    compare_records(P.dp_pix_store(recs[0]), rec, means, sums, etas, O.DT_F32)
    print("checked build ok")


def test_checked_build_parity_and_a_check_that_fires():
    env = dict(os.environ, DPPIX_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", "import tests.test_gpu_checked as t; t._body()"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "checked build ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
