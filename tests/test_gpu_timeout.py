"""Failure detection without a GPU fault: the release kernels' waits for their staged rows are bounded, and a
wait that runs out reports DP_PIX_E_TIMEOUT through dp_pix_status instead of hanging.  The test makes the
wait run out on purpose (a plan knob announces 16 bytes more than a block's first work item delivers, so that
item's barrier phase can never complete), checks the status and its detail word, and then checks that the
same device still releases correctly."""
import time

import numpy as np
import pytest
import torch

import oracle as O
import paper_2511_04261_b300 as P
from paper_2511_04261_b300 import _lib as L
from tests.gpu_util import compare_records

pytestmark = pytest.mark.gpu

M, N, GRIDS, EPS = 200, 264, [24, 8], [1.0, 0.5]


def _inputs():
    rng = np.random.default_rng(77)
    img = rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8)
    lab = rng.integers(0, 2, size=(-(-M // 24), -(-N // 24)), dtype=np.uint8)
    return img, lab


def test_wait_that_runs_out_reports_timeout_and_device_stays_usable():
    torch.cuda.set_device(0)
    img, lab = _inputs()
    kw = dict(M=M, N=N, C=3, grids=GRIDS, eps=EPS, m=16, source=P.SRC_TILE_LABELS, dtype=P.REC_F32, seed=5)
    frames = torch.from_numpy(np.stack([img] * 4)).cuda()
    labels = torch.from_numpy(np.stack([lab] * 4)).cuda()
    bad = P.Plan(**kw).tune(P.TUNE_WAIT_TRIES, 256).tune(P.TUNE_TEST_SHORT_TX, 1)
    assert bad.tuning(P.TUNE_TEST_SHORT_TX) == 1 and bad.tuning(P.TUNE_WAIT_TRIES) == 256
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bad.release(frames, labels)  # the launch itself succeeds
    with pytest.raises(P.DppixError) as e:
        P.dp_pix_status()
    dt = time.perf_counter() - t0
    assert e.value.code == L.E_TIMEOUT
    assert "0x500" in str(e.value)
    assert dt < 1.0, dt
    assert P.dp_pix_status() == 0  # reading the status cleared it
    # the same device, right after: a normal release agrees with the oracle
    good = P.Plan(**kw)
    recs = good.release(frames[:1], labels[:1])
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    rec, means, sums, etas = O.release(img, lab, M=M, N=N, C=3, grids=GRIDS, eps=EPS, m=16,
                                       source=O.SRC_TILE_LABELS, dtype=O.DT_F32, seed=5)
    compare_records(P.dp_pix_store(recs[0]), rec, means, sums, etas, O.DT_F32)


def test_timeout_knobs_are_checked():
    plan = P.Plan(M=M, N=N, C=3, grids=GRIDS, eps=EPS, source=P.SRC_TILE_LABELS)
    for knob, value in [(P.TUNE_WAIT_TRIES, 0), (P.TUNE_WAIT_TRIES, (1 << 22) + 1), (P.TUNE_TEST_SHORT_TX, 2)]:
        with pytest.raises(P.DppixError):
            plan.tune(knob, value)
    assert plan.tuning(P.TUNE_WAIT_TRIES) == 1 << 22 and plan.tuning(P.TUNE_TEST_SHORT_TX) == 0
