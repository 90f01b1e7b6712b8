"""The serving loop (dp_pix_server_*) and the keyed release: every record a request gets back, whatever else
was batched with it, is byte-identical to dp_pix_release of that frame alone with (stream_id = camera,
frame_idx = its arrival rank at the camera), and the records agree with the oracle."""
import random
import threading
import time

import numpy as np
import pytest
import torch

import oracle as O
import paper_2511_04261_b300 as P
from paper_2511_04261_b300 import synth
from tests.gpu_util import compare_records, gpu_release

pytestmark = pytest.mark.gpu

VAR = dict(C=3, grids=[32, 16, 8, 4], eps=[2.0, 1.0, 0.5, 0.25], R=255.0, m=16.0, seed=6)
SIZES = [(96, 160), (130, 250), (96, 160), (200, 352)]  # cameras 0 and 2 share a resolution


def _pools(n_per_cam, seed=0):
    return [synth.moving_rect_clip(seed=seed + c, frames=n_per_cam, M=M, N=N) for c, (M, N) in enumerate(SIZES)]


def _alone(cam, fidx, frame):
    M, N = SIZES[cam]
    kw = dict(M=M, N=N, source=O.SRC_VARIANCE, dtype=O.DT_F32, **VAR)
    _, _, rec = gpu_release(frame, None, stream_id=cam, frame_idx0=fidx, **kw)
    return rec[0]


def test_keyed_release_matches_per_frame_releases():
    M, N = 130, 250
    clip = synth.moving_rect_clip(seed=3, frames=5, M=M, N=N)
    plan = P.Plan(M=M, N=N, source=P.SRC_VARIANCE, dtype=P.REC_F32, **VAR)
    keys = [(7, 0), (2, 41), (7, 1), (0, 2**40 + 3), (2**24 - 1, 5)]
    recs = P.dp_pix_release_keyed(plan, torch.from_numpy(clip).cuda(), keys)
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    for i, (sid, fidx) in enumerate(keys):
        got = P.dp_pix_store(recs[i])
        _, _, single = gpu_release(clip[i], None, stream_id=sid, frame_idx0=fidx, M=M, N=N, source=O.SRC_VARIANCE,
                                   dtype=O.DT_F32, **VAR)
        assert got == single[0], i
        hdr = P.record_header(got)
        assert (hdr["stream_id"], hdr["frame_idx"]) == (sid, fidx)


def test_server_results_equal_alone_under_concurrent_submitters():
    pools = _pools(4)
    srv = P.Server(SIZES, arena_bytes=64 << 20, n_streams=3, **{k: v for k, v in VAR.items() if k != "C"})
    try:
        sent = {c: [] for c in range(len(SIZES))}  # per camera, in submission order: (ticket, frame)
        lock = threading.Lock()
        host = [[torch.from_numpy(p[i]).pin_memory() for i in range(len(p))] for p in pools]

        def submitter(cams, seed):
            rng = random.Random(seed)
            for k in range(12):
                c = cams[k % len(cams)]
                fr = host[c][rng.randrange(len(host[c]))]
                with lock:  # the rank a frame gets is its order of submission at its camera
                    t = srv.submit(c, fr, srv.record_buffer(c))
                    sent[c].append((t, fr))
                time.sleep(rng.random() * 0.002)

        th = [threading.Thread(target=submitter, args=([0, 1], 1)), threading.Thread(target=submitter, args=([2, 3], 2)),
              threading.Thread(target=submitter, args=([1, 3, 0], 3))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for c, lst in sent.items():
            for rank, (t, fr) in enumerate(lst):
                r = srv.wait(t, timeout_ms=30000)
                assert r is not None and r["status"] == 0
                assert r["camera"] == c and r["frame_idx"] == rank
                got = bytes(r["record"][: r["record_bytes"]].numpy())
                assert got == _alone(c, rank, fr.numpy()), (c, rank)
        st = srv.stats()
        assert st["completed"] == st["submitted"] == 36
        assert st["frames_in_flight_max"] >= 1
    finally:
        srv.close()


def test_server_admits_by_memory_and_batches_bursts():
    """An arena with room for one slot per resolution still completes every request (they wait for slots);
    a large arena batches a burst into few launches."""
    pools = _pools(3, seed=10)
    srv = None
    try:
        srv = P.Server(SIZES, arena_bytes=64 << 20, **{k: v for k, v in VAR.items() if k != "C"})
        sizes_bytes = srv.slot_bytes
        srv.close()
        # one slot per resolution: shares follow frame bytes, so give each class a little more than a slot
        frame_b = [M * N * 3 for (M, N) in SIZES]
        tot = sum(frame_b)
        need = max(sizes_bytes[c] * tot / (frame_b[c] * (2 if c in (0, 2) else 1)) for c in range(len(SIZES)))
        srv = P.Server(SIZES, arena_bytes=int(need * 1.3), n_streams=2, **{k: v for k, v in VAR.items() if k != "C"})
        assert all(1 <= srv.slots(c) <= 3 for c in range(len(SIZES)))
        host = [[torch.from_numpy(p[i]).pin_memory() for i in range(len(p))] for p in pools]
        tickets = []
        for k in range(20):
            c = k % len(SIZES)
            fr = host[c][k % 3]
            tickets.append((c, srv.submit(c, fr, srv.record_buffer(c)), fr))
        ranks = {c: 0 for c in range(len(SIZES))}
        for c, t, fr in tickets:
            r = srv.wait(t, timeout_ms=30000)
            assert r is not None and r["status"] == 0 and r["frame_idx"] == ranks[c]
            assert bytes(r["record"][: r["record_bytes"]].numpy()) == _alone(c, ranks[c], fr.numpy())
            ranks[c] += 1
        st = srv.stats()
        assert st["completed"] == 20
        assert st["frames_in_flight_max"] <= sum(srv.slots(c) for c in (0, 1, 3))
    finally:
        if srv is not None:
            srv.close()


def test_server_records_agree_with_oracle():
    pools = _pools(1, seed=20)
    srv = P.Server(SIZES, arena_bytes=64 << 20, **{k: v for k, v in VAR.items() if k != "C"})
    try:
        host = [torch.from_numpy(p[0]).pin_memory() for p in pools]
        ts = [srv.submit(c, host[c], srv.record_buffer(c)) for c in range(len(SIZES))]
        for c, t in enumerate(ts):
            r = srv.wait(t, timeout_ms=30000)
            got = bytes(r["record"][: r["record_bytes"]].numpy())
            M, N = SIZES[c]
            rec, means, sums, etas = O.release(pools[c][0], None, M=M, N=N, source=O.SRC_VARIANCE, dtype=O.DT_F32,
                                               stream_id=c, frame_idx=0, **VAR)
            compare_records(got, rec, means, sums, etas, O.DT_F32)
    finally:
        srv.close()


def test_server_rejects_bad_requests():
    srv = P.Server(SIZES[:1], arena_bytes=32 << 20, **{k: v for k, v in VAR.items() if k != "C"})
    try:
        fr = torch.zeros((96, 160, 3), dtype=torch.uint8).pin_memory()
        with pytest.raises(P.DppixError):
            srv.submit(3, fr, srv.record_buffer(0))
        with pytest.raises(P.DppixError):
            srv.submit(0, fr, torch.empty(16, dtype=torch.uint8))
        with pytest.raises(P.DppixError):
            srv.wait(12345)
    finally:
        srv.close()
    with pytest.raises(P.DppixError):
        P.Server(SIZES, arena_bytes=1 << 16, **{k: v for k, v in VAR.items() if k != "C"})
