"""The serving loop (dp_pix_server_*) and the keyed release: every record (and pixelized image) a request gets
back, whatever else was batched with it, is byte-identical to releasing that frame alone with (stream_id =
camera, frame_idx = its rank among the camera's submissions, counted from the camera's first index), and the
records agree with the oracle -- at the serving workload's own resolutions too.  A server created with the
counters of an earlier one continues every camera's count, so no noise key is drawn twice."""
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


def _alone_recon(cam, fidx, frame, sizes=None):
    M, N = (sizes or SIZES)[cam]
    plan = P.Plan(M=M, N=N, source=P.SRC_VARIANCE, dtype=P.REC_F32, **VAR)
    recs, img = plan.release_reconstruct(torch.from_numpy(frame).cuda(), None, stream_id=cam, frame_idx0=fidx)
    torch.cuda.synchronize()
    return P.dp_pix_store(recs[0]), img.cpu().numpy()


def test_keyed_release_reconstruct_matches_per_frame_calls():
    M, N = 200, 352
    clip = synth.moving_rect_clip(seed=4, frames=4, M=M, N=N)
    plan = P.Plan(M=M, N=N, source=P.SRC_VARIANCE, dtype=P.REC_F32, **VAR)
    keys = [(3, 9), (0, 0), (3, 10), (2**24 - 1, 2**33 + 1)]
    recs, imgs = P.dp_pix_release_reconstruct_keyed(plan, torch.from_numpy(clip).cuda(), keys)
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    imgs = imgs.cpu().numpy()
    for i, (sid, fidx) in enumerate(keys):
        r1, i1 = plan.release_reconstruct(torch.from_numpy(clip[i]).cuda(), None, stream_id=sid, frame_idx0=fidx)
        torch.cuda.synchronize()
        assert P.dp_pix_store(recs[i]) == P.dp_pix_store(r1[0]), i
        assert np.array_equal(imgs[i], i1.cpu().numpy()), i


def _heap_head(n_cams, n_streams):
    a256 = lambda x: (x + 255) // 256 * 256
    return a256(8 * n_cams) + n_streams * a256(256 * 16)


def test_server_admits_by_memory_and_batches_bursts():
    """Memory is handed out per batch, not split per resolution: an arena that holds four frames of the
    largest camera (with their images) at once takes a burst of that camera's frames four at a time, and a
    mixed burst beyond the arena still completes, every result equal to the frame released alone."""
    pools = _pools(3, seed=10)
    big = 3  # 200 x 352
    probe = P.Server(SIZES, arena_bytes=64 << 20, **{k: v for k, v in VAR.items() if k != "C"})
    per_big = probe.slot_bytes[big] + probe.recon_bytes[big]
    probe.close()
    arena = _heap_head(len(SIZES), 2) + 4 * per_big + 1024
    srv = P.Server(SIZES, arena_bytes=arena, n_streams=2, **{k: v for k, v in VAR.items() if k != "C"})
    try:
        host = [[torch.from_numpy(p[i]).pin_memory() for i in range(len(p))] for p in pools]
        # a burst of the largest camera only: memory, not a per-resolution share, limits it
        sent = []
        for k in range(8):
            fr = host[big][k % 3]
            out = srv.image_buffer(big)
            sent.append((big, srv.submit(big, fr, srv.record_buffer(big), out), fr, out))
        # then a mixed burst, some with images and some without
        for k in range(16):
            c = k % len(SIZES)
            fr = host[c][k % 3]
            out = srv.image_buffer(c) if k % 3 else None
            sent.append((c, srv.submit(c, fr, srv.record_buffer(c), out), fr, out))
        ranks = {c: 0 for c in range(len(SIZES))}
        for c, t, fr, out in sent:
            r = srv.wait(t, timeout_ms=30000)
            assert r is not None and r["status"] == 0 and r["frame_idx"] == ranks[c]
            rec, img = _alone_recon(c, ranks[c], fr.numpy())
            assert bytes(r["record"][: r["record_bytes"]].numpy()) == rec
            if out is not None:
                assert np.array_equal(out.numpy(), img), (c, ranks[c])
            ranks[c] += 1
        st = srv.stats()
        assert st["completed"] == 24
        assert st["arena_bytes_in_use_max"] <= st["arena_heap_bytes"] < arena
        assert 2 <= st["frames_in_flight_max"]
        assert srv.counters() == [ranks[c] for c in range(len(SIZES))]
    finally:
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


SERVE_SIZES = [(720, 1280), (1080, 1920), (2160, 3840)]  # the serving workload's three camera resolutions


def test_server_config5_resolutions_agree_with_oracle():
    """Two frames of each of the serving workload's resolutions (1280 x 720, 1920 x 1080, 3840 x 2160) through
    the server with their images: records against the oracle value by value, images equal to the oracle's
    reconstruction of the served record and, up to rint ties, of the oracle's own record (Sec. VI-F)."""
    clips = [synth.moving_rect_clip(seed=60 + c, frames=2, M=M, N=N) for c, (M, N) in enumerate(SERVE_SIZES)]
    srv = P.Server(SERVE_SIZES, arena_bytes=512 << 20, n_streams=3, first_frame=[5, 0, 2**32 + 7],
                   **{k: v for k, v in VAR.items() if k != "C"})
    try:
        sent = []
        for i in range(2):
            for c in range(len(SERVE_SIZES)):
                fr = torch.from_numpy(clips[c][i]).pin_memory()
                out = srv.image_buffer(c)
                sent.append((c, i, srv.submit(c, fr, srv.record_buffer(c), out), out))
        first = [5, 0, 2**32 + 7]
        for c, i, t, out in sent:
            r = srv.wait(t, timeout_ms=60000)
            assert r is not None and r["status"] == 0
            assert r["frame_idx"] == first[c] + i
            got = bytes(r["record"][: r["record_bytes"]].numpy())
            M, N = SERVE_SIZES[c]
            rec, means, sums, etas = O.release(clips[c][i], None, M=M, N=N, source=O.SRC_VARIANCE, dtype=O.DT_F32,
                                               stream_id=c, frame_idx=first[c] + i, **VAR)
            compare_records(got, rec, means, sums, etas, O.DT_F32)
            img = out.numpy()
            assert np.array_equal(img, O.reconstruct(np.frombuffer(got, dtype=np.uint8), 0))
            ref = O.reconstruct(rec, 0).astype(np.int16)
            d = np.abs(img.astype(np.int16) - ref)
            assert d.max() <= 1 and (d > 0).mean() < 1e-3
        assert srv.counters() == [first[c] + 2 for c in range(len(SERVE_SIZES))]
    finally:
        srv.close()


def test_server_restart_continues_frame_counters():
    """Serve k frames per camera, read the device counters, restart with them: the new server keys the next
    frames k.., so its records differ from those of a fresh server (which would redraw the first server's
    noise: the same keys give the same draws) and equal the frames released alone with keys k.."""
    cams = SIZES[:2]
    pools = [synth.moving_rect_clip(seed=70 + c, frames=3, M=M, N=N) for c, (M, N) in enumerate(cams)]
    host = [[torch.from_numpy(p[i]).pin_memory() for i in range(3)] for p in pools]
    kw = {k: v for k, v in VAR.items() if k != "C"}

    def serve(srv):
        sent = [(c, i, srv.submit(c, host[c][i], srv.record_buffer(c))) for i in range(3) for c in range(2)]
        res = {}
        for c, i, t in sent:
            r = srv.wait(t, timeout_ms=30000)
            assert r["status"] == 0
            res[(c, i)] = (r["frame_idx"], bytes(r["record"][: r["record_bytes"]].numpy()))
        return res

    a = P.Server(cams, arena_bytes=64 << 20, **kw)
    try:
        ra = serve(a)
        counters = a.counters()
    finally:
        a.close()
    assert counters == [3, 3]
    b = P.Server(cams, arena_bytes=64 << 20, first_frame=counters, **kw)
    try:
        rb = serve(b)
        assert b.counters() == [6, 6]
    finally:
        b.close()
    fresh = P.Server(cams, arena_bytes=64 << 20, **kw)
    try:
        rf = serve(fresh)
    finally:
        fresh.close()
    for (c, i), (fidx, rec) in rb.items():
        assert fidx == 3 + i
        assert rec == _alone(c, 3 + i, pools[c][i])
        assert ra[(c, i)][0] == i and rf[(c, i)] == ra[(c, i)]  # same keys, same records
        pa = O.record_payload(np.frombuffer(ra[(c, i)][1], dtype=np.uint8))
        pb = O.record_payload(np.frombuffer(rec, dtype=np.uint8))
        assert pa.shape == pb.shape and np.mean(pa != pb) > 0.3  # fresh noise for the same frame


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
        with pytest.raises(ValueError):
            srv.submit(0, fr, srv.record_buffer(0), torch.zeros(16, dtype=torch.uint8))
    finally:
        srv.close()
    with pytest.raises(P.DppixError):
        P.Server(SIZES, arena_bytes=1 << 16, **{k: v for k, v in VAR.items() if k != "C"})
    with pytest.raises(ValueError):
        P.Server(SIZES, arena_bytes=64 << 20, first_frame=[0], **{k: v for k, v in VAR.items() if k != "C"})


def test_keys_advance_in_a_captured_graph():
    """dp_pix_keys_advance and the keyed release + reconstruction captured in one CUDA graph: every replay
    releases the next frames of the stream (fresh keys), byte-identical to direct calls at those indices."""
    F, M, N = 3, 130, 250
    clip = torch.from_numpy(synth.moving_rect_clip(seed=5, frames=F, M=M, N=N)).cuda()
    plan = P.Plan(M=M, N=N, source=P.SRC_VARIANCE, dtype=P.REC_F32, **VAR)
    keys = P.key_table([(7, 100 + i) for i in range(F)])
    recs, ws = plan.alloc_records(F), plan.alloc_workspace(F)
    out = torch.empty((F, M, N, 3), dtype=torch.uint8, device="cuda")

    def step():
        P.dp_pix_keys_advance(keys, F)
        P.dp_pix_release_reconstruct_keyed(plan, clip, keys, records=recs, out=out, ws=ws)

    step()  # frames 100 + F ..
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for k in range(2):  # frames 100 + 2F .., then 100 + 3F ..
        g.replay()
        torch.cuda.synchronize()
        assert P.dp_pix_status() == 0
        ref_r, ref_o = plan.release_reconstruct(clip, None, stream_id=7, frame_idx0=100 + (2 + k) * F)
        torch.cuda.synchronize()
        for i in range(F):
            got = P.dp_pix_store(recs[i])
            assert got == P.dp_pix_store(ref_r[i]), (k, i)
            assert P.record_header(got)["frame_idx"] == 100 + (2 + k) * F + i
        assert torch.equal(out, ref_o)
