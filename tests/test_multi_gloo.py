"""The N > 1 host logic of bench.py on CPU: two gloo ranks on 127.0.0.1.

The path shards by whole clips with no data-path collective (cells, tiles and frames are independent,
Thm 3), so what needs checking off the GPU is the launch plumbing: rank/world discovery, the barrier, the
max-over-ranks step time and the whole-job aggregate, the reference arm running on rank 0 only, and that
the noise of a rank depends on its stream id and not on where it runs (the keyed counter of Sec. IV-B)."""
import io
import json
import os
import socket
from contextlib import redirect_stdout

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    try:
        import torch.distributed as dist

        import oracle as O
        w, r, _ = bench.dist_setup(world)
        assert (w, r) == (world, rank)
        assert dist.get_backend() == "gloo"
        bench.barrier(w)
        ms = bench.max_over_ranks(1.0 + 2.5 * rank, w)  # rank 1 is the slow one
        # each rank releases its own tiny frame with stream id = rank (as bench.py does)
        rng = np.random.default_rng(5)
        img = rng.integers(0, 256, size=(40, 56, 3), dtype=np.uint8)
        kw = dict(M=40, N=56, C=3, grids=[8, 4], eps=[1.0, 0.5], source=O.SRC_VARIANCE, dtype=O.DT_F32, seed=3, m=16)
        mine, *_ = O.release(img, None, stream_id=rank, **kw)
        recs = [None] * w
        dist.all_gather_object(recs, bytes(mine))
        # what rank 1 released, recomputed here: placement does not change a record
        other, *_ = O.release(img, None, stream_id=1 - rank, **kw)
        bench.barrier(w)
        dist.destroy_process_group()
        q.put((rank, ms, recs, bytes(other)))
    except Exception as e:  # report to the parent instead of hanging it
        q.put((rank, repr(e), None, None))


@pytest.mark.timeout(180)
def test_two_gloo_ranks_barrier_max_and_placement():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        rank, ms, recs, other = q.get(timeout=150)
        res[rank] = (ms, recs, other)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank in range(2):
        ms, recs, other = res[rank]
        assert not isinstance(ms, str), ms
        assert ms == pytest.approx(3.5)  # the max over ranks, on every rank
        assert recs[0] != recs[1]  # stream ids give independent noise
        assert other == recs[1 - rank]  # and a record does not depend on the rank that made it
    assert res[0][1] == res[1][1]


def test_reference_arm_runs_on_rank0_only(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        gpus, steps, warmup = 2, 3, 3
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(A()) == 0
    assert buf.getvalue() == ""


def test_whole_job_value_is_units_of_all_ranks_over_max_time():
    # value = world * frames * M * N / max-over-ranks step time
    for world in (1, 2, 8):
        v = bench.whole_job_mpx_per_s(world, 4.0)
        assert v == pytest.approx(world * bench.F * bench.M * bench.N / 1e6 / 4e-3)


def test_finish_prints_one_json_line_on_rank0_only():
    class A:
        steps, warmup, path = 5, 3, "fused"
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.finish(A(), 1, 1, 1.0, 1.0, {}, None, None, {}, 0, {})
    assert buf.getvalue() == ""
    with redirect_stdout(buf):
        bench.finish(A(), 0, 1, 123.0, 2.0, {"bound": "hbm"}, None, None, {}, 3, {})
    lines = buf.getvalue().strip().splitlines()
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches"):
        assert k in d, k
    assert d["scaling"] == "weak" and d["config"]["workload"] == bench.WORKLOAD
