"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI and compare with the oracle.

Tolerance for fp32 noisy means (documented reading of the 2e-5 relative bar): the CUDA value v_g and the
oracle's fp64 value v_o may differ by at most 2e-5 * max(|v_o|, |mu|, |eta|), i.e. relative to the largest
operand of the final add, so cancellation cells (mu + eta near 0) are measured against the operands that
produced them.  Integer results (maps, layouts, sums, u8 away from .5 ties) must match exactly.
"""
import numpy as np
import torch

import oracle as O
import paper_2511_04261_b300 as P

REL_TOL = 2e-5


def gpu_release(img, src=None, frames=1, pitch=None, frame_idx0=0, stream_id=0, **kw):
    """img: numpy u8 [F, M, N, C] / [M, N, C] (or [F, M, pitch] with pitch).  Returns list of host record bytes."""
    plan = P.Plan(pitch=pitch, **kw)
    t = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    s = None
    if src is not None:
        s = torch.from_numpy(np.ascontiguousarray(src)).cuda()
    recs = plan.release(t, s, stream_id=stream_id, frame_idx0=frame_idx0)
    torch.cuda.synchronize()
    assert P.dp_pix_status() == 0
    out = [P.dp_pix_store(recs[i]) for i in range(recs.shape[0])]
    return plan, recs, out


def oracle_kw(kw):
    k = dict(kw)
    k["source"] = k.pop("source", 0)
    return k


def compare_records(rec_gpu: bytes, rec_ora: np.ndarray, means, sums, etas, dtype):
    g = np.frombuffer(rec_gpu, dtype=np.uint8)
    o = np.asarray(rec_ora, dtype=np.uint8)
    assert len(g) == len(o), (len(g), len(o))
    hg, ho = O.record_info(g), O.record_info(o)
    for k in hg:
        if k == "sigma":
            np.testing.assert_allclose(hg[k], ho[k], rtol=1e-15)
        else:
            assert hg[k] == ho[k], (k, hg[k], ho[k])
    # header, tile-row index, map and the alignment gaps: bit-exact
    pay = ho["payload_offset"]
    assert np.array_equal(g[:pay], o[:pay])
    es = 1 if dtype == O.DT_U8 else 4
    for r in range(ho["K"]):  # zero gap after each region's payload
        end = ho["region_offset"][r] + ho["count"][r] * ho["cells_side"][r] ** 2 * ho["C"] * es
        assert not g[end:(end + 15) // 16 * 16].any()
    vg = O.record_payload(g)
    vo = O.record_payload(o)
    if dtype == O.DT_SUM:
        assert np.array_equal(vg, vo)
        assert np.array_equal(vg, sums)
    elif dtype == O.DT_F32:
        bound = REL_TOL * np.maximum(np.maximum(np.abs(means), np.abs(sums_mean(sums, hg))), np.abs(etas))
        err = np.abs(vg - means)
        bad = err > bound + 1e-30
        assert not bad.any(), "%d of %d values out of tolerance, worst %g" % (bad.sum(), bad.size, err.max())
    else:  # u8: exact except at .5 ties within fp32 error
        d = np.abs(vg - vo)
        assert d.max() <= 1
        frac = np.abs(means - np.floor(means) - 0.5)
        assert np.all(frac[d > 0] < 1e-3)
    return hg


def sums_mean(sums, info):
    """mu = S / b^2 per value in record order."""
    mu = np.zeros(len(sums), dtype=np.float64)
    k = 0
    for r in range(info["K"]):
        n = info["count"][r] * info["cells_side"][r] ** 2 * info["C"]
        mu[k:k + n] = sums[k:k + n] / float(info["b"][r] ** 2)
        k += n
    return mu
