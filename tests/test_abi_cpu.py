"""The C-ABI library on a machine without a GPU: it loads, exports every declared entry point, and its
host-only plan agrees with the oracle's geometry and validation (no compute call is made here)."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_2511_04261_b300 as P
from paper_2511_04261_b300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^DPPIX_API\s+[\w\s\*]+?\b(dp_pix_\w+)\s*\(", txt, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    names = declared_symbols()
    assert {"dp_pix_plan", "dp_pix_release", "dp_pix_store", "dp_pix_reconstruct"} <= names
    lib = ct.CDLL(_lib.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_version_and_last_error():
    L = _lib.lib()
    assert L.dp_pix_version() >= 10000
    with pytest.raises(P.DppixError) as e:
        P.Plan(M=0, N=5, C=3, grids=[4], eps=[1])
    assert e.value.code == _lib.E_INVALID_ARG
    assert b"M and N" in L.dp_pix_last_error()


def test_compute_calls_fail_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("has a GPU")
    L = _lib.lib()
    rc = L.dp_pix_status(None, None)
    assert rc == _lib.E_CUDA


@pytest.mark.parametrize("seed", range(40))
def test_plan_geometry_matches_oracle(seed):
    rng = np.random.default_rng(seed)
    K = int(rng.integers(1, 5))
    pool = [1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24, 32]
    grids = [int(rng.choice(pool)) for _ in range(K)]
    M, N, C = int(rng.integers(1, 300)), int(rng.integers(1, 300)), int(rng.choice([1, 3, 4]))
    eps = [float(rng.uniform(0.1, 3)) for _ in range(K)]
    pad = int(rng.integers(0, 2))
    dtype = int(rng.integers(0, 3))
    kw = dict(M=M, N=N, C=C, grids=grids, eps=eps, pad_mode=pad, dtype=dtype, m=float(rng.uniform(1, 64)))
    orc = O.geometry_rc(**kw)
    try:
        plan = P.Plan(**kw)
    except P.DppixError as e:
        # the library may refuse what it does not support; a padding refusal must be the oracle's too
        assert e.code in (_lib.E_UNSUPPORTED, _lib.E_PAD_TOO_LARGE), e
        if e.code == _lib.E_PAD_TOO_LARGE:
            assert orc == -2
        return
    assert orc == 0
    g = O.geometry(**kw)
    assert (plan.T, plan.GR, plan.GC) == (g["T"], g["GR"], g["GC"])
    assert plan.record_bytes == g["capacity"]
    np.testing.assert_allclose(plan.sigma, g["sigma"], rtol=1e-15)


def test_plan_limits():
    with pytest.raises(P.DppixError) as e:
        P.Plan(M=200, N=200, C=3, grids=[129], eps=[1])
    assert e.value.code == _lib.E_UNSUPPORTED
    # the paper's largest grid (b = 128) and its region-adaptive pairs {128, 128 / n} fit
    assert P.Plan(M=1080, N=1920, C=3, grids=[128], eps=[0.5]).T == 128
    assert P.Plan(M=1152, N=1536, C=3, grids=[128, 1], eps=[0.5, 0.5], source=_lib.SRC_MATTE_F32).T == 128
    # one-pixel cells of a 1080p frame: 2,073,600 tiles, finalised from global memory
    p1 = P.Plan(M=1080, N=1920, C=1, grids=[1], eps=[0.5])
    assert (p1.GR, p1.GC) == (1080, 1920)
    with pytest.raises(P.DppixError) as e:
        P.Plan(M=8192, N=8192, C=1, grids=[1], eps=[0.5])  # 2^26 tiles
    assert e.value.code == _lib.E_UNSUPPORTED
    with pytest.raises(P.DppixError) as e:
        P.Plan(M=100, N=100, C=3, grids=[64, 3], eps=[1, 1])  # T = 192
    assert e.value.code == _lib.E_UNSUPPORTED
    with pytest.raises(P.DppixError) as e:
        P.Plan(M=100, N=100, C=3, grids=[8, 4], eps=[1, 1], source=_lib.SRC_MASK_U8, pad_mode=7)
    assert e.value.code == _lib.E_INVALID_ARG
    with pytest.raises(P.DppixError) as e:
        P.Plan(M=100, N=100, C=3, grids=[8, 4, 2], eps=[1, 1, 1], source=_lib.SRC_MASK_U8)
    assert e.value.code == _lib.E_INVALID_ARG
    with pytest.raises(P.DppixError) as e:
        P.Plan(M=4000, N=4000, C=3, grids=[32, 16], eps=[1, 1], source=_lib.SRC_VARIANCE)  # 15625 tiles ok
        P.Plan(M=8000, N=8000, C=3, grids=[32, 16], eps=[1, 1], source=_lib.SRC_VARIANCE)  # 62500 > 16384
    assert e.value.code == _lib.E_UNSUPPORTED
    with pytest.raises(P.DppixError) as e:
        P.Plan(M=10, N=10, C=3, grids=[8], eps=[-1])
    assert e.value.code == _lib.E_INVALID_ARG
    P.Plan(M=10, N=10, C=3, grids=[8], eps=[0], noise_free=True)


def test_variance_plan_paths():
    one = P.Plan(M=1080, N=1920, C=3, grids=[32, 16, 8, 4], eps=[2, 1, .5, .25], source=_lib.SRC_VARIANCE)
    two = P.Plan(M=1080, N=1920, C=3, grids=[6, 20], eps=[.5, 1.5], source=_lib.SRC_VARIANCE)
    # one-pass keeps (T/g)^2 * C u16 g-cell sums per tile in the workspace; two-pass keeps only keys/offsets
    assert one.ws_per_frame > 2040 * 64 * 3 * 2
    assert two.ws_per_frame < 20 * 1024


def test_plan_tuning_knobs():
    plan = P.Plan(M=1080, N=1920, C=3, grids=[32, 16, 8, 4], eps=[2, 1, .5, .25], source=P.SRC_VARIANCE)
    assert plan.tuning(P.TUNE_FUSED_PX) == 1024 and plan.tuning(P.TUNE_FUSED_THREADS) == 128
    plan.tune(P.TUNE_FUSED_PX, 512).tune(P.TUNE_FUSED_THREADS, 256)
    assert plan.tuning(P.TUNE_FUSED_PX) == 512 and plan.tuning(P.TUNE_FUSED_THREADS) == 256
    assert plan.tuning(P.TUNE_SPLIT) == 1
    plan.tune(P.TUNE_SPLIT, 4)
    assert plan.tuning(P.TUNE_SPLIT) == 4
    assert plan.tuning(P.TUNE_FUSED_CAP) == 0
    plan.tune(P.TUNE_FUSED_CAP, 3)
    assert plan.tuning(P.TUNE_FUSED_CAP) == 3
    for knob, bad in [(P.TUNE_FUSED_PX, 63), (P.TUNE_FUSED_PX, 4096), (P.TUNE_FUSED_THREADS, 160),
                      (P.TUNE_SPLIT, 0), (P.TUNE_SPLIT, 17), (P.TUNE_FUSED_CAP, -1), (P.TUNE_FUSED_CAP, 33), (99, 1)]:
        with pytest.raises(P.DppixError) as e:
            plan.tune(knob, bad)
        assert e.value.code == _lib.E_INVALID_ARG
    assert plan.tuning(P.TUNE_FUSED_PX) == 512


def test_soft_sizes_and_validation():
    """dp_pix_soft_sizes is host-only: the per-cell buffer size and the argument checks."""
    spec = P.SoftSpec(grids=(8, 16), eps=(0.5, 1.0), R=1.0, m=16.0)
    import torch
    x = torch.empty((32, 3, 1024, 1024), device="meta")
    d = spec.desc(x)
    nb = ct.c_uint64(0)
    assert _lib.lib().dp_pix_soft_sizes(ct.byref(d), ct.byref(nb)) == 0
    assert nb.value == 4 * 32 * 3 * (128 * 128 + 64 * 64)
    d.grid[1] = 0
    assert _lib.lib().dp_pix_soft_sizes(ct.byref(d), ct.byref(nb)) == _lib.E_INVALID_ARG or \
        _lib.lib().dp_pix_soft_sizes(ct.byref(d), ct.byref(nb)) == _lib.E_UNSUPPORTED
    d.grid[1] = 16
    d.H, d.W = 5, 5  # 16-pixel cells need 11 mirrored rows, more than a 5-row image has
    assert _lib.lib().dp_pix_soft_sizes(ct.byref(d), ct.byref(nb)) == _lib.E_PAD_TOO_LARGE
    d.H, d.W = 9, 9
    assert _lib.lib().dp_pix_soft_sizes(ct.byref(d), ct.byref(nb)) == 0
    assert nb.value == 4 * 32 * 3 * (2 * 2 + 1)
