"""Pins of the CPU oracle against things other than itself (CPU only).

Each test ties one oracle function to a library routine, a closed form from the paper, an invariant the
paper's theorems imply, or brute force on tiny inputs, chosen so that a dropped term, a wrong sign or
index, or a transposed operand fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NP_MODE = {0: "reflect", 1: "symmetric"}


# ------------------------------------------------------------------------------------------------------
# Philox
# ------------------------------------------------------------------------------------------------------
def _numpy_philox_block(ctr, key):
    """numpy's Philox (4x64-10) returns the block of counter c+1 when its state counter is c."""
    c = int(ctr[0]) | int(ctr[1]) << 64 | int(ctr[2]) << 128 | int(ctr[3]) << 192
    c = (c - 1) % (1 << 256)
    cw = [(c >> (64 * i)) & (2**64 - 1) for i in range(4)]
    # uint64 arrays: numpy would round large python ints through float64
    g = np.random.Philox(counter=np.array(cw, dtype=np.uint64), key=np.array([int(key[0]), int(key[1])], dtype=np.uint64))
    return np.array(g.random_raw(4), dtype=np.uint64)


def test_philox4x64_matches_numpy():
    rng = np.random.default_rng(7)
    cases = [([0, 0, 0, 0], [0, 0]), ([1, 0, 0, 0], [0, 0]), ([2**64 - 1] * 4, [2**64 - 1] * 2)]
    for _ in range(200):
        cases.append((rng.integers(0, 2**64, size=4, dtype=np.uint64), rng.integers(0, 2**64, size=2, dtype=np.uint64)))
    for ctr, key in cases:
        got = O.philox4x64_10(ctr, key)
        exp = _numpy_philox_block(ctr, key)
        assert np.array_equal(got, exp), (ctr, key, got, exp)


def test_philox4x32_uniform_and_balanced():
    # 4x32 shares the round/key-schedule macro pinned above; its constants are pinned by the known-answer test below.
    words = []
    for i in range(30000):
        words.extend(O.philox4x32_10([i, 7, 3, 0], [0x12345678, 0x9ABCDEF0]))
    w = np.array(words, dtype=np.uint64)
    u = (w.astype(np.float64) + 0.5) / 2**32
    assert stats.kstest(u, "uniform").pvalue > 0.01
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint64)) & 1).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 0.01)
    # distinct counters / keys give distinct blocks
    a = O.philox4x32_10([0, 0, 0, 0], [0, 0])
    assert not np.array_equal(a, O.philox4x32_10([1, 0, 0, 0], [0, 0]))
    assert not np.array_equal(a, O.philox4x32_10([0, 0, 0, 0], [1, 0]))
    assert not np.array_equal(a, O.philox4x32_10([0, 0, 0, 1], [0, 0]))


def test_philox4x32_known_answer_vectors():
    """Philox4x32-10's multipliers (0xD2511F53, 0xCD9E8D57) and Weyl constants (0x9E3779B9, 0xBB67AE85)
    are pinned by the published known-answer vectors of the generator (Salmon, Moraes, Dror, Shaw,
    "Parallel random numbers: as easy as 1, 2, 3", SC'11; the Random123 distribution's kat_vectors file,
    rows "philox4x32 10"): counter and key all zero, all ones, and the row built from the hex digits of pi.
    A single mistyped constant changes every output word of every row."""
    rows = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for ctr, key, exp in rows:
        got = O.philox4x32_10(ctr, key)
        assert [int(w) for w in got] == exp, (ctr, key, ["%08x" % int(w) for w in got])


# ------------------------------------------------------------------------------------------------------
# Laplace sampler (Eq. 9)
# ------------------------------------------------------------------------------------------------------
def test_laplace_inverse_cdf_closed_form():
    sigma = 3.7
    for x in [0, 1, 2, 12345, 2**31 - 2, 2**31 - 1, 2**31, 2**31 + 1, 2**32 - 3, 2**32 - 1, 987654321, 3456789012]:
        eta = O.laplace_from_word(x, sigma)
        # the draw is the inverse CDF at the cell midpoint u = (x + 1/2) / 2^32
        u = stats.laplace.cdf(eta, loc=0.0, scale=sigma)
        assert u == pytest.approx((x + 0.5) / 2**32, rel=1e-12, abs=1e-300)


def test_laplace_antisymmetric_and_monotone():
    sigma = 1.0
    xs = np.random.default_rng(3).integers(0, 2**32, size=2000, dtype=np.uint64)
    for x in xs[:500]:
        assert O.laplace_from_word(int(x), sigma) == -O.laplace_from_word(2**32 - 1 - int(x), sigma)
    srt = np.sort(xs)
    vals = [O.laplace_from_word(int(x), sigma) for x in srt]
    assert all(b >= a for a, b in zip(vals, vals[1:]))
    assert O.laplace_from_word(0, 1.0) == pytest.approx(-32 * math.log(2))


def test_laplace_ks_and_scale():
    sigma = 127.5
    xs = np.random.default_rng(11).integers(0, 2**32, size=100000, dtype=np.uint64)
    eta = np.array([O.laplace_from_word(int(x), sigma) for x in xs])
    assert stats.kstest(eta / sigma, "laplace").pvalue > 0.01
    assert np.mean(np.abs(eta)) == pytest.approx(sigma, rel=0.02)  # E|eta| = sigma for Laplace(0, sigma)


# ------------------------------------------------------------------------------------------------------
# Geometry, padding and sensitivity (Eq. 11, Alg. 2 steps 1-4, Alg. 3 steps 1-3, Eq. 16-17)
# ------------------------------------------------------------------------------------------------------
def test_reflect_matches_numpy_pad():
    for n in range(1, 40):
        for mode in (0, 1):
            pmax = n - 1 if mode == 0 else n
            if pmax == 0:
                continue
            arr = np.arange(n)
            padded = np.pad(arr, (0, pmax), mode=NP_MODE[mode])
            got = [O.reflect(p, n, mode) for p in range(n + pmax)]
            assert got == list(padded)


def test_geometry_closed_forms():
    with open(os.path.join(GOLDEN, "paper_settings.json")) as f:
        settings = json.load(f)["settings"]
    for s in settings:
        g = O.geometry(M=s["M"], N=s["N"], C=1, grids=[s["b"]], eps=[s["eps"]], m=s["m"])
        # Eq. 11 with Eq. 8: sigma = 255 m / (b^2 eps)
        assert g["sigma"][0] * s["b"] ** 2 * s["eps"] == pytest.approx(255 * s["m"], rel=1e-15)
        # G_R = ceil(M / b), P_R = G_R b - M (Table II, Alg. 3 steps 1-2)
        assert g["GR"] == -(-s["M"] // s["b"]) and g["GC"] == -(-s["N"] // s["b"])
        assert g["PR"] == g["GR"] * s["b"] - s["M"] and g["PC"] == g["GC"] * s["b"] - s["N"]
    # Eq. 16-17: b = n s_b, Delta = Delta_s / n^2, T = b (the simple grid) when s_b divides b
    for b, n in [(32, 8), (24, 3), (16, 4), (128, 8), (12, 1)]:
        sb = b // n
        g = O.geometry(M=300, N=400, C=3, grids=[b, sb], eps=[0.5, 0.5], m=32)
        assert g["T"] == b
        assert g["sigma"][0] == pytest.approx(g["sigma"][1] / n**2, rel=1e-15)
    # general K: T = lcm{b_r}
    g = O.geometry(M=1000, N=1000, C=3, grids=[6, 20], eps=[0.5, 1.5], m=32)
    assert g["T"] == math.lcm(6, 20) == 60
    g = O.geometry(M=1080, N=1920, C=3, grids=[32, 16, 8, 4], eps=[2, 1, 0.5, 0.25], m=16)
    assert g["T"] == 32 and g["GR"] == 34 and g["GC"] == 60
    assert g["sigma"] == pytest.approx([255 * 16 / (b * b * e) for b, e in [(32, 2), (16, 1), (8, .5), (4, .25)]])


def test_geometry_rejects_padding_beyond_image():
    # reflect needs P <= n - 1, symmetric P <= n
    assert O.geometry_rc(M=5, N=8, C=1, grids=[8], eps=[1]) == 0  # P_R = 3 <= 4
    assert O.geometry_rc(M=3, N=8, C=1, grids=[8], eps=[1]) == -2  # P_R = 5 > 2
    assert O.geometry_rc(M=4, N=8, C=1, grids=[8], eps=[1], pad_mode=1) == 0  # P_R = 4 <= 4
    assert O.geometry_rc(M=4, N=8, C=1, grids=[8], eps=[1], pad_mode=0) == -2
    assert O.geometry_rc(M=8, N=8, C=1, grids=[8], eps=[0]) == -1
    assert O.geometry_rc(M=8, N=8, C=1, grids=[8], eps=[0], noise_free=True) == 0


# ------------------------------------------------------------------------------------------------------
# Cell sums and block means by brute force / numpy (Eq. 2, Alg. 2 steps 4-6)
# ------------------------------------------------------------------------------------------------------
def _np_cell_sums(img, b, T, mode):
    """numpy reference: mirror-pad to whole tiles, reshape into b x b cells, sum; [GR*T/b, GC*T/b, C]."""
    M, N, C = img.shape
    GR, GC = -(-M // T), -(-N // T)
    P = np.pad(img.astype(np.int64), ((0, GR * T - M), (0, GC * T - N), (0, 0)), mode=NP_MODE[mode])
    return P.reshape(GR * T // b, b, GC * T // b, b, C).sum(axis=(1, 3))


def _np_expected_payload(img, labels, grids, T, mode):
    """Record-order payload of exact sums built from numpy cell sums and the documented order."""
    out = []
    for r, b in enumerate(grids):
        S = _np_cell_sums(img, b, T, mode)
        cs = T // b
        for ty, tx in zip(*np.nonzero(labels == r)):
            blk = S[ty * cs:(ty + 1) * cs, tx * cs:(tx + 1) * cs, :]
            out.append(blk.reshape(-1))
    return np.concatenate(out) if out else np.zeros(0, dtype=np.int64)


@pytest.mark.parametrize("M,N,C,grids,mode", [
    (17, 23, 3, [4, 2], 0), (24, 24, 3, [8, 24], 0), (31, 45, 1, [6, 20], 0), (13, 29, 4, [4, 8, 16], 1),
    (50, 70, 3, [5], 0), (9, 9, 3, [1, 3, 9], 1), (61, 61, 3, [6, 20], 1), (33, 35, 3, [32, 16, 8, 4], 0),
])
def test_cell_sums_brute_force(M, N, C, grids, mode):
    rng = np.random.default_rng(M * 100 + N)
    img = rng.integers(0, 256, size=(M, N, C), dtype=np.uint8)
    T = math.lcm(*grids)
    GR, GC = -(-M // T), -(-N // T)
    if (mode == 0 and (GR * T - M > M - 1 or GC * T - N > N - 1)) or (GR * T - M > M or GC * T - N > N):
        pytest.skip("padding larger than the image")
    labels = rng.integers(0, len(grids), size=(GR, GC), dtype=np.uint8)
    rec, means, sums, eta = O.release(img, labels, grids=grids, eps=[1.0] * len(grids), pad_mode=mode,
                                      source=O.SRC_TILE_LABELS, dtype=O.DT_SUM, seed=5)
    exp = _np_expected_payload(img, labels, grids, T, mode)
    assert np.array_equal(sums, exp)
    assert np.array_equal(O.record_payload(rec), exp)
    # the tiny cases also by a pure-python loop over the definition (Eq. 2)
    if M * N <= 600:
        k = 0
        for r, b in enumerate(grids):
            for ty in range(GR):
                for tx in range(GC):
                    if labels[ty, tx] != r:
                        continue
                    for cy in range(T // b):
                        for cx in range(T // b):
                            for ch in range(C):
                                s = 0
                                for y in range(ty * T + cy * b, ty * T + cy * b + b):
                                    for x in range(tx * T + cx * b, tx * T + cx * b + b):
                                        yy = y if y < M else (2 * (M - 1) - y if mode == 0 else 2 * M - 1 - y)
                                        xx = x if x < N else (2 * (N - 1) - x if mode == 0 else 2 * N - 1 - x)
                                        s += int(img[yy, xx, ch])
                                assert sums[k] == s
                                k += 1


def _np_block_mean_image(img, labels, grids, T, mode):
    M, N, C = img.shape
    GR, GC = labels.shape
    out = np.zeros((GR * T, GC * T, C))
    for r, b in enumerate(grids):
        S = _np_cell_sums(img, b, T, mode).astype(np.float64) / (b * b)
        full = np.repeat(np.repeat(S, b, axis=0), b, axis=1)
        m = np.repeat(np.repeat(labels == r, T, axis=0), T, axis=1)
        out[m] = full[m]
    return out[:M, :N]


@pytest.mark.parametrize("grids", [[16], [24, 8], [32, 16, 8, 4], [6, 20]])
def test_noise_free_reconstruction_is_block_mean(grids):
    """Eq. 2-3: without noise the released image is the block-mean image (Alg. 2 / Alg. 3)."""
    rng = np.random.default_rng(sum(grids))
    M, N = 97, 131
    img = rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8)
    T = math.lcm(*grids)
    GR, GC = -(-M // T), -(-N // T)
    labels = rng.integers(0, len(grids), size=(GR, GC), dtype=np.uint8)
    rec, means, sums, eta = O.release(img, labels, grids=grids, eps=[1.0] * len(grids), noise_free=True,
                                      source=O.SRC_TILE_LABELS, dtype=O.DT_F32)
    exp = _np_block_mean_image(img, labels, grids, T, 0)
    got = O.reconstruct(rec, out_type=2)
    assert np.allclose(got, exp, rtol=0, atol=255 * 2**-24)
    assert np.all(eta == 0)
    got8 = O.reconstruct(rec, out_type=0)
    assert np.array_equal(got8, np.rint(exp.astype(np.float32)).astype(np.uint8))


def test_sum_record_reconstructs_block_mean():
    """A record of exact sums rebuilds the noise-free block means (Eq. 2-3), in f32 like the means."""
    rng = np.random.default_rng(31)
    M, N, grids = 61, 77, [6, 20]
    img = rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8)
    labels = rng.integers(0, 2, size=(2, 2), dtype=np.uint8)
    rec, means, sums, eta = O.release(img, labels, grids=grids, eps=[1, 1], source=O.SRC_TILE_LABELS,
                                      dtype=O.DT_SUM)
    exp = _np_block_mean_image(img, labels, grids, 60, 0)
    got = O.reconstruct(rec, 1)
    assert np.allclose(got, exp.astype(np.float32), rtol=2**-23, atol=0)
    assert np.array_equal(O.reconstruct(rec, 0), np.rint(exp.astype(np.float32)).astype(np.uint8))


def test_uniform_special_cases():
    """n = 1 (b = s_b) makes Alg. 3 equal Alg. 2; b = 1 keeps every sample (no pixelization)."""
    rng = np.random.default_rng(2)
    img = rng.integers(0, 256, size=(40, 56, 3), dtype=np.uint8)
    mask = rng.integers(0, 2, size=(40, 56), dtype=np.uint8)
    two, *_ = O.release(img, mask, grids=[8, 8], eps=[1, 1], source=O.SRC_MASK, noise_free=True)
    one, *_ = O.release(img, np.zeros((5, 7), np.uint8), grids=[8], eps=[1], source=O.SRC_TILE_LABELS,
                        noise_free=True)
    assert np.array_equal(O.reconstruct(two, 2), O.reconstruct(one, 2))
    ident, *_ = O.release(img, np.zeros((40, 56), np.uint8), grids=[1], eps=[1], source=O.SRC_TILE_LABELS,
                          noise_free=True)
    assert np.array_equal(O.reconstruct(ident, 0), img)


# ------------------------------------------------------------------------------------------------------
# Classification (Alg. 3 steps 5-6 and the region sources)
# ------------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("M,N,T,mode", [(576, 768, 24, 0), (100, 130, 24, 0), (61, 200, 60, 1), (33, 47, 8, 0)])
def test_mask_classification_matches_numpy_mean(M, N, T, mode):
    rng = np.random.default_rng(M + N)
    mask = (rng.random((M, N)) < 0.5).astype(np.uint8)
    mask[: M // 3] = 1
    GR, GC = -(-M // T), -(-N // T)
    Mp = np.pad(mask.astype(np.float64), ((0, GR * T - M), (0, GC * T - N)), mode=NP_MODE[mode])
    mu = Mp.reshape(GR, T, GC, T).mean(axis=(1, 3))
    exp = np.where(mu > 0.5, 0, 1)  # Alg. 3 step 6: simple (region 0) iff mask mean > 0.5
    img = np.zeros((M, N, 3), np.uint8)
    got = O.classify(img, mask, grids=[T, T // 2 if T % 2 == 0 else T], eps=[1, 1], source=O.SRC_MASK,
                     pad_mode=mode)
    assert np.array_equal(got, exp)


def test_mask_tie_goes_to_complex():
    T = 8
    mask = np.zeros((8, 16), np.uint8)
    mask[:4, :8] = 1  # exactly half of tile 0 simple -> mean 0.5 -> complex
    mask[:5, 8:] = 1  # more than half of tile 1 simple -> simple
    got = O.classify(np.zeros((8, 16, 3), np.uint8), mask, grids=[8, 4], eps=[1, 1], source=O.SRC_MASK)
    assert got.tolist() == [[1, 0]]


def test_matte_classification():
    rng = np.random.default_rng(9)
    M, N, T = 130, 190, 60
    alpha = rng.random((M, N)).astype(np.float32)
    alpha[:, :70] = 0.9
    alpha[5, 5] = np.float32(0.5)  # exactly the threshold counts as complex (alpha >= thr)
    GR, GC = -(-M // T), -(-N // T)
    cplx = np.pad((alpha >= np.float32(0.5)).astype(np.int64), ((0, GR * T - M), (0, GC * T - N)), mode="reflect")
    n_simple = (1 - cplx).reshape(GR, T, GC, T).sum(axis=(1, 3))
    exp = np.where(2 * n_simple > T * T, 0, 1)
    got = O.classify(np.zeros((M, N, 3), np.uint8), alpha, grids=[20, 6], eps=[1.5, .5], source=O.SRC_MATTE)
    assert np.array_equal(got, exp)


def test_variance_quantile_classes_match_numpy_var():
    rng = np.random.default_rng(21)
    M, N, T, K = 200, 330, 32, 4
    img = rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8)
    # give tiles very different spreads so that float variances rank exactly like the integer keys
    GR, GC = -(-M // T), -(-N // T)
    spread = rng.permutation(GR * GC).reshape(GR, GC) + 1
    for ty in range(GR):
        for tx in range(GC):
            blk = img[ty * T:(ty + 1) * T, tx * T:(tx + 1) * T]
            blk[...] = (128 + (blk.astype(np.int64) - 128) * spread[ty, tx] // (GR * GC)).astype(np.uint8)
    P = np.pad(img.astype(np.float64), ((0, GR * T - M), (0, GC * T - N), (0, 0)), mode="reflect")
    var = P.reshape(GR, T, GC, T, 3).transpose(0, 2, 1, 3, 4).reshape(GR * GC, -1).var(axis=1)
    order = np.argsort(var, kind="stable")
    exp = np.zeros(GR * GC, np.uint8)
    exp[order] = (K * np.arange(GR * GC)) // (GR * GC)
    got = O.classify(img, None, grids=[32, 16, 8, 4], eps=[2, 1, .5, .25], source=O.SRC_VARIANCE)
    assert np.array_equal(got.reshape(-1), exp)
    # equal-count classes: floor(K rank / n)
    assert np.array_equal(np.bincount(got.reshape(-1), minlength=K), np.bincount(exp, minlength=K))


def test_variance_ties_ranked_by_tile_index():
    img = np.full((64, 96, 3), 77, np.uint8)  # every tile constant -> key 0 for all
    got = O.classify(img, None, grids=[32, 16], eps=[1, 1], source=O.SRC_VARIANCE)
    assert got.reshape(-1).tolist() == [0, 0, 0, 1, 1, 1]


# ------------------------------------------------------------------------------------------------------
# Record (Table III / Table IV, size formula of Sec. VI-F) and reconstruction
# ------------------------------------------------------------------------------------------------------
def test_record_size_formula_and_layout():
    rng = np.random.default_rng(4)
    M, N = 70, 100
    grids, eps = [24, 8], [1.0, 0.5]
    img = rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8)
    mask = rng.integers(0, 2, size=(M, N), dtype=np.uint8)
    for dtype, es in [(O.DT_F32, 4), (O.DT_U8, 1), (O.DT_SUM, 4)]:
        rec, means, sums, eta = O.release(img, mask, grids=grids, eps=eps, source=O.SRC_MASK, dtype=dtype, seed=9,
                                          frame_idx=3, stream_id=2)
        info = O.record_info(rec)
        T, GR, GC, K, C = 24, 3, 5, 2, 3
        a16 = lambda x: (x + 15) // 16 * 16
        exp_total = 512 + a16(GR * K * 4) + a16(GR * GC)
        for r in range(K):
            exp_total += a16(info["count"][r] * (T // grids[r]) ** 2 * C * es)
        assert info["total_bytes"] == exp_total == len(rec)
        assert sum(info["count"]) == GR * GC
        assert info["M"] == M and info["N"] == N and info["T"] == T and info["b"] == grids
        assert info["seed"] == 9 and info["frame_idx"] == 3 and info["stream_id"] == 2
        assert np.array_equal(O.record_map(rec), O.classify(img, mask, grids=grids, eps=eps, source=O.SRC_MASK))


def test_u8_record_rounds_f32_mean_half_to_even():
    """The u8 record (the paper stores uint8 noisy means, Sec. VII-A) holds the f32 mean rounded half to
    even (numpy rint), neither truncated (numpy astype) nor rounded from the fp64 value."""
    # noise-free, b = 2: a cell's mean is its sample sum / 4; sums 4k + 2 put it exactly on k + 1/2
    M, N = 8, 16
    ks = np.arange(M // 2 * N // 2) % 254
    img = np.zeros((M, N, 1), dtype=np.uint8)
    for i, k in enumerate(ks):
        cy, cx = divmod(i, N // 2)
        # samples k, k, k+1, k+1 sum to 4k + 2
        img[2 * cy:2 * cy + 2, 2 * cx:2 * cx + 2, 0] = [[k, k + 1], [k + 1, k]]
    labels = np.zeros((M // 2, N // 2), dtype=np.uint8)
    rec, means, _, _ = O.release(img, labels, grids=[2], eps=[1.0], source=O.SRC_TILE_LABELS, dtype=O.DT_U8,
                                 noise_free=True)
    assert np.array_equal(means, ks + 0.5)
    got = O.record_payload(rec)
    assert np.array_equal(got, np.rint(np.float32(means)))
    assert np.array_equal(got[ks % 2 == 0], ks[ks % 2 == 0])          # k + 1/2 -> k for even k
    assert np.array_equal(got[ks % 2 == 1], ks[ks % 2 == 1] + 1)      # k + 1/2 -> k + 1 for odd k
    # noisy release: the u8 payload is rint of the f32 payload of the same release, value by value
    rng = np.random.default_rng(12)
    img = rng.integers(0, 256, size=(70, 90, 3), dtype=np.uint8)
    mask = rng.integers(0, 2, size=(70, 90), dtype=np.uint8)
    kw = dict(grids=[24, 8], eps=[1.0, 0.5], source=O.SRC_MASK, seed=5, frame_idx=2)
    rec32, means32, _, _ = O.release(img, mask, dtype=O.DT_F32, **kw)
    rec8, means8, _, _ = O.release(img, mask, dtype=O.DT_U8, **kw)
    assert np.array_equal(means32, means8)
    f32 = O.record_payload(rec32)
    assert np.array_equal(f32, np.float32(means32).astype(np.float64))
    u8 = O.record_payload(rec8)
    assert np.array_equal(u8, np.rint(np.float32(means32)))
    frac = np.float32(means32) - np.floor(np.float32(means32))
    assert np.any(frac > 0.5) and np.any((frac > 0) & (frac < 0.5))   # both rounding directions occur


def test_reconstruct_broadcasts_record_values():
    """Reconstruction puts each stored value on every pixel of its cell (Sec. VI-F), built here from the
    record's documented order by numpy repeat."""
    rng = np.random.default_rng(5)
    M, N, grids = 64, 90, [16, 4]
    img = rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8)
    T = 16
    GR, GC = 4, 6
    labels = rng.integers(0, 2, size=(GR, GC), dtype=np.uint8)
    rec, means, sums, eta = O.release(img, labels, grids=grids, eps=[.5, .25], source=O.SRC_TILE_LABELS, seed=77)
    vals = O.record_payload(rec)
    full = np.zeros((GR * T, GC * T, 3))
    k = 0
    for r, b in enumerate(grids):
        cs = T // b
        for ty, tx in zip(*np.nonzero(labels == r)):
            blk = vals[k:k + cs * cs * 3].reshape(cs, cs, 3)
            k += cs * cs * 3
            full[ty * T:(ty + 1) * T, tx * T:(tx + 1) * T] = np.repeat(np.repeat(blk, b, 0), b, 1)
    assert np.array_equal(O.reconstruct(rec, 2), full[:M, :N])
    assert np.all((vals >= 0) & (vals <= 255))  # clip keeps [0, 255]


# ------------------------------------------------------------------------------------------------------
# Privacy invariants: noise scale, parallel composition (Thm 1, 3, 5), sensitivity (Eq. 11)
# ------------------------------------------------------------------------------------------------------
def test_noise_residuals_are_laplace_with_region_scale():
    rng = np.random.default_rng(6)
    M, N = 480, 640
    img = rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8)
    grids, eps = [16, 4], [1.0, 0.25]
    labels = (rng.random((M // 16, N // 16)) < 0.5).astype(np.uint8)
    rec, means, sums, eta = O.release(img, labels, grids=grids, eps=eps, source=O.SRC_TILE_LABELS, m=16, seed=1)
    info = O.record_info(rec)
    k = 0
    for r, b in enumerate(grids):
        n = info["count"][r] * (16 // b) ** 2 * 3
        e = eta[k:k + n]
        sigma = 255 * 16 / (b * b * eps[r])
        assert info["sigma"][r] == pytest.approx(sigma)
        assert stats.kstest(e / sigma, "laplace").pvalue > 0.01
        # residual of the unclipped mean equals eta (mean = S / b^2)
        pre = sums[k:k + n] / (b * b) + e
        assert np.allclose(np.clip(pre, 0, 255), means[k:k + n], rtol=0, atol=1e-9)
        k += n


def test_parallel_composition_cells_independent():
    rng = np.random.default_rng(8)
    M, N, grids = 96, 96, [32, 8]
    img = rng.integers(0, 256, size=(M, N, 3), dtype=np.uint8)
    labels = np.array([[0, 1, 0], [1, 1, 0], [0, 0, 1]], np.uint8)
    kw = dict(grids=grids, eps=[1, .5], source=O.SRC_TILE_LABELS, seed=3)
    rec_a, ma, *_ = O.release(img, labels, **kw)
    img2 = img.copy()
    img2[40:48, 72:80] = 255 - img2[40:48, 72:80]  # one b=8 cell inside tile (1, 2) is region 0 (b = 32)
    rec_b, mb, *_ = O.release(img2, labels, **kw)
    diff = np.nonzero(ma != mb)[0]
    # region 0 tiles in row-major order: (0,0) (0,2) (1,2) (2,0) (2,1); tile (1,2) is the third -> values 6..8
    assert set(diff.tolist()) <= {6, 7, 8} and len(diff) > 0
    # every other cell is bit-identical, including all noise draws
    keep = np.setdiff1d(np.arange(len(ma)), [6, 7, 8])
    assert np.array_equal(ma[keep], mb[keep])
    # releasing one region alone (other tiles relabelled) leaves region-1 values unchanged
    rec_c, mc, *_ = O.release(img, labels, **kw)
    assert np.array_equal(ma, mc)


def test_sensitivity_bound():
    """Neighbouring images differing in at most m samples by at most 255 change the noise-free
    pixelization vector by at most 255 m / b^2 in L1 (Eq. 11), away from mirrored samples."""
    rng = np.random.default_rng(10)
    M, N, b, m = 64, 64, 8, 16
    img = rng.integers(0, 256, size=(M, N, 1), dtype=np.uint8)
    labels = np.zeros((8, 8), np.uint8)
    kw = dict(grids=[b], eps=[1.0], source=O.SRC_TILE_LABELS, noise_free=True, m=m)
    _, a, *_ = O.release(img, labels, **kw)
    worst = 0.0
    for trial in range(20):
        img2 = img.copy()
        idx = rng.choice(M * N, size=m, replace=False)
        flat = img2.reshape(-1)
        flat[idx] = np.where(flat[idx] < 128, 255, 0)
        _, c, *_ = O.release(img2, labels, **kw)
        worst = max(worst, float(np.abs(a - c).sum()))
    assert worst <= 255 * m / b**2 + 1e-9
    img3 = img.copy()
    img3.reshape(-1)[:m] = np.where(img3.reshape(-1)[:m] < 128, 255, 0)
    _, c, *_ = O.release(img3, labels, **kw)
    assert np.abs(a - c).sum() > 0


# ------------------------------------------------------------------------------------------------------
# Soft layer: analytic adjoint vs central finite differences of the forward (noise constant)
# ------------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("m", [0.05, 40.0])
def test_soft_layer_gradient_matches_finite_differences(m):
    """m = 0.05 keeps every cell unclipped; m = 40 clips many cells (zero gradient through the clip)."""
    rng = np.random.default_rng(12)
    B, C, H, W = 1, 3, 16, 16
    x = rng.random((B, C, H, W))
    w = rng.random((B, 1, H, W))
    g = rng.standard_normal((B, C, H, W))
    kw = dict(grids=(8, 16), eps=(0.5, 1.0), R=1.0, m=m, seed=4, frame0=0)
    dx, dw = O.soft_backward(x, w, g, **kw)
    _, p = O.soft_forward(x, w, **kw)
    if m > 1:
        assert np.mean((p == 0) | (p == 1)) > 0.2  # the clip is active somewhere
    h = 1e-3
    L = lambda xx, ww: float((g * O.soft_forward(xx, ww, **kw)[0]).sum())
    pts = [(ci, yi, xi) for ci in range(C) for yi in (0, 5, 8, 15) for xi in (0, 7, 9, 15)]
    for (ci, yi, xi) in pts:
        xp, xm = x.copy(), x.copy()
        xp[0, ci, yi, xi] += h
        xm[0, ci, yi, xi] -= h
        fd = (L(xp, w) - L(xm, w)) / (2 * h)
        assert dx[0, ci, yi, xi] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    for (yi, xi) in [(0, 0), (7, 7), (15, 2), (9, 13)]:
        wp, wm = w.copy(), w.copy()
        wp[0, 0, yi, xi] += h
        wm[0, 0, yi, xi] -= h
        fd = (L(x, wp) - L(x, wm)) / (2 * h)
        assert dw[0, 0, yi, xi] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_soft_layer_gradient_with_mirror_padding():
    """Padded cells count mirrored samples twice: the adjoint scatters back with multiplicity."""
    rng = np.random.default_rng(14)
    B, C, H, W = 1, 1, 13, 11
    x = rng.random((B, C, H, W))
    w = rng.random((B, 1, H, W))
    g = rng.standard_normal((B, C, H, W))
    kw = dict(grids=(4, 8), eps=(0.5, 1.0), R=1.0, m=0.05, seed=2)
    dx, dw = O.soft_backward(x, w, g, **kw)
    h = 1e-3
    L = lambda xx: float((g * O.soft_forward(xx, w, **kw)[0]).sum())
    for yi in range(H):
        for xi in (0, 5, 9, 10):
            xp, xm = x.copy(), x.copy()
            xp[0, 0, yi, xi] += h
            xm[0, 0, yi, xi] -= h
            assert dx[0, 0, yi, xi] == pytest.approx((L(xp) - L(xm)) / (2 * h), rel=1e-6, abs=1e-9)


def test_soft_layer_noise_free_is_blend_of_block_means():
    rng = np.random.default_rng(13)
    B, C, H, W = 2, 3, 32, 48
    x = rng.random((B, C, H, W))
    w = rng.random((B, 1, H, W))
    y, p = O.soft_forward(x, w, grids=(8, 16), eps=(0.5, 1), R=1.0, noise_free=True)
    def bm(b):
        m = x.reshape(B, C, H // b, b, W // b, b).mean(axis=(3, 5))
        return np.repeat(np.repeat(m, b, axis=2), b, axis=3)
    assert np.allclose(y, w * bm(8) + (1 - w) * bm(16), rtol=0, atol=1e-12)
