"""ctypes wrapper over the C oracle (oracle/dppix_oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests/, the package smoke check and the benchmark's CPU-baseline leg.

A problem is described by keyword arguments (the same names the product binding uses, defined here
independently):
    M, N, C, grids (list of b_r), eps (list of eps_r), R=255, m=16, pad_mode=0 (reflect) | 1 (symmetric) |
    2 (no padding: edge cells use their valid samples only),
    source: 0 tile labels | 1 simple-mask u8 | 2 alpha matte f32 | 3 variance quantiles,
    matte_thr=0.5, dtype: 0 f32 | 1 u8 | 2 u32 sums, noise_free=False, stream_id=0, seed=0, frame_idx=0.
"""
import ctypes as ct
import os

import numpy as np

from . import build as _build

MAXK = 8
SRC_TILE_LABELS, SRC_MASK, SRC_MATTE, SRC_VARIANCE = 0, 1, 2, 3
PAD_REFLECT, PAD_SYMMETRIC, PAD_NONE = 0, 1, 2
DT_F32, DT_U8, DT_SUM = 0, 1, 2


class OraError(RuntimeError):
    pass


class _Desc(ct.Structure):
    _fields_ = [
        ("M", ct.c_int32), ("N", ct.c_int32), ("C", ct.c_int32), ("K", ct.c_int32),
        ("pitch", ct.c_int64),
        ("b", ct.c_int32 * MAXK), ("eps", ct.c_double * MAXK),
        ("R", ct.c_double), ("m", ct.c_double),
        ("pad_mode", ct.c_int32), ("source", ct.c_int32), ("matte_thr", ct.c_float),
        ("dtype", ct.c_int32), ("noise_free", ct.c_int32), ("stream_id", ct.c_uint32),
        ("seed", ct.c_uint64), ("frame_idx", ct.c_uint64),
    ]


class _Geom(ct.Structure):
    _fields_ = [
        ("T", ct.c_int32), ("GR", ct.c_int32), ("GC", ct.c_int32), ("PR", ct.c_int32), ("PC", ct.c_int32),
        ("cells_side", ct.c_int32 * MAXK), ("sigma", ct.c_double * MAXK),
        ("header_bytes", ct.c_uint64), ("rowidx_bytes", ct.c_uint64), ("map_offset", ct.c_uint64),
        ("payload_offset", ct.c_uint64), ("capacity", ct.c_uint64),
    ]


class _SoftDesc(ct.Structure):
    _fields_ = [
        ("B", ct.c_int32), ("C", ct.c_int32), ("H", ct.c_int32), ("W", ct.c_int32),
        ("b", ct.c_int32 * 2), ("eps", ct.c_double * 2), ("R", ct.c_double), ("m", ct.c_double),
        ("pad_mode", ct.c_int32), ("noise_free", ct.c_int32), ("stream_id", ct.c_uint32),
        ("seed", ct.c_uint64), ("frame0", ct.c_uint64),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ct.CDLL(path)
        P = ct.c_void_p
        L.ora_philox4x32_10.argtypes = [P, P, P]
        L.ora_philox4x64_10.argtypes = [P, P, P]
        L.ora_laplace_from_word.argtypes = [ct.c_uint32, ct.c_double]
        L.ora_laplace_from_word.restype = ct.c_double
        L.ora_geometry.argtypes = [ct.POINTER(_Desc), ct.POINTER(_Geom)]
        L.ora_reflect.argtypes = [ct.c_int64, ct.c_int64, ct.c_int]
        L.ora_reflect.restype = ct.c_int64
        L.ora_classify.argtypes = [ct.POINTER(_Desc), P, P, ct.c_int64, P]
        L.ora_release.argtypes = [ct.POINTER(_Desc), P, P, ct.c_int64, P, ct.c_uint64, P, P, P]
        L.ora_record_info.argtypes = [P, ct.c_uint64, P]
        L.ora_reconstruct.argtypes = [P, ct.c_uint64, ct.c_int, P, ct.c_int64]
        L.ora_soft_forward.argtypes = [ct.POINTER(_SoftDesc), P, P, P, P]
        L.ora_soft_backward.argtypes = [ct.POINTER(_SoftDesc), P, P, P, P, P]
        L.ora_header_size.restype = ct.c_uint64
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise OraError("%s failed with oracle code %d" % (what, rc))


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().ora_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().ora_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def laplace_from_word(x, sigma):
    return lib().ora_laplace_from_word(int(x) & 0xFFFFFFFF, float(sigma))


def reflect(p, n, pad_mode=0):
    return lib().ora_reflect(int(p), int(n), int(pad_mode))


def make_desc(M, N, C=3, grids=(8,), eps=(1.0,), R=255.0, m=16.0, pad_mode=0, source=SRC_TILE_LABELS,
              matte_thr=0.5, dtype=DT_F32, noise_free=False, stream_id=0, seed=0, frame_idx=0, pitch=None):
    d = _Desc()
    d.M, d.N, d.C = int(M), int(N), int(C)
    d.K = len(grids)
    if len(eps) != len(grids) or not (1 <= d.K <= MAXK):
        raise ValueError("grids and eps must have the same length in 1..8")
    d.pitch = int(pitch if pitch is not None else N * C)
    for i, (b, e) in enumerate(zip(grids, eps)):
        d.b[i] = int(b)
        d.eps[i] = float(e)
    d.R, d.m = float(R), float(m)
    d.pad_mode, d.source, d.matte_thr = int(pad_mode), int(source), float(matte_thr)
    d.dtype, d.noise_free, d.stream_id = int(dtype), int(bool(noise_free)), int(stream_id)
    d.seed, d.frame_idx = int(seed) & (2**64 - 1), int(frame_idx) & (2**64 - 1)
    return d


def geometry(**kw):
    d = make_desc(**kw)
    g = _Geom()
    _check(lib().ora_geometry(ct.byref(d), ct.byref(g)), "geometry")
    K = d.K
    return dict(T=g.T, GR=g.GR, GC=g.GC, PR=g.PR, PC=g.PC, cells_side=list(g.cells_side[:K]),
                sigma=list(g.sigma[:K]), header_bytes=g.header_bytes, rowidx_bytes=g.rowidx_bytes,
                map_offset=g.map_offset, payload_offset=g.payload_offset, capacity=g.capacity)


def geometry_rc(**kw):
    """Return code of the geometry check (0 or a negative oracle code)."""
    d = make_desc(**kw)
    g = _Geom()
    return lib().ora_geometry(ct.byref(d), ct.byref(g))


def _frame_arg(img, kw):
    img = np.ascontiguousarray(img, dtype=np.uint8)
    if img.ndim == 2:
        img = img[:, :, None]
    M, N, C = img.shape
    kw = dict(kw)
    kw.setdefault("M", M)
    kw.setdefault("N", N)
    kw.setdefault("C", C)
    return img, kw


def _src_arg(src, source):
    if src is None:
        return None, 0
    if source == SRC_MATTE:
        a = np.ascontiguousarray(src, dtype=np.float32)
    else:
        a = np.ascontiguousarray(src, dtype=np.uint8)
    pitch = a.strides[0] if a.ndim >= 2 else 0
    return a, pitch


def classify(img, src=None, **kw):
    img, kw = _frame_arg(img, kw)
    d = make_desc(**kw)
    g = geometry(**kw)
    s, sp = _src_arg(src, d.source)
    out = np.zeros(g["GR"] * g["GC"], dtype=np.uint8)
    _check(lib().ora_classify(ct.byref(d), _ptr(img), _ptr(s), sp, _ptr(out)), "classify")
    return out.reshape(g["GR"], g["GC"])


def release(img, src=None, **kw):
    """Returns (record bytes as uint8 array of length total_bytes, means f64, sums i64, eta f64),
    the last three in record order."""
    img, kw = _frame_arg(img, kw)
    d = make_desc(**kw)
    g = geometry(**kw)
    s, sp = _src_arg(src, d.source)
    cap = int(g["capacity"])
    rec = np.zeros(cap, dtype=np.uint8)
    nmax = g["GR"] * g["GC"] * max(c * c for c in g["cells_side"]) * d.C
    means = np.zeros(nmax, dtype=np.float64)
    sums = np.zeros(nmax, dtype=np.int64)
    etas = np.zeros(nmax, dtype=np.float64)
    _check(lib().ora_release(ct.byref(d), _ptr(img), _ptr(s), sp, _ptr(rec), cap, _ptr(means), _ptr(sums),
                             _ptr(etas)), "release")
    info = record_info(rec)
    n = info["n_values"]
    return rec[: info["total_bytes"]].copy(), means[:n].copy(), sums[:n].copy(), etas[:n].copy()


def record_info(rec):
    """Parse the header of a record (numpy u8 array or bytes) with plain little-endian reads."""
    rec = np.frombuffer(bytes(rec[:512]), dtype=np.uint8) if not isinstance(rec, np.ndarray) else rec
    h = rec[:512].tobytes()
    if h[:4] != b"DPPX":
        raise OraError("bad record magic")
    u32 = lambda o: int.from_bytes(h[o:o + 4], "little")
    u64 = lambda o: int.from_bytes(h[o:o + 8], "little")
    f64 = lambda o: float(np.frombuffer(h[o:o + 8], dtype="<f8")[0])
    K = u32(32)
    info = dict(version=u32(4), header_bytes=u32(8), flags=u32(12), M=u32(16), N=u32(20), C=u32(24),
                T=u32(28), K=K, GR=u32(36), GC=u32(40), pad_mode=u32(44), dtype=u32(48), source=u32(52),
                stream_id=u32(56), seed=u64(64), frame_idx=u64(72), R=f64(80), m=f64(88),
                total_bytes=u64(96), map_offset=u64(104), row_offset=u64(368), payload_offset=u64(376),
                b=[u32(112 + 4 * r) for r in range(K)], eps=[f64(144 + 8 * r) for r in range(K)],
                sigma=[f64(208 + 8 * r) for r in range(K)], count=[u32(272 + 4 * r) for r in range(K)],
                region_offset=[u64(304 + 8 * r) for r in range(K)])
    cs = [info["T"] // b for b in info["b"]]
    info["cells_side"] = cs
    info["n_values"] = sum(info["count"][r] * cs[r] * cs[r] * info["C"] for r in range(K))
    return info


def record_payload(rec, dtype=None):
    """Payload values of a record in record order, as float64 (f32/u8 records) or int64 (sum records)."""
    info = record_info(rec)
    rec = np.asarray(rec, dtype=np.uint8)
    dt = info["dtype"] if dtype is None else dtype
    parts = []
    for r in range(info["K"]):
        n = info["count"][r] * info["cells_side"][r] ** 2 * info["C"]
        off = info["region_offset"][r]
        if dt == DT_F32:
            parts.append(rec[off:off + 4 * n].view("<f4").astype(np.float64))
        elif dt == DT_U8:
            parts.append(rec[off:off + n].astype(np.float64))
        else:
            parts.append(rec[off:off + 4 * n].view("<u4").astype(np.int64))
    return np.concatenate(parts) if parts else np.zeros(0)


def record_map(rec):
    info = record_info(rec)
    rec = np.asarray(rec, dtype=np.uint8)
    n = info["GR"] * info["GC"]
    return rec[info["map_offset"]:info["map_offset"] + n].reshape(info["GR"], info["GC"]).copy()


def reconstruct(rec, out_type=0):
    """out_type 0: u8 [M, N, C]; 1: f32; 2: f64."""
    rec = np.ascontiguousarray(rec, dtype=np.uint8)
    info = record_info(rec)
    M, N, C = info["M"], info["N"], info["C"]
    dt = {0: np.uint8, 1: np.float32, 2: np.float64}[out_type]
    out = np.zeros((M, N, C), dtype=dt)
    _check(lib().ora_reconstruct(_ptr(rec), rec.size, out_type, _ptr(out), out.strides[0]), "reconstruct")
    return out


def _soft_desc(B, C, H, W, grids=(8, 16), eps=(0.5, 1.0), R=1.0, m=16.0, pad_mode=0, noise_free=False,
               stream_id=0, seed=0, frame0=0):
    s = _SoftDesc()
    s.B, s.C, s.H, s.W = int(B), int(C), int(H), int(W)
    s.b[0], s.b[1] = int(grids[0]), int(grids[1])
    s.eps[0], s.eps[1] = float(eps[0]), float(eps[1])
    s.R, s.m, s.pad_mode, s.noise_free = float(R), float(m), int(pad_mode), int(bool(noise_free))
    s.stream_id, s.seed, s.frame0 = int(stream_id), int(seed) & (2**64 - 1), int(frame0) & (2**64 - 1)
    return s


def soft_forward(x, w, **kw):
    """x [B, C, H, W], w [B, 1, H, W] -> (y [B, C, H, W], p [B, 2, C, H, W]) in float64."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    B, C, H, W = x.shape
    s = _soft_desc(B, C, H, W, **kw)
    y = np.zeros((B, C, H, W), dtype=np.float64)
    p = np.zeros((B, 2, C, H, W), dtype=np.float64)
    _check(lib().ora_soft_forward(ct.byref(s), _ptr(x), _ptr(w), _ptr(y), _ptr(p)), "soft_forward")
    return y, p


def soft_backward(x, w, g, **kw):
    """Gradients of L = sum(g * y) with respect to x and w (noise constant), float64."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    B, C, H, W = x.shape
    s = _soft_desc(B, C, H, W, **kw)
    dx = np.zeros_like(x)
    dw = np.zeros((B, 1, H, W), dtype=np.float64)
    _check(lib().ora_soft_backward(ct.byref(s), _ptr(x), _ptr(w), _ptr(g), _ptr(dx), _ptr(dw)), "soft_backward")
    return dx, dw


__all__ = [
    "PAD_REFLECT", "PAD_SYMMETRIC", "PAD_NONE",
    "OraError", "SRC_TILE_LABELS", "SRC_MASK", "SRC_MATTE", "SRC_VARIANCE", "DT_F32", "DT_U8", "DT_SUM",
    "philox4x32_10", "philox4x64_10", "laplace_from_word", "reflect", "geometry", "geometry_rc", "classify",
    "release", "record_info", "record_payload", "record_map", "reconstruct", "soft_forward", "soft_backward",
]
