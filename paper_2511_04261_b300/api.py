"""Python binding of libdppix: the C-ABI calls with the same names, with torch supplying device memory
and streams.  Every step of the release runs in the library's CUDA kernels; this module only marshals
arguments and allocates caller-owned buffers."""
from __future__ import annotations

import ctypes as ct
from dataclasses import dataclass, field
from typing import Optional, Sequence

import torch

from . import _lib as L

__all__ = ["Plan", "dp_pix_plan", "dp_pix_release", "dp_pix_release_reconstruct", "dp_pix_store", "dp_pix_store_batch", "dp_pix_reconstruct", "dp_pix_debug_noise",
           "dp_pix_status", "prof_enable", "prof_read", "prof_reset", "record_header", "DppixError"]

DppixError = L.DppixError


def _stream_handle(stream: Optional[torch.cuda.Stream]) -> ct.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ct.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[ct.c_void_p]:
    return None if t is None else ct.c_void_p(t.data_ptr())


@dataclass
class PlanSpec:
    M: int
    N: int
    C: int = 3
    grids: Sequence[int] = (8,)
    eps: Sequence[float] = (1.0,)
    R: float = 255.0
    m: float = 16.0
    pad_mode: int = L.PAD_REFLECT
    source: int = L.SRC_TILE_LABELS
    matte_thr: float = 0.5
    dtype: int = L.REC_F32
    noise_free: bool = False
    seed: int = 0
    pitch: Optional[int] = None


class Plan:
    """dp_pix_plan: an immutable, validated problem description with its sizes (host only)."""

    def __init__(self, M, N, C=3, grids=(8,), eps=(1.0,), R=255.0, m=16.0, pad_mode=L.PAD_REFLECT,
                 source=L.SRC_TILE_LABELS, matte_thr=0.5, dtype=L.REC_F32, noise_free=False, seed=0, pitch=None):
        self.spec = PlanSpec(M, N, C, tuple(grids), tuple(eps), R, m, pad_mode, source, matte_thr, dtype,
                             noise_free, seed, pitch)
        d = L.Desc()
        d.M, d.N, d.C, d.K = int(M), int(N), int(C), len(grids)
        if len(eps) != len(grids) or not (1 <= d.K <= L.MAXK):
            raise ValueError("grids and eps must have the same length in 1..8")
        d.row_pitch = int(pitch if pitch is not None else N * C)
        for i, (b, e) in enumerate(zip(grids, eps)):
            d.grid[i] = int(b)
            d.eps[i] = float(e)
        d.value_range, d.m = float(R), float(m)
        d.pad_mode, d.region_source, d.matte_threshold = int(pad_mode), int(source), float(matte_thr)
        d.record_dtype, d.noise_free, d.seed = int(dtype), int(bool(noise_free)), int(seed) & (2**64 - 1)
        self.desc = d
        h = ct.c_void_p()
        sz = L.Sizes()
        L.check(L.lib().dp_pix_plan(ct.byref(d), ct.byref(h), ct.byref(sz)), "dp_pix_plan")
        self._h = h
        self.sizes = sz
        self.K = d.K
        self.record_bytes = int(sz.record_bytes)
        self.ws_per_frame = int(sz.workspace_per_frame)
        self.T, self.GR, self.GC = int(sz.T), int(sz.GR), int(sz.GC)
        self.sigma = [float(sz.sigma[i]) for i in range(d.K)]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                L.lib().dp_pix_plan_destroy(h)
            except Exception:
                pass
            self._h = None

    @property
    def handle(self):
        return self._h

    def tune(self, knob: int, value: int) -> "Plan":
        """dp_pix_plan_tune: set a knob (the TUNE_* constants; the launch-shape knobs never change results)."""
        L.check(L.lib().dp_pix_plan_tune(self._h, int(knob), int(value)), "dp_pix_plan_tune")
        return self

    def tuning(self, knob: int) -> int:
        v = ct.c_int(0)
        L.check(L.lib().dp_pix_plan_tuning(self._h, int(knob), ct.byref(v)), "dp_pix_plan_tuning")
        return int(v.value)

    def record_stride(self) -> int:
        return (self.record_bytes + 255) // 256 * 256

    def alloc_records(self, n_frames: int, device="cuda") -> torch.Tensor:
        return torch.empty((n_frames, self.record_stride()), dtype=torch.uint8, device=device)

    def alloc_workspace(self, n_frames: int, device="cuda") -> torch.Tensor:
        return torch.empty((max(1, n_frames * self.ws_per_frame),), dtype=torch.uint8, device=device)

    def release(self, frames: torch.Tensor, region_src: Optional[torch.Tensor] = None, stream_id: int = 0,
                frame_idx0: int = 0, records: Optional[torch.Tensor] = None, ws: Optional[torch.Tensor] = None,
                stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
        """frames: u8 CUDA tensor [F, M, N, C] or [M, N, C] (rows may be padded via the plan's pitch when
        the tensor is [F, M, pitch] / [M, pitch]).  Returns the records tensor [F, record_stride]."""
        return dp_pix_release(self, frames, region_src, stream_id, frame_idx0, records, ws, stream)

    def release_reconstruct(self, frames: torch.Tensor, region_src: Optional[torch.Tensor] = None,
                            stream_id: int = 0, frame_idx0: int = 0, out_type: int = L.OUT_U8,
                            records: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
                            ws: Optional[torch.Tensor] = None, stream: Optional[torch.cuda.Stream] = None):
        """Release and reconstruct in one call; returns (records [F, stride], images [F, M, N, C])."""
        return dp_pix_release_reconstruct(self, frames, region_src, stream_id, frame_idx0, out_type, records, out,
                                          ws, stream)


def dp_pix_plan(**kw) -> Plan:
    return Plan(**kw)


def _release_args(plan: Plan, frames: torch.Tensor, region_src, records, ws):
    if frames.device.type != "cuda" or frames.dtype != torch.uint8:
        raise ValueError("frames must be a uint8 CUDA tensor")
    spec = plan.spec
    single = frames.dim() == (3 if spec.pitch is None else 2)
    fr = frames.unsqueeze(0) if single else frames
    n = fr.shape[0]
    frame_stride = fr.stride(0) * fr.element_size()
    src_pitch, src_frame_stride = 0, 0
    if region_src is not None:
        rs = region_src.unsqueeze(0) if single else region_src
        if rs.device.type != "cuda":
            raise ValueError("region source must be a CUDA tensor")
        src_frame_stride = rs.stride(0) * rs.element_size()
        src_pitch = rs.stride(1) * rs.element_size() if rs.dim() >= 3 else 0
        region_src = rs
    if records is None:
        records = plan.alloc_records(n, device=frames.device)
    if ws is None:
        ws = plan.alloc_workspace(n, device=frames.device)
    return single, fr, n, frame_stride, region_src, src_pitch, src_frame_stride, records, ws


def dp_pix_release(plan: Plan, frames: torch.Tensor, region_src: Optional[torch.Tensor] = None, stream_id: int = 0,
                   frame_idx0: int = 0, records: Optional[torch.Tensor] = None, ws: Optional[torch.Tensor] = None,
                   stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    _, fr, n, frame_stride, region_src, src_pitch, src_frame_stride, records, ws = _release_args(
        plan, frames, region_src, records, ws)
    rc = L.lib().dp_pix_release(plan.handle, _ptr(fr), frame_stride, _ptr(region_src), src_pitch, src_frame_stride,
                                n, int(stream_id), int(frame_idx0) & (2**64 - 1), _ptr(records),
                                records.stride(0) * records.element_size(), _ptr(ws), ws.numel() * ws.element_size(),
                                _stream_handle(stream))
    L.check(rc, "dp_pix_release")
    return records


def dp_pix_release_reconstruct(plan: Plan, frames: torch.Tensor, region_src: Optional[torch.Tensor] = None,
                               stream_id: int = 0, frame_idx0: int = 0, out_type: int = L.OUT_U8,
                               records: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
                               ws: Optional[torch.Tensor] = None, stream: Optional[torch.cuda.Stream] = None):
    """dp_pix_release then dp_pix_reconstruct in one call.  out: [F, M, N, C] (or [M, N, C]) u8 / f32 with
    rows of any pitch.  Returns (records, images)."""
    single, fr, n, frame_stride, region_src, src_pitch, src_frame_stride, records, ws = _release_args(
        plan, frames, region_src, records, ws)
    spec = plan.spec
    dt = torch.uint8 if out_type == L.OUT_U8 else torch.float32
    if out is None:
        out = torch.empty((n, spec.M, spec.N, spec.C), dtype=dt, device=frames.device)
    o = out.unsqueeze(0) if out.dim() == 3 else out
    es = o.element_size()
    rc = L.lib().dp_pix_release_reconstruct(
        plan.handle, _ptr(fr), frame_stride, _ptr(region_src), src_pitch, src_frame_stride, n, int(stream_id),
        int(frame_idx0) & (2**64 - 1), _ptr(records), records.stride(0) * records.element_size(), _ptr(o),
        o.stride(0) * es, o.stride(1) * es, int(out_type), _ptr(ws), ws.numel() * ws.element_size(),
        _stream_handle(stream))
    L.check(rc, "dp_pix_release_reconstruct")
    return records, (out[0] if single and out.dim() == 4 else out)


def dp_pix_store(record: torch.Tensor, stream: Optional[torch.cuda.Stream] = None) -> bytes:
    """Copy one device record's used bytes to host memory (synchronizes the stream)."""
    cap = record.numel()
    buf = ct.create_string_buffer(cap)
    written = ct.c_uint64(0)
    L.check(L.lib().dp_pix_store(_ptr(record), buf, cap, ct.byref(written), 1, _stream_handle(stream)), "dp_pix_store")
    return buf.raw[: written.value]


def dp_pix_store_batch(records: torch.Tensor, host_out: torch.Tensor, stream: Optional[torch.cuda.Stream] = None):
    """Copy the used bytes of every device record [F, stride] into host_out [F, dst_stride] (pinned for
    speed); returns the list of sizes.  Synchronizes the stream."""
    n = records.shape[0]
    written = (ct.c_uint64 * max(1, n))()
    L.check(L.lib().dp_pix_store_batch(_ptr(records), records.stride(0) * records.element_size(), n,
                                       ct.c_void_p(host_out.data_ptr()), host_out.stride(0) * host_out.element_size(),
                                       written, _stream_handle(stream)), "dp_pix_store_batch")
    return [int(written[i]) for i in range(n)]


def dp_pix_reconstruct(records: torch.Tensor, M: int, N: int, C: int, out_type: int = L.OUT_U8,
                       out: Optional[torch.Tensor] = None, stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """records: u8 CUDA tensor [F, stride] (or [stride]); returns [F, M, N, C] u8 / f32 (or [M, N, C])."""
    single = records.dim() == 1
    rec = records.unsqueeze(0) if single else records
    n = rec.shape[0]
    dt = torch.uint8 if out_type == L.OUT_U8 else torch.float32
    if out is None:
        out = torch.empty((n, M, N, C), dtype=dt, device=records.device)
    o = out.unsqueeze(0) if out.dim() == 3 else out
    es = o.element_size()
    L.check(L.lib().dp_pix_reconstruct(_ptr(rec), rec.stride(0) * rec.element_size(), n, _ptr(o), o.stride(0) * es,
                                       o.stride(1) * es, int(out_type), int(M), int(N), int(C), _stream_handle(stream)),
            "dp_pix_reconstruct")
    return out[0] if single and out.dim() == 4 else out


def dp_pix_debug_noise(seed: int, ctr: torch.Tensor, sigma: float, stream=None):
    """ctr: u32-valued CUDA tensor [n, 4] (int32 or int64 holding u32 values).  Returns (words int64 [n, 4],
    eta f32 [n, 4])."""
    c = ctr.to(torch.int64).to(torch.int32).contiguous() if ctr.dtype != torch.int32 else ctr.contiguous()
    n = c.shape[0]
    words = torch.empty((n, 4), dtype=torch.int32, device=c.device)
    eta = torch.empty((n, 4), dtype=torch.float32, device=c.device)
    L.check(L.lib().dp_pix_debug_noise(int(seed) & (2**64 - 1), _ptr(c), n, _ptr(words), _ptr(eta), float(sigma),
                                       _stream_handle(stream)), "dp_pix_debug_noise")
    return words.to(torch.int64) & 0xFFFFFFFF, eta


def dp_pix_status(stream=None) -> int:
    detail = ct.c_uint32(0)
    rc = L.lib().dp_pix_status(_stream_handle(stream), ct.byref(detail))
    return L.check(rc, "dp_pix_status (detail 0x%x)" % detail.value)


def prof_enable(timing: bool = True):
    L.lib().dp_pix_prof_enable(int(bool(timing)))


def prof_reset():
    L.lib().dp_pix_prof_reset()


def prof_read() -> dict:
    arr = (L.ProfEntry * 64)()
    n = L.check(L.lib().dp_pix_prof_read(arr, 64), "dp_pix_prof_read")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(min(n, 64))}


def record_header(rec_bytes) -> dict:
    """Parse a record header from host bytes (little-endian fields of dp_pix_record_header)."""
    import struct
    h = bytes(rec_bytes[:512])
    if h[:4] != b"DPPX":
        raise ValueError("not a record")
    (ver, hb, flags, M, N, C, T, K, GR, GC, pad, dtype, src, sid, _r0) = struct.unpack_from("<15I", h, 4)
    seed, frame = struct.unpack_from("<QQ", h, 64)
    R, m = struct.unpack_from("<dd", h, 80)
    total, map_off = struct.unpack_from("<QQ", h, 96)
    grid = list(struct.unpack_from("<8I", h, 112))[:K]
    eps = list(struct.unpack_from("<8d", h, 144))[:K]
    sigma = list(struct.unpack_from("<8d", h, 208))[:K]
    count = list(struct.unpack_from("<8I", h, 272))[:K]
    roff = list(struct.unpack_from("<8Q", h, 304))[:K]
    row_off, pay_off = struct.unpack_from("<QQ", h, 368)
    return dict(version=ver, header_bytes=hb, flags=flags, M=M, N=N, C=C, T=T, K=K, GR=GR, GC=GC, pad_mode=pad,
                dtype=dtype, source=src, stream_id=sid, seed=seed, frame_idx=frame, R=R, m=m, total_bytes=total,
                map_offset=map_off, grid=grid, eps=eps, sigma=sigma, count=count, region_offset=roff,
                rowidx_offset=row_off, payload_offset=pay_off)
