"""Python binding of the serving loop (dp_pix_server_*) and of the keyed release: frames of many cameras
submitted from host memory, continuously batched onto the GPU by the library's worker thread.  Argument
marshalling only."""
from __future__ import annotations

import ctypes as ct
from typing import Optional, Sequence

import torch

from . import _lib as L

__all__ = ["Server", "dp_pix_release_keyed", "dp_pix_release_reconstruct_keyed", "key_table", "dp_pix_keys_advance"]


def _desc(C, grids, eps, R, m, pad_mode, source, dtype, noise_free, seed):
    d = L.Desc()
    d.M, d.N, d.C, d.K = 1, 1, int(C), len(grids)
    d.row_pitch = int(C)
    for i, (b, e) in enumerate(zip(grids, eps)):
        d.grid[i] = int(b)
        d.eps[i] = float(e)
    d.value_range, d.m, d.pad_mode, d.region_source = float(R), float(m), int(pad_mode), int(source)
    d.record_dtype, d.noise_free, d.seed = int(dtype), int(bool(noise_free)), int(seed) & (2**64 - 1)
    return d


def dp_pix_keys_advance(keys: torch.Tensor, delta: int, stream=None):
    """keys: a device key table (key_table); adds delta to every frame index on the device."""
    n = keys.numel() // ct.sizeof(L.FrameKey)
    s = ct.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    L.check(L.lib().dp_pix_keys_advance(ct.c_void_p(keys.data_ptr()), n, int(delta) & (2**64 - 1), s),
            "dp_pix_keys_advance")


def key_table(keys, device="cuda") -> torch.Tensor:
    """Device key table (u8 tensor of dp_pix_frame_key entries) for F pairs (stream_id, frame_idx)."""
    return _key_table(keys, device)


def _key_table(keys, device):
    n = len(keys)
    kt = (L.FrameKey * n)()
    for i, (sid, fidx) in enumerate(keys):
        kt[i].stream_id, kt[i].frame_idx, kt[i].reserved = int(sid), int(fidx) & (2**64 - 1), 0
    return torch.frombuffer(bytearray(bytes(kt)), dtype=torch.uint8).to(device)


def dp_pix_release_keyed(plan, frames: torch.Tensor, keys: Sequence[Sequence[int]], records=None, ws=None,
                         stream=None) -> torch.Tensor:
    """frames [F, M, N, C] u8 on the GPU; keys: F pairs (stream_id, frame_idx).  Returns records [F, stride]."""
    n = frames.shape[0]
    kd = _key_table(keys, frames.device)
    if records is None:
        records = plan.alloc_records(n, device=frames.device)
    if ws is None:
        ws = plan.alloc_workspace(n, device=frames.device)
    s = ct.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    L.check(L.lib().dp_pix_release_keyed(plan.handle, ct.c_void_p(frames.data_ptr()),
                                         frames.stride(0) * frames.element_size(), None, 0, 0, n,
                                         ct.c_void_p(kd.data_ptr()), ct.c_void_p(records.data_ptr()),
                                         records.stride(0), ct.c_void_p(ws.data_ptr()), ws.numel(), s),
            "dp_pix_release_keyed")
    torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()  # kd is freed on return
    return records


def dp_pix_release_reconstruct_keyed(plan, frames: torch.Tensor, keys, out_type=L.OUT_U8,
                                     records=None, out=None, ws=None, stream=None):
    """dp_pix_release_reconstruct with one (stream_id, frame_idx) key per frame.  frames [F, M, N, C] u8 on the
    GPU; keys: F pairs (stream_id, frame_idx), or a device key table (key_table, used in place, so that a
    captured graph sees dp_pix_keys_advance's updates); out: [F, M, N, C] u8 / f32 (any row pitch).
    Returns (records [F, stride], images)."""
    n = frames.shape[0]
    spec = plan.spec
    on_device = isinstance(keys, torch.Tensor)
    kd = keys if on_device else _key_table(keys, frames.device)
    if records is None:
        records = plan.alloc_records(n, device=frames.device)
    if ws is None:
        ws = plan.alloc_workspace(n, device=frames.device)
    if out is None:
        dt = torch.uint8 if out_type == L.OUT_U8 else torch.float32
        out = torch.empty((n, spec.M, spec.N, spec.C), dtype=dt, device=frames.device)
    es = out.element_size()
    s = ct.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    L.check(L.lib().dp_pix_release_reconstruct_keyed(
        plan.handle, ct.c_void_p(frames.data_ptr()), frames.stride(0) * frames.element_size(), None, 0, 0, n,
        ct.c_void_p(kd.data_ptr()), ct.c_void_p(records.data_ptr()), records.stride(0), ct.c_void_p(out.data_ptr()),
        out.stride(0) * es, out.stride(1) * es, int(out_type), ct.c_void_p(ws.data_ptr()), ws.numel(), s),
        "dp_pix_release_reconstruct_keyed")
    if not on_device:  # the temporary key table is freed on return
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    return records, out


class Server:
    """dp_pix_server_create for cameras of sizes (M[c], N[c]) (VARIANCE classes), with an arena of
    `arena_bytes` of device memory allocated here by torch and owned by this object.  first_frame: each
    camera's first frame index (counters() of an earlier server with the same seed), default 0."""

    def __init__(self, sizes: Sequence[Sequence[int]], arena_bytes: int, C=3, grids=(32, 16, 8, 4),
                 eps=(2.0, 1.0, 0.5, 0.25), R=255.0, m=16.0, pad_mode=L.PAD_REFLECT, dtype=L.REC_F32,
                 noise_free=False, seed=0, n_streams=3, first_frame: Optional[Sequence[int]] = None, device="cuda"):
        self.desc = _desc(C, grids, eps, R, m, pad_mode, L.SRC_VARIANCE, dtype, noise_free, seed)
        self.sizes = [(int(a), int(b)) for a, b in sizes]
        self.C = int(C)
        n = len(self.sizes)
        self.record_bytes, self.slot_bytes, self.recon_bytes = [], [], []
        for (M, N) in self.sizes:
            sb, rb, ob = ct.c_uint64(0), ct.c_uint64(0), ct.c_uint64(0)
            L.check(L.lib().dp_pix_server_sizes(ct.byref(self.desc), M, N, ct.byref(sb), ct.byref(rb), ct.byref(ob)),
                    "dp_pix_server_sizes")
            self.slot_bytes.append(int(sb.value))
            self.record_bytes.append(int(rb.value))
            self.recon_bytes.append(int(ob.value))
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=device)
        Ms = (ct.c_int32 * n)(*[a for a, _ in self.sizes])
        Ns = (ct.c_int32 * n)(*[b for _, b in self.sizes])
        ff = None
        if first_frame is not None:
            if len(first_frame) != n:
                raise ValueError("first_frame needs one index per camera")
            ff = (ct.c_uint64 * n)(*[int(v) & (2**64 - 1) for v in first_frame])
        h = ct.c_void_p()
        L.check(L.lib().dp_pix_server_create(ct.byref(self.desc), Ms, Ns, n, ff, int(n_streams),
                                             ct.c_void_p(self.arena.data_ptr()), int(arena_bytes), ct.byref(h)),
                "dp_pix_server_create")
        self._h = h
        self._keep = {}

    def record_buffer(self, camera: int) -> torch.Tensor:
        return torch.empty(self.record_bytes[camera], dtype=torch.uint8).pin_memory()

    def image_buffer(self, camera: int) -> torch.Tensor:
        M, N = self.sizes[camera]
        return torch.empty((M, N, self.C), dtype=torch.uint8).pin_memory()

    def submit(self, camera: int, frame: torch.Tensor, record: torch.Tensor, out: Optional[torch.Tensor] = None) -> int:
        """frame: host u8 [M, N, C] contiguous (pinned for asynchronous copies); record: host u8 buffer of
        record_bytes[camera] bytes; out: optional host u8 [M, N, C] for the pixelized image.  All are kept
        alive here until wait() returns the ticket."""
        if frame.device.type != "cpu" or record.device.type != "cpu" or not frame.is_contiguous():
            raise ValueError("frame and record must be contiguous host tensors")
        if out is not None:
            M, N = self.sizes[camera]
            if out.device.type != "cpu" or not out.is_contiguous() or out.dtype != torch.uint8 or \
                    out.numel() != M * N * self.C:
                raise ValueError("out must be a contiguous host u8 tensor of M * N * C elements")
        t = ct.c_uint64(0)
        L.check(L.lib().dp_pix_server_submit(self._h, int(camera), ct.c_void_p(frame.data_ptr()),
                                             ct.c_void_p(record.data_ptr()), record.numel(),
                                             ct.c_void_p(out.data_ptr()) if out is not None else None, ct.byref(t)),
                "dp_pix_server_submit")
        self._keep[int(t.value)] = (frame, record, out)
        return int(t.value)

    def counters(self) -> list:
        """Next frame index of every camera, once every submitted request has been released."""
        n = len(self.sizes)
        v = (ct.c_uint64 * n)()
        L.check(L.lib().dp_pix_server_counters(self._h, v, n), "dp_pix_server_counters")
        return [int(x) for x in v]

    def wait(self, ticket: int, timeout_ms: int = -1) -> Optional[dict]:
        r = L.ServerResult()
        rc = L.lib().dp_pix_server_wait(self._h, int(ticket), int(timeout_ms), ct.byref(r))
        if rc == L.E_TIMEOUT:
            return None
        L.check(rc, "dp_pix_server_wait")
        frame, record, out = self._keep.pop(int(ticket))
        return dict(ticket=int(r.ticket), frame_idx=int(r.frame_idx), record_bytes=int(r.record_bytes),
                    camera=int(r.camera), status=int(r.status), queue_us=float(r.queue_us),
                    latency_us=float(r.latency_us), record=record, image=out)

    def stats(self) -> dict:
        st = L.ServerStats()
        L.check(L.lib().dp_pix_server_stats_get(self._h, ct.byref(st)), "dp_pix_server_stats_get")
        return {k: getattr(st, k) for k, _ in L.ServerStats._fields_}

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            L.lib().dp_pix_server_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
