"""Python binding of the ragged-batch calls (dp_pix_batch_*): many images of different sizes released, and
optionally reconstructed, with one set of region parameters; each phase is one persistent launch over all
images, replayed from a CUDA graph.  Argument marshalling only."""
from __future__ import annotations

import ctypes as ct
from typing import List, Optional, Sequence

import torch

from . import _lib as L

__all__ = ["BatchPlan"]


def _stream(stream):
    return ct.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)


class BatchPlan:
    """dp_pix_batch_plan for images of sizes (M[i], N[i]); region parameters as for Plan."""

    def __init__(self, sizes: Sequence[Sequence[int]], C=3, grids=(6, 20), eps=(0.5, 1.5), R=255.0, m=32.0,
                 pad_mode=L.PAD_REFLECT, source=L.SRC_MATTE_F32, matte_thr=0.5, dtype=L.REC_F32, noise_free=False,
                 seed=0):
        d = L.Desc()
        d.M, d.N, d.C, d.K = 1, 1, int(C), len(grids)
        d.row_pitch = int(C)
        for i, (b, e) in enumerate(zip(grids, eps)):
            d.grid[i] = int(b)
            d.eps[i] = float(e)
        d.value_range, d.m = float(R), float(m)
        d.pad_mode, d.region_source, d.matte_threshold = int(pad_mode), int(source), float(matte_thr)
        d.record_dtype, d.noise_free, d.seed = int(dtype), int(bool(noise_free)), int(seed) & (2**64 - 1)
        self.desc, self.C, self.source = d, int(C), int(source)
        self.sizes = [(int(a), int(b)) for a, b in sizes]
        n = len(self.sizes)
        Ms = (ct.c_int32 * n)(*[a for a, _ in self.sizes])
        Ns = (ct.c_int32 * n)(*[b for _, b in self.sizes])
        h = ct.c_void_p()
        L.check(L.lib().dp_pix_batch_plan(ct.byref(d), Ms, Ns, n, ct.byref(h)), "dp_pix_batch_plan")
        self._h = h
        rb = (ct.c_uint64 * n)()
        wb = ct.c_uint64(0)
        L.check(L.lib().dp_pix_batch_sizes(h, rb, ct.byref(wb)), "dp_pix_batch_sizes")
        self.record_bytes: List[int] = [int(v) for v in rb]
        self.ws_bytes = int(wb.value)
        self._imgs = None
        self._keep = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                L.lib().dp_pix_batch_destroy(h)
            except Exception:
                pass
            self._h = None

    def alloc_records(self, device="cuda") -> List[torch.Tensor]:
        return [torch.empty(nb, dtype=torch.uint8, device=device) for nb in self.record_bytes]

    def alloc_workspace(self, device="cuda") -> torch.Tensor:
        return torch.empty(max(1, self.ws_bytes), dtype=torch.uint8, device=device)

    def bind(self, frames: Sequence[torch.Tensor], region_src: Sequence[Optional[torch.Tensor]],
             records: Sequence[torch.Tensor], ws: torch.Tensor, outs: Optional[Sequence[Optional[torch.Tensor]]] = None,
             out_type: int = L.OUT_U8, stream_ids: Optional[Sequence[int]] = None,
             frame_idx: Optional[Sequence[int]] = None, stream=None):
        """frames[i]: u8 [M, N, C] (rows may be strided); region_src[i]: labels / mask / matte as for Plan.release;
        records[i]: record_bytes[i] bytes; outs[i]: [M, N, C] u8 / f32 or None."""
        n = len(self.sizes)
        arr = (L.BatchImage * n)()
        for i in range(n):
            f = frames[i]
            im = arr[i]
            im.frame = f.data_ptr()
            im.row_pitch = f.stride(0) * f.element_size()
            src = region_src[i] if region_src is not None else None
            if src is not None:
                im.region_src = src.data_ptr()
                im.src_pitch = src.stride(0) * src.element_size() if src.dim() >= 2 else 0
            im.record = records[i].data_ptr()
            o = outs[i] if outs is not None else None
            if o is not None:
                im.out = o.data_ptr()
                im.out_pitch = o.stride(0) * o.element_size()
            im.stream_id = int(stream_ids[i]) if stream_ids is not None else 0
            im.frame_idx = int(frame_idx[i]) & (2**64 - 1) if frame_idx is not None else i
        L.check(L.lib().dp_pix_batch_bind(self._h, arr, int(out_type), ct.c_void_p(ws.data_ptr()),
                                          ws.numel() * ws.element_size(), _stream(stream)), "dp_pix_batch_bind")
        self._imgs = arr
        self._out_type = int(out_type)
        self._keep = (list(frames), list(region_src) if region_src is not None else None, list(records), ws,
                      list(outs) if outs is not None else None)
        return self

    def run(self, use_graph: bool = True, stream=None):
        L.check(L.lib().dp_pix_batch_run(self._h, int(bool(use_graph)), _stream(stream)), "dp_pix_batch_run")

    def autotune(self, reps: int = 3, stream=None) -> int:
        if self._imgs is None:
            raise RuntimeError("bind the batch first")
        L.check(L.lib().dp_pix_batch_autotune(self._h, self._imgs, int(reps), _stream(stream)), "dp_pix_batch_autotune")
        return self.seg_tiles()

    def seg_tiles(self) -> int:
        return self.tuning()[0]

    def tuning(self):
        """(segment tiles, release path DP_PIX_BATCH_PATH_*) in use."""
        v, p = ct.c_int(0), ct.c_int(0)
        L.check(L.lib().dp_pix_batch_tuning(self._h, ct.byref(v), ct.byref(p)), "dp_pix_batch_tuning")
        return int(v.value), int(p.value)

    def set_path(self, path: int, seg_tiles: int = 0):
        """dp_pix_batch_set_path: fix the release path (-1: default) and width (0: the path's); rebinds the
        images bound last."""
        L.check(L.lib().dp_pix_batch_set_path(self._h, int(path), int(seg_tiles)), "dp_pix_batch_set_path")
        if self._imgs is not None:
            frames, srcs, recs, ws, outs = self._keep
            L.check(L.lib().dp_pix_batch_bind(self._h, self._imgs, self._out_type, ct.c_void_p(ws.data_ptr()),
                                              ws.numel() * ws.element_size(), _stream(None)), "dp_pix_batch_bind")
        return self
