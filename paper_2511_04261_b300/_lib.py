"""ctypes declarations of libdppix (include/dppix.h).  Argument marshalling only.

The shared library is built in-tree (paper_2511_04261_b300/libdppix.so).  There is no fallback: if the
library is missing or fails to load, importing the binding raises.
"""
import ctypes as ct
import os

MAXK = 8
HERE = os.path.dirname(os.path.abspath(__file__))
# DPPIX_CHECKED=1 loads the bounds-checked build (every checked device access tested against its buffer)
LIB_PATH = os.path.join(HERE, "libdppix_checked.so" if os.environ.get("DPPIX_CHECKED") == "1" else "libdppix.so")

OK = 0
E_INVALID_ARG, E_UNSUPPORTED, E_PAD_TOO_LARGE, E_BUFFER_TOO_SMALL = -1, -2, -3, -4
E_BAD_RECORD, E_CUDA, E_TIMEOUT, E_DEVICE = -5, -6, -7, -8
ERROR_NAMES = {
    -1: "DP_PIX_E_INVALID_ARG", -2: "DP_PIX_E_UNSUPPORTED", -3: "DP_PIX_E_PAD_TOO_LARGE",
    -4: "DP_PIX_E_BUFFER_TOO_SMALL", -5: "DP_PIX_E_BAD_RECORD", -6: "DP_PIX_E_CUDA", -7: "DP_PIX_E_TIMEOUT",
    -8: "DP_PIX_E_DEVICE",
}
PAD_REFLECT, PAD_SYMMETRIC, PAD_NONE = 0, 1, 2
SRC_TILE_LABELS, SRC_MASK_U8, SRC_MATTE_F32, SRC_VARIANCE = 0, 1, 2, 3
REC_F32, REC_U8, REC_SUM_U32 = 0, 1, 2
OUT_U8, OUT_F32 = 0, 1
TUNE_FUSED_PX, TUNE_FUSED_THREADS, TUNE_SPLIT, TUNE_WAIT_TRIES, TUNE_TEST_SHORT_TX, TUNE_FUSED_CAP = 1, 2, 4, 8, 16, 32
TUNE_TEST_SHRINK = 64
BATCH_PATH_STAGED, BATCH_PATH_STREAM, BATCH_PATH_STREAM_FUSED, BATCH_PATH_TILES = 0, 1, 2, 3


class SoftDesc(ct.Structure):
    _fields_ = [
        ("B", ct.c_int32), ("C", ct.c_int32), ("H", ct.c_int32), ("W", ct.c_int32),
        ("grid", ct.c_int32 * 2), ("eps", ct.c_double * 2), ("value_range", ct.c_double), ("m", ct.c_double),
        ("pad_mode", ct.c_int32), ("noise_free", ct.c_int32), ("stream_id", ct.c_uint32),
        ("seed", ct.c_uint64), ("frame0", ct.c_uint64),
    ]


class BatchImage(ct.Structure):
    _fields_ = [
        ("frame", ct.c_void_p), ("row_pitch", ct.c_int64), ("region_src", ct.c_void_p), ("src_pitch", ct.c_int64),
        ("record", ct.c_void_p), ("out", ct.c_void_p), ("out_pitch", ct.c_int64), ("stream_id", ct.c_uint32),
        ("frame_idx", ct.c_uint64),
    ]


class FrameKey(ct.Structure):
    _fields_ = [("frame_idx", ct.c_uint64), ("stream_id", ct.c_uint32), ("reserved", ct.c_uint32)]


class ServerResult(ct.Structure):
    _fields_ = [("ticket", ct.c_uint64), ("frame_idx", ct.c_uint64), ("record_bytes", ct.c_uint64),
                ("camera", ct.c_uint32), ("status", ct.c_int32), ("queue_us", ct.c_double),
                ("latency_us", ct.c_double)]


class ServerStats(ct.Structure):
    _fields_ = [("submitted", ct.c_uint64), ("completed", ct.c_uint64), ("batches", ct.c_uint64),
                ("launches", ct.c_uint64), ("frames_in_flight_max", ct.c_uint64), ("mean_batch_frames", ct.c_double),
                ("arena_bytes_in_use_max", ct.c_uint64), ("arena_heap_bytes", ct.c_uint64)]


class Desc(ct.Structure):
    _fields_ = [
        ("M", ct.c_int32), ("N", ct.c_int32), ("C", ct.c_int32), ("K", ct.c_int32),
        ("row_pitch", ct.c_int64),
        ("grid", ct.c_int32 * MAXK), ("eps", ct.c_double * MAXK),
        ("value_range", ct.c_double), ("m", ct.c_double),
        ("pad_mode", ct.c_int32), ("region_source", ct.c_int32), ("matte_threshold", ct.c_float),
        ("record_dtype", ct.c_int32), ("noise_free", ct.c_int32), ("reserved0", ct.c_int32),
        ("seed", ct.c_uint64),
    ]


class Sizes(ct.Structure):
    _fields_ = [
        ("record_bytes", ct.c_uint64), ("workspace_per_frame", ct.c_uint64), ("workspace_fixed", ct.c_uint64),
        ("T", ct.c_uint32), ("GR", ct.c_uint32), ("GC", ct.c_uint32), ("PR", ct.c_uint32), ("PC", ct.c_uint32),
        ("num_tiles", ct.c_uint32), ("max_values", ct.c_uint64), ("sigma", ct.c_double * MAXK),
    ]


class Utility(ct.Structure):
    _fields_ = [("sse", ct.c_uint64), ("windows", ct.c_uint64), ("ssim_sum", ct.c_double), ("mse", ct.c_double),
                ("ssim", ct.c_double)]


class ProfEntry(ct.Structure):
    _fields_ = [("name", ct.c_char * 48), ("launches", ct.c_uint64), ("total_ms", ct.c_double)]


class DppixError(RuntimeError):
    def __init__(self, code, what, msg):
        self.code = code
        super().__init__("%s failed: %s (%d): %s" % (what, ERROR_NAMES.get(code, "?"), code, msg))


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libdppix.so not built (run paper_2511_04261_b300/build.py); no fallback exists")
    L = ct.CDLL(LIB_PATH)
    P, I32, I64, U32, U64 = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_uint32, ct.c_uint64
    L.dp_pix_plan.argtypes = [ct.POINTER(Desc), ct.POINTER(P), ct.POINTER(Sizes)]
    L.dp_pix_plan_destroy.argtypes = [P]
    L.dp_pix_plan_tune.argtypes = [P, ct.c_int, ct.c_int]
    L.dp_pix_plan_tuning.argtypes = [P, ct.c_int, ct.POINTER(ct.c_int)]
    L.dp_pix_release.argtypes = [P, P, I64, P, I64, I64, U32, U32, U64, P, I64, P, U64, P]
    L.dp_pix_release_reconstruct.argtypes = [P, P, I64, P, I64, I64, U32, U32, U64, P, I64, P, I64, I64, ct.c_int, P,
                                             U64, P]
    L.dp_pix_soft_sizes.argtypes = [ct.POINTER(SoftDesc), ct.POINTER(U64)]
    L.dp_pix_soft_forward.argtypes = [ct.POINTER(SoftDesc), P, P, P, P, P]
    L.dp_pix_soft_backward.argtypes = [ct.POINTER(SoftDesc), P, P, P, P, P, P, P]
    L.dp_pix_batch_plan.argtypes = [ct.POINTER(Desc), ct.POINTER(I32), ct.POINTER(I32), U32, ct.POINTER(P)]
    L.dp_pix_batch_destroy.argtypes = [P]
    L.dp_pix_batch_sizes.argtypes = [P, ct.POINTER(U64), ct.POINTER(U64)]
    L.dp_pix_batch_bind.argtypes = [P, ct.POINTER(BatchImage), ct.c_int, P, U64, P]
    L.dp_pix_batch_run.argtypes = [P, ct.c_int, P]
    L.dp_pix_batch_autotune.argtypes = [P, ct.POINTER(BatchImage), ct.c_int, P]
    L.dp_pix_batch_tuning.argtypes = [P, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]
    L.dp_pix_batch_set_path.argtypes = [P, ct.c_int, ct.c_int]
    L.dp_pix_release_keyed.argtypes = [P, P, I64, P, I64, I64, U32, P, P, I64, P, U64, P]
    L.dp_pix_keys_advance.argtypes = [P, U32, U64, P]
    L.dp_pix_release_reconstruct_keyed.argtypes = [P, P, I64, P, I64, I64, U32, P, P, I64, P, I64, I64, ct.c_int,
                                                   P, U64, P]
    L.dp_pix_server_sizes.argtypes = [ct.POINTER(Desc), I32, I32, ct.POINTER(U64), ct.POINTER(U64), ct.POINTER(U64)]
    L.dp_pix_server_create.argtypes = [ct.POINTER(Desc), ct.POINTER(I32), ct.POINTER(I32), U32, P, U32, P, U64,
                                       ct.POINTER(P)]
    L.dp_pix_server_submit.argtypes = [P, U32, P, P, U64, P, ct.POINTER(U64)]
    L.dp_pix_server_wait.argtypes = [P, U64, ct.c_int, ct.POINTER(ServerResult)]
    L.dp_pix_server_counters.argtypes = [P, P, U32]
    L.dp_pix_server_stats_get.argtypes = [P, ct.POINTER(ServerStats)]
    L.dp_pix_server_destroy.argtypes = [P]
    L.dp_pix_release_noalloc.argtypes = [P, P, I64, P, I64, I64, U32, U32, U64, P, I64, P]
    L.dp_pix_store.argtypes = [P, P, U64, ct.POINTER(U64), ct.c_int, P]
    L.dp_pix_store_batch.argtypes = [P, I64, U32, P, I64, P, P]
    L.dp_pix_reconstruct.argtypes = [P, I64, U32, P, I64, I64, ct.c_int, I32, I32, I32, P]
    L.dp_pix_debug_noise.argtypes = [U64, P, U64, P, P, ct.c_float, P]
    L.dp_pix_status.argtypes = [P, ct.POINTER(U32)]
    L.dp_pix_sobel_mask.argtypes = [P, I32, I32, I32, I64, I64, U32, I32, U32, P, I64, I64, P]
    L.dp_pix_utility.argtypes = [P, P, I32, I32, I32, I64, I64, I64, I64, U32, P, P]
    L.dp_pix_last_error.restype = ct.c_char_p
    L.dp_pix_last_error.argtypes = []
    L.dp_pix_version.restype = ct.c_int
    L.dp_pix_prof_enable.argtypes = [ct.c_int]
    L.dp_pix_prof_read.argtypes = [ct.POINTER(ProfEntry), ct.c_int]
    L.dp_pix_prof_reset.argtypes = []
    for name in ("dp_pix_plan", "dp_pix_plan_destroy", "dp_pix_plan_tune", "dp_pix_plan_tuning", "dp_pix_release", "dp_pix_release_reconstruct",
                 "dp_pix_release_noalloc", "dp_pix_store", "dp_pix_soft_sizes", "dp_pix_soft_forward",
                 "dp_pix_soft_backward", "dp_pix_batch_plan", "dp_pix_batch_destroy", "dp_pix_batch_sizes",
                 "dp_pix_batch_bind", "dp_pix_batch_run", "dp_pix_batch_autotune", "dp_pix_batch_tuning",
                 "dp_pix_batch_set_path",
                 "dp_pix_release_keyed", "dp_pix_server_sizes", "dp_pix_server_create", "dp_pix_server_submit",
                 "dp_pix_server_wait", "dp_pix_server_stats_get", "dp_pix_server_counters", "dp_pix_server_destroy",
                 "dp_pix_release_reconstruct_keyed", "dp_pix_keys_advance",
                 "dp_pix_store_batch",
                 "dp_pix_reconstruct",
                 "dp_pix_debug_noise", "dp_pix_status", "dp_pix_prof_enable", "dp_pix_prof_read",
                 "dp_pix_sobel_mask", "dp_pix_utility",
                 "dp_pix_prof_reset"):
        getattr(L, name).restype = ct.c_int
    _lib = L
    return L


def check(rc, what):
    if rc < 0:
        msg = lib().dp_pix_last_error().decode(errors="replace")
        raise DppixError(rc, what, msg)
    return rc
