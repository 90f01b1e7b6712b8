"""B300-native region-adaptive differentially private pixelization (arxiv 2511.04261).

The compute path is libdppix.so (hand-written CUDA for sm_103a behind the C ABI of include/dppix.h);
this package is its Python binding.  The library is loaded on first use and there is no fallback: a
missing or unloadable library raises.
"""
from . import _lib
from ._lib import (DppixError, OUT_F32, OUT_U8, PAD_NONE, PAD_REFLECT, PAD_SYMMETRIC, REC_F32, REC_SUM_U32, REC_U8,
                   SRC_MASK_U8, SRC_MATTE_F32, SRC_TILE_LABELS, SRC_VARIANCE, TUNE_FUSED_PX, TUNE_FUSED_THREADS, TUNE_SPLIT,
                   TUNE_TEST_SHORT_TX, TUNE_WAIT_TRIES, TUNE_FUSED_CAP, TUNE_TEST_SHRINK, BATCH_PATH_STAGED, BATCH_PATH_STREAM, BATCH_PATH_STREAM_FUSED,
                   BATCH_PATH_TILES)
from .api import (Plan, dp_pix_debug_noise, dp_pix_plan, dp_pix_reconstruct, dp_pix_release,
                  dp_pix_release_reconstruct, dp_pix_status,
                  dp_pix_store, dp_pix_store_batch, prof_enable, prof_read, prof_reset, record_header)

from .batch import BatchPlan
from .serve import Server, dp_pix_keys_advance, dp_pix_release_keyed, dp_pix_release_reconstruct_keyed, key_table
from .soft import SoftPixelize, SoftSpec, soft_backward, soft_forward, soft_pixelize
from .utility import dp_pix_sobel_mask, dp_pix_utility, utility_values

__version__ = "0.1.0"
