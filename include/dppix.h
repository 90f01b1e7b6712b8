/*
 * dppix.h -- C ABI of libdppix: region-adaptive differentially private pixelization on NVIDIA B300.
 *
 * The calls follow the paper's statement of the problem (Alg. 3 inputs: image I, grid sizes, privacy
 * budget eps, max variation m, region mask; outputs: the compact noisy-statistics record of Table IV and
 * the restored image I').  A frame is M x N pixels of C interleaved uint8 samples (C = 1..4).  The frame
 * is split into K <= 8 regions; region r gets grid side b_r and budget eps_r, and every b_r x b_r cell of
 * it is released as clip(mean + Laplace(0, sigma_r), 0, R) with sigma_r = R*m / (b_r^2 eps_r) (Eq. 11,
 * Eq. 8).  Regions live on square tiles of side T = lcm{b_r}; each tile belongs to one region (the
 * paper's b x b grid with its subgrids, Eq. 16).
 *
 * Conventions shared by every call:
 *  - Every pointer named d_* is a device pointer owned by the caller; the library never allocates device
 *    memory on these paths.  Host pointers are named h_* or documented as host.
 *  - Calls are asynchronous on `cuda_stream` (a cudaStream_t, NULL = legacy default stream) unless the
 *    comment says they synchronize.
 *  - Every call returns DP_PIX_OK (0) or a negative DP_PIX_E_* code and never throws or aborts.  The
 *    thread-local message of the last failure is returned by dp_pix_last_error().
 *  - A plan is immutable after dp_pix_plan(); it may be used from several host threads and streams at
 *    once.  Calls that share a workspace or output buffer must be ordered by the caller.
 *  - No CPU fallback exists: without a usable CUDA device the compute calls return DP_PIX_E_CUDA.
 */
#ifndef DPPIX_H
#define DPPIX_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DPPIX_API __attribute__((visibility("default")))
#else
#define DPPIX_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define DP_PIX_MAX_REGIONS 8
#define DP_PIX_RECORD_HEADER_BYTES 512

/* ---- return codes ---------------------------------------------------------------------------------- */
#define DP_PIX_OK 0
#define DP_PIX_E_INVALID_ARG (-1)      /* a null pointer, a size or a field out of its documented range */
#define DP_PIX_E_UNSUPPORTED (-2)      /* valid but beyond this library's limits (e.g. T > 128) */
#define DP_PIX_E_PAD_TOO_LARGE (-3)    /* mirror padding would reach past the opposite edge */
#define DP_PIX_E_BUFFER_TOO_SMALL (-4) /* record, workspace or destination capacity too small */
#define DP_PIX_E_BAD_RECORD (-5)       /* record header malformed */
#define DP_PIX_E_CUDA (-6)             /* a CUDA runtime call failed (message has the CUDA error) */
#define DP_PIX_E_TIMEOUT (-7)          /* a bounded device-side wait gave up */
#define DP_PIX_E_DEVICE (-8)           /* a device-side check failed (see dp_pix_status) */

/* ---- enumerations ------------------------------------------------------------------------------------ */
/* Mirror padding of the last tile row/column (Alg. 2 step 4, Alg. 3 step 3).  reflect: the edge sample is
 * not repeated (numpy "reflect"); symmetric: it is (numpy "symmetric"). */
#define DP_PIX_PAD_REFLECT 0
#define DP_PIX_PAD_SYMMETRIC 1
/* No padding, privacy-strict edges (Alg. 1's partial cells, Sec. IV-D): a cell crossing the frame's last
 * row or column holds only its h x w samples inside the frame; its mean is S / (h w) and its noise scale
 * R m / (h w eps_r), so that a sample weighs at most R m / (h w) in it (with mirroring a sample can appear
 * twice in an edge cell).  A cell wholly outside the frame stores 0.  Mask and matte tiles are classified on
 * their pixels inside the frame.  Not with DP_PIX_SRC_VARIANCE (UNSUPPORTED); no padding limit applies. */
#define DP_PIX_PAD_NONE 2

/* Where the tile -> region map comes from (Alg. 3 steps 5-6 and their generalisations).
 *  TILE_LABELS: caller passes u8 labels [G_R][G_C] (values < K), copied into the record.
 *  MASK_U8:     K = 2.  Caller passes the paper's simple-region mask (u8, nonzero = simple) of M x N.
 *               A tile is simple (region 0) iff more than half of its T*T mirror-padded mask samples are
 *               simple (mask mean > 1/2), else complex (region 1); a tie goes to complex.
 *  MATTE_F32:   K = 2.  Caller passes an f32 alpha matte of M x N; a pixel is complex iff
 *               alpha >= matte_threshold; then as MASK_U8.
 *  VARIANCE:    K classes by local variance: per tile S = sum x and Q = sum x^2 over the C*T*T padded
 *               samples, key = n*Q - S^2 (n = C*T*T), tiles ranked ascending by (key, tile index) within the
 *               frame, class q = floor(K * rank / #tiles) -> region q (region 0 = lowest variance). */
#define DP_PIX_SRC_TILE_LABELS 0
#define DP_PIX_SRC_MASK_U8 1
#define DP_PIX_SRC_MATTE_F32 2
#define DP_PIX_SRC_VARIANCE 3

/* Record payload element type: clipped noisy means as f32 or as u8 (round half to even of the f32
 * value), or the exact u32 cell sums (diagnostic: no noise, for integer parity checks). */
#define DP_PIX_REC_F32 0
#define DP_PIX_REC_U8 1
#define DP_PIX_REC_SUM_U32 2

/* Reconstructed image element type: u8 (round half to even) or f32, C interleaved samples per pixel. */
#define DP_PIX_OUT_U8 0
#define DP_PIX_OUT_F32 1

/* ---- problem description ------------------------------------------------------------------------------ */
typedef struct dp_pix_desc {
    int32_t M, N, C;              /* frame rows, columns, interleaved channels (1..4) */
    int32_t K;                    /* number of regions, 1..8 */
    int64_t row_pitch;            /* bytes between consecutive frame rows, >= N*C */
    int32_t grid[DP_PIX_MAX_REGIONS]; /* b_r, 1..64; T = lcm{b_r} <= 128 and T*T*C <= 49152 */
    double eps[DP_PIX_MAX_REGIONS];   /* eps_r > 0 (ignored when noise_free) */
    double value_range;           /* R: samples lie in [0, R]; 255 for u8 frames */
    double m;                     /* max number of samples two neighbouring frames differ in (> 0) */
    int32_t pad_mode;             /* DP_PIX_PAD_* */
    int32_t region_source;        /* DP_PIX_SRC_* */
    float matte_threshold;        /* MATTE_F32 only */
    int32_t record_dtype;         /* DP_PIX_REC_* */
    int32_t noise_free;           /* 1: eta = 0 (the eps -> infinity limit; testing only) */
    int32_t reserved0;
    uint64_t seed;                /* Philox key: (seed mod 2^32, seed >> 32) */
} dp_pix_desc;

typedef struct dp_pix_sizes {
    uint64_t record_bytes;        /* capacity one frame's record buffer must have (worst case) */
    uint64_t workspace_per_frame; /* workspace bytes needed per frame of a dp_pix_release call */
    uint64_t workspace_fixed;     /* plus this many bytes per call */
    uint32_t T, GR, GC, PR, PC;   /* tile side, tile rows/cols, padded rows/cols (Alg. 3 steps 1-2) */
    uint32_t num_tiles;           /* GR * GC */
    uint64_t max_values;          /* max payload elements of one record */
    double sigma[DP_PIX_MAX_REGIONS]; /* Laplace scale of each region */
} dp_pix_sizes;

/* The 512-byte record header, little-endian, at the start of every record (Table IV generalised).
 * The tile-row index, map and payload follow at the offsets it gives. */
/* Noise key of one frame: the Philox counter of its cells carries stream_id (< 2^24) and frame_idx (Eq. 9
 * draws are keyed by (seed, frame, region, cell)).  Used where one call releases frames of several streams. */
typedef struct dp_pix_frame_key {
    uint64_t frame_idx;
    uint32_t stream_id;
    uint32_t reserved;            /* 0 */
} dp_pix_frame_key;

typedef struct dp_pix_record_header {
    char magic[4];                /* "DPPX" */
    uint32_t version;             /* 1 */
    uint32_t header_bytes;        /* 512 */
    uint32_t flags;               /* bit 0: noise-free release */
    uint32_t M, N, C, T, K, GR, GC;
    uint32_t pad_mode, record_dtype, region_source, stream_id, reserved0;
    uint64_t seed, frame_idx;
    double value_range, m;
    uint64_t total_bytes;         /* bytes in use (multiple of 16): what dp_pix_store copies */
    uint64_t map_offset;          /* u8 map [GR][GC] */
    uint32_t grid[DP_PIX_MAX_REGIONS];
    double eps[DP_PIX_MAX_REGIONS];
    double sigma[DP_PIX_MAX_REGIONS];
    uint32_t count[DP_PIX_MAX_REGIONS];          /* tiles of region r */
    uint64_t region_offset[DP_PIX_MAX_REGIONS];  /* byte offset of region r's payload */
    uint64_t rowidx_offset;       /* u32 [GR][K]: region-r tiles in tile rows above */
    uint64_t payload_offset;      /* start of region 0's payload */
    uint8_t reserved[128];
} dp_pix_record_header;

typedef struct dp_pix_plan_s *dp_pix_plan_t;

/* Validates `d`, derives the geometry and sizes (Alg. 2 steps 1-3, Alg. 3 steps 1-2) and returns an
 * immutable plan.  Host only: no CUDA call.  `sz` may be NULL.  Errors: INVALID_ARG, UNSUPPORTED (b_r > 128,
 * T > 128, T*T*C > 49152, more than 2^25 tiles per frame; VARIANCE: more than 16384 tiles or T*C not a
 * multiple of 4), PAD_TOO_LARGE (reflect needs P_R <= M-1 and P_C <= N-1; symmetric P_R <= M, P_C <= N). */
DPPIX_API int dp_pix_plan(const dp_pix_desc *d, dp_pix_plan_t *out, dp_pix_sizes *sz);

/* Frees a plan (host only).  NULL is allowed. */
DPPIX_API int dp_pix_plan_destroy(dp_pix_plan_t plan);

/* Launch-shape knobs of a plan (no counterpart in the paper: they change speed, never results).  Set them
 * before the plan is shared; a call must not race with releases that use the plan.
 *   DP_PIX_TUNE_FUSED_PX       pixel columns per work item of the fused release + reconstruction,
 *                              64..2048 (default 1024; rounded down to whole, aligned tiles)
 *   DP_PIX_TUNE_FUSED_THREADS  threads per block of that kernel, 96, 128, 192 or 256 (default 128)
 *   DP_PIX_TUNE_SPLIT          variance-class dp_pix_release_reconstruct runs its frames as a pipeline of this
 *                              many chunks: every chunk's statistics and rank on the caller's stream, each
 *                              chunk's emission (records and images) on a library side stream once its rank is
 *                              done, forked from and joined to the caller's stream with events, 1..16 (default
 *                              1: everything on the caller's stream)
 *   DP_PIX_TUNE_FUSED_CAP      blocks per SM of the fused emission inside that pipeline, so that it leaves room
 *                              for the next chunk's statistics pass, 0..32 (default 0: its occupancy limit)
 *   DP_PIX_TUNE_WAIT_TRIES     tries of the release kernels' bounded waits for their staged rows before a
 *                              wait gives up with DP_PIX_E_TIMEOUT (through dp_pix_status), 1..2^22
 *                              (default 2^22, seconds: far beyond any copy's latency)
 * And one knob for testing the timeout path, which does change results:
 *   DP_PIX_TUNE_TEST_SHORT_TX  1: every block of the staged release (TILE_LABELS, MASK_U8, MATTE_F32 plans)
 *                              announces 16 bytes more than its first work item's copies deliver, so that
 *                              wait runs out: the call reports DP_PIX_E_TIMEOUT and its records are
 *                              undefined; every copy still lands, and the device stays usable.  0: off
 *                              (default).
 *   DP_PIX_TUNE_TEST_SHRINK    bytes (0..2^20) taken off the records' extent that the bounds-checked build
 *                              (libdppix_checked.so) checks the record writes against, so that a test can make
 *                              a check fire while every access stays inside the real buffer: the writes past
 *                              the shrunken extent are skipped and DP_PIX_E_DEVICE (detail 0x601) is raised.
 *                              No effect in the normal build.  0: off (default).
 * dp_pix_plan_tune returns INVALID_ARG for an unknown knob or a value out of range; dp_pix_plan_tuning
 * writes the current value to *value. */
#define DP_PIX_TUNE_FUSED_PX 1
#define DP_PIX_TUNE_FUSED_THREADS 2
#define DP_PIX_TUNE_SPLIT 4
#define DP_PIX_TUNE_FUSED_CAP 32
#define DP_PIX_TUNE_WAIT_TRIES 8
#define DP_PIX_TUNE_TEST_SHORT_TX 16
#define DP_PIX_TUNE_TEST_SHRINK 64
DPPIX_API int dp_pix_plan_tune(dp_pix_plan_t plan, int knob, int value);
DPPIX_API int dp_pix_plan_tuning(dp_pix_plan_t plan, int knob, int *value);

/*
 * Releases n_frames frames (Alg. 3, generalised to K regions): classifies tiles, reduces every cell of
 * its tile's grid to an exact integer sum, adds Laplace noise drawn from Philox4x32-10 with
 * key (seed mod 2^32, seed >> 32) and counter (cell index in the frame's padded b_r-grid,
 * r | stream_id << 8, frame mod 2^32, frame >> 32) -- word ch for channel ch, inverse-CDF sampler
 * eta = +-sigma_r * ln((k + 1/2) / 2^31) -- clips to [0, R] and writes one self-describing record per
 * frame (Table IV generalised).
 *   d_frames:         frame i starts at d_frames + i*frame_stride (bytes); rows are row_pitch apart.
 *   d_region_src:     per the plan's region_source: u8 labels [G_R][G_C] (src_pitch ignored, frames
 *                     src_frame_stride apart), u8 mask / f32 matte rows src_pitch bytes apart, or NULL
 *                     for VARIANCE.
 *   stream_id:        < 2^24; frame i uses frame index frame_idx0 + i.
 *   d_records:        record i at d_records + i*record_stride; record_stride >= sizes.record_bytes and a
 *                     multiple of 16; d_records 16-byte aligned.
 *   d_ws / ws_bytes:  workspace of >= workspace_fixed + n_frames * workspace_per_frame bytes, 256-byte
 *                     aligned; its contents need not be initialised and are scratch after the call.
 * Record layout (little-endian): 512-byte header, then u32 tile-row index [G_R][K] (number of region-r
 * tiles above each tile row), then the u8 region map [G_R][G_C], then region-major payload: region r's
 * tiles in row-major tile order, each tile's (T/b_r)^2 cells row-major, C channel values per cell; each
 * section starts on a 16-byte boundary.  Header fields are those of dp_pix_record_header above.
 */
DPPIX_API int dp_pix_release(dp_pix_plan_t plan, const void *d_frames, int64_t frame_stride, const void *d_region_src,
                   int64_t src_pitch, int64_t src_frame_stride, uint32_t n_frames, uint32_t stream_id,
                   uint64_t frame_idx0, void *d_records, int64_t record_stride, void *d_ws, uint64_t ws_bytes,
                   void *cuda_stream);

/*
 * dp_pix_release with a noise key per frame instead of (stream_id, frame_idx0 + i): frame i of the call is
 * released with d_keys[i] (device array of n_frames keys), so frames of different streams share one call.
 * Records are byte-identical to releasing each frame alone with its key.  A key whose stream_id is >= 2^24
 * is reported through dp_pix_status() (DP_PIX_E_DEVICE) and its frame's record is undefined.  Other
 * arguments and errors: as dp_pix_release.
 */
DPPIX_API int dp_pix_release_keyed(dp_pix_plan_t plan, const void *d_frames, int64_t frame_stride,
                                   const void *d_region_src, int64_t src_pitch, int64_t src_frame_stride,
                                   uint32_t n_frames, const dp_pix_frame_key *d_keys, void *d_records,
                                   int64_t record_stride, void *d_ws, uint64_t ws_bytes, void *cuda_stream);

/*
 * dp_pix_release followed by dp_pix_reconstruct of the same frames, in one call (Alg. 3 with its
 * restoring steps; Sec. VI-F).  Writes the same records and the same images as the two calls would.
 * When the images' rows are 16-byte aligned and the release uses variance classes with a common grid
 * divisor g in 4..16, the noisy cell means are turned into image rows in the same kernel that writes the
 * records, so the records are not read back; otherwise the two calls run in turn.
 *   Release arguments: as dp_pix_release.  Image arguments: as dp_pix_reconstruct, with the plan's M, N, C
 *   as the bounds: image i at d_out + i*out_frame_stride, rows out_pitch bytes apart, out_type DP_PIX_OUT_*.
 *   The caller owns every buffer.  Returns DP_PIX_OK, or the error codes of the two calls (argument
 *   errors are found before anything is launched; kernel-side errors arrive through dp_pix_status()).
 */
DPPIX_API int dp_pix_release_reconstruct(dp_pix_plan_t plan, const void *d_frames, int64_t frame_stride,
                                         const void *d_region_src, int64_t src_pitch, int64_t src_frame_stride,
                                         uint32_t n_frames, uint32_t stream_id, uint64_t frame_idx0, void *d_records,
                                         int64_t record_stride, void *d_out, int64_t out_frame_stride, int64_t out_pitch,
                                         int out_type, void *d_ws, uint64_t ws_bytes, void *cuda_stream);

/*
 * dp_pix_release_reconstruct with a noise key per frame (as dp_pix_release_keyed): frame i is released
 * with d_keys[i] and its image rebuilt from that record.  Records and images are byte-identical to
 * dp_pix_release_reconstruct of each frame alone with its (stream_id, frame_idx).  Other arguments and
 * errors: as dp_pix_release_reconstruct; INVALID_ARG when d_keys is NULL.
 */
DPPIX_API int dp_pix_release_reconstruct_keyed(dp_pix_plan_t plan, const void *d_frames, int64_t frame_stride,
                                               const void *d_region_src, int64_t src_pitch, int64_t src_frame_stride,
                                               uint32_t n_frames, const dp_pix_frame_key *d_keys, void *d_records,
                                               int64_t record_stride, void *d_out, int64_t out_frame_stride,
                                               int64_t out_pitch, int out_type, void *d_ws, uint64_t ws_bytes,
                                               void *cuda_stream);

/*
 * Adds delta to the frame_idx of each of the n keys at d_keys (device, 8-byte aligned), asynchronously on
 * cuda_stream.  With a keyed release captured in a CUDA graph together with this call, every replay releases
 * the next frames of each stream (fresh noise keys) while the host submits nothing.  Errors: INVALID_ARG, CUDA.
 */
DPPIX_API int dp_pix_keys_advance(dp_pix_frame_key *d_keys, uint32_t n, uint64_t delta, void *cuda_stream);

/* ---- ragged batches (no counterpart in the paper, which releases one frame at a time) ----------------- */
/* Many images of different sizes released with one set of region parameters.  Each image is released
 * exactly as dp_pix_release would release it alone with a plan for its size (same record bytes, same noise:
 * its own stream_id and frame_idx key the draws); the batch runs each phase as one persistent launch over
 * the work items of all images, largest images first, and replays the launches as a CUDA graph.  Region
 * sources: TILE_LABELS, MASK_U8, MATTE_F32 (VARIANCE ranks a whole frame: UNSUPPORTED here). */
typedef struct dp_pix_batch_s *dp_pix_batch_t;

typedef struct dp_pix_batch_image {
    const void *frame;            /* device u8 image, C interleaved samples per pixel */
    int64_t row_pitch;            /* bytes between rows, >= N*C */
    const void *region_src;       /* TILE_LABELS: u8 [G_R][G_C]; MASK_U8: u8 rows src_pitch apart; MATTE_F32:
                                     f32 rows src_pitch apart (4-byte aligned) */
    int64_t src_pitch;
    void *record;                 /* device, dp_pix_batch_sizes bytes for this image, 16-byte aligned */
    void *out;                    /* device reconstruction [M][N][C] (u8 or f32 per out_type), or NULL */
    int64_t out_pitch;            /* bytes between output rows */
    uint32_t stream_id;           /* < 2^24 */
    uint64_t frame_idx;
} dp_pix_batch_image;

/* Plans a batch of n images, image i of M[i] x N[i] (host only).  common: the region parameters as for
 * dp_pix_plan (its M, N and row_pitch are ignored).  Errors: as dp_pix_plan for any image; UNSUPPORTED for
 * VARIANCE. */
DPPIX_API int dp_pix_batch_plan(const dp_pix_desc *common, const int32_t *M, const int32_t *N, uint32_t n,
                                dp_pix_batch_t *out);
DPPIX_API int dp_pix_batch_destroy(dp_pix_batch_t b);

/* record_bytes[i] (array of n, may be NULL): capacity to allocate for image i's record; ws_bytes: device
 * workspace of the whole batch (the image table plus each image's workspace). */
DPPIX_API int dp_pix_batch_sizes(dp_pix_batch_t b, uint64_t *record_bytes, uint64_t *ws_bytes);

/* Binds the images (caller order) and a 256-byte aligned workspace, and uploads the image table on
 * cuda_stream (the host array may be reused on return).  out_type: DP_PIX_OUT_U8 or DP_PIX_OUT_F32 for the
 * images whose `out` is set.  Rebinding drops the captured graph.  Errors: INVALID_ARG (a missing buffer, a
 * pitch or alignment), BUFFER_TOO_SMALL, CUDA. */
DPPIX_API int dp_pix_batch_bind(dp_pix_batch_t b, const dp_pix_batch_image *imgs, int out_type, void *d_ws,
                                uint64_t ws_bytes, void *cuda_stream);

/* Releases every bound image (and reconstructs those with an output), asynchronously on cuda_stream.
 * use_graph != 0: the first call captures the launches into a CUDA graph (on a private stream), and every
 * call launches that graph on cuda_stream.
 * Device-side problems (a bad label) arrive through dp_pix_status().  Errors: INVALID_ARG (not bound), CUDA. */
DPPIX_API int dp_pix_batch_run(dp_pix_batch_t b, int use_graph, void *cuda_stream);

/* Release paths of a batch (all give the same bytes):
 *   DP_PIX_BATCH_PATH_STAGED        each item's rows arrive in shared memory by bulk copies; the CTA's threads
 *                                   share out the item's (tile, cell, row part) units; the images, if any, are
 *                                   written by a separate reconstruction launch
 *   DP_PIX_BATCH_PATH_STREAM        each lane streams its 16-byte column chunk of the item's rows straight into
 *                                   registers (rows realigned by funnel shifts); separate reconstruction
 *   DP_PIX_BATCH_PATH_STREAM_FUSED  as STREAM, and the same launch writes the u8 images from the cell values
 *   DP_PIX_BATCH_PATH_TILES         rows staged as in STAGED, whole warps per tile of the item (segment width
 *                                   1, 2, 4 or 8 tiles sharing the CTA's 8 warps; default 2); separate
 *                                   reconstruction.  The default path (-1).
 * The streaming paths need T * C >= 16 (and their per-item sums within shared memory); the fused one u8
 * images and f32 or u8 records.  Where a path does not apply the batch takes the staged one. */
#define DP_PIX_BATCH_PATH_STAGED 0
#define DP_PIX_BATCH_PATH_STREAM 1
#define DP_PIX_BATCH_PATH_STREAM_FUSED 2
#define DP_PIX_BATCH_PATH_TILES 3

/* Times the release paths and their segment widths (tiles per work item) on the bound batch -- reps runs
 * each, overwriting its records and outputs -- keeps the fastest, rebinds `imgs` (the images bound last) and
 * drops the graph.  Synchronizes cuda_stream.  dp_pix_batch_tuning reports the width and path in use (path
 * may be NULL). */
DPPIX_API int dp_pix_batch_autotune(dp_pix_batch_t b, const dp_pix_batch_image *imgs, int reps, void *cuda_stream);
DPPIX_API int dp_pix_batch_tuning(dp_pix_batch_t b, int *seg_tiles, int *path);

/* Chooses a release path (DP_PIX_BATCH_PATH_*, or -1: the default, whole warps per tile)
 * and segment width (0: the path's default) without timing; takes effect at the next dp_pix_batch_bind.
 * Errors: INVALID_ARG. */
DPPIX_API int dp_pix_batch_set_path(dp_pix_batch_t b, int path, int seg_tiles);

/* ---- serving loop (no counterpart in the paper; its deployment motivation is many cameras) --------------- */
/* A request loop for frames arriving from many cameras.  Requests are queued from host memory by any
 * thread; a worker thread owned by the server issues every CUDA call after creation.  Up to n_streams
 * batches are in flight at once: whenever one is free, the worker admits the queued requests, oldest first,
 * that the free part of the caller's arena holds (the memory budget), copies their frames in, releases all
 * frames of one resolution in one keyed launch (with the reconstruction when a request asks for it), and
 * copies the records (and images) back -- so requests that arrive while others are on the GPU join the
 * next batch, and its copies and kernels overlap the running ones.
 * Noise keys: frame f of camera c is released with stream_id c and frame_idx f, where f counts the
 * camera's frames in submission order, starting from first_frame[c].  The counters live in device memory
 * and are advanced on the device as batches are formed; each record is byte-identical to dp_pix_release
 * of its frame alone with that key.  dp_pix_server_counters reads the counters back: creating the next
 * server with them continues every camera's count, so a restarted server never draws one key twice (the
 * parallel composition of Thm 1 needs independent noise).  Region source: VARIANCE (no per-frame side
 * input); other sources are UNSUPPORTED here. */
typedef struct dp_pix_server_s *dp_pix_server_t;

typedef struct dp_pix_server_result {
    uint64_t ticket;
    uint64_t frame_idx;           /* the frame's key index (from its record's header) */
    uint64_t record_bytes;        /* header.total_bytes of the record now in the request's host buffer */
    uint32_t camera;
    int32_t status;               /* DP_PIX_OK or a DP_PIX_E_* code of the batch that carried the frame */
    double queue_us;              /* submit -> admitted into a batch */
    double latency_us;            /* submit -> results in host memory */
} dp_pix_server_result;

typedef struct dp_pix_server_stats {
    uint64_t submitted, completed, batches, launches;
    uint64_t frames_in_flight_max;  /* most frames on the device at once */
    double mean_batch_frames;
    uint64_t arena_bytes_in_use_max; /* most arena bytes held by batches at once */
    uint64_t arena_heap_bytes;       /* arena bytes available to batches (the arena minus counters and keys) */
} dp_pix_server_stats;

/* Device bytes one admitted frame of an M x N camera holds while its batch runs (frame + record +
 * workspace), the host record capacity every request of that camera must provide, and the bytes a
 * reconstruction adds.  Any pointer may be NULL.  Host only. */
DPPIX_API int dp_pix_server_sizes(const dp_pix_desc *common, int32_t M, int32_t N, uint64_t *slot_bytes,
                                  uint64_t *record_bytes, uint64_t *recon_bytes);

/* Creates a server for n_cameras cameras of M[c] x N[c] (common: the region parameters as for dp_pix_plan;
 * M, N, row_pitch ignored).  first_frame: n_cameras starting frame indices (the values dp_pix_server_counters
 * returned for an earlier server with the same seed), or NULL for 0.  d_arena: arena_bytes of device memory,
 * 256-byte aligned, owned by the caller and untouched by anyone else until dp_pix_server_destroy returns.
 * Its first bytes hold the counters (8 per camera) and the key tables (4 KiB per stream); the rest is handed
 * to batches.  n_streams: batches in flight (1..8).  Synchronizes the calling thread with the counter upload.
 * Errors: as dp_pix_plan, UNSUPPORTED (source), BUFFER_TOO_SMALL (no room for one frame of the largest
 * resolution with its reconstruction), CUDA. */
DPPIX_API int dp_pix_server_create(const dp_pix_desc *common, const int32_t *M, const int32_t *N, uint32_t n_cameras,
                                   const uint64_t *first_frame, uint32_t n_streams, void *d_arena,
                                   uint64_t arena_bytes, dp_pix_server_t *out);

/* Queues frame `host_frame` (M*N*C bytes, rows dense; pinned memory copies asynchronously) of `camera`; its
 * record will be written to host_record (record_cap >= dp_pix_server_sizes' record_bytes) and, when
 * host_out is not NULL, its pixelized image (M*N*C u8, rows dense) to host_out.  Every buffer must stay
 * valid until dp_pix_server_wait has returned the request's result.  *ticket identifies the request.
 * Thread-safe; a camera's frames take consecutive indices in the order their submit calls return.
 * Errors: INVALID_ARG (camera, buffer), BUFFER_TOO_SMALL (record_cap). */
DPPIX_API int dp_pix_server_submit(dp_pix_server_t s, uint32_t camera, const void *host_frame, void *host_record,
                                   uint64_t record_cap, void *host_out, uint64_t *ticket);

/* Waits up to timeout_ms (< 0: forever; 0: poll) for request `ticket` and fills *res once (the result is then
 * forgotten).  Returns DP_PIX_OK, DP_PIX_E_TIMEOUT (not done yet), or INVALID_ARG (unknown ticket).
 * Thread-safe. */
DPPIX_API int dp_pix_server_wait(dp_pix_server_t s, uint64_t ticket, int timeout_ms, dp_pix_server_result *res);

/* Waits until every submitted request has been released, then copies the first n cameras' next frame
 * indices (device counters) to next_frame (host, n entries).  Requests submitted by other threads during
 * the call may or may not be counted.  Errors: INVALID_ARG (n > cameras, NULL), CUDA. */
DPPIX_API int dp_pix_server_counters(dp_pix_server_t s, uint64_t *next_frame, uint32_t n);

DPPIX_API int dp_pix_server_stats_get(dp_pix_server_t s, dp_pix_server_stats *st);

/* Finishes the queued requests, stops the worker and frees the server's host state (the arena is the
 * caller's).  NULL is allowed. */
DPPIX_API int dp_pix_server_destroy(dp_pix_server_t s);

/* ---- differentiable soft layer (a training pattern on top of the release; not in the paper) ------------ */
/* y = w * P~_{b0}(x) + (1 - w) * P~_{b1}(x) on planar f32 images, where P~_b is the uniform release of
 * Alg. 2 (mirror pad, cell mean, Laplace noise of scale R m / (b^2 eps) (Eq. 11 with Eq. 8), clip to [0, R],
 * repeat, crop) of every channel plane.  The noise of grid j, cell (cy, cx) of image n is drawn with the
 * Philox counter (cy * G_C,j + cx, j | stream_id << 8, (frame0 + n) mod 2^32, (frame0 + n) >> 32) and the
 * release's sampler, so a backward pass sees the forward's draws (the noise is a constant of the layer). */
typedef struct dp_pix_soft_desc {
    int32_t B, C, H, W;           /* images, channels (1..4), rows, columns: x [B][C][H][W], w [B][1][H][W] */
    int32_t grid[2];              /* b0 (weighted by w), b1 (weighted by 1 - w); 1..128 */
    double eps[2];                /* eps_0, eps_1 > 0 (ignored when noise_free) */
    double value_range;           /* R (1 for images in [0, 1]) */
    double m;                     /* max-variation m */
    int32_t pad_mode;             /* DP_PIX_PAD_* */
    int32_t noise_free;           /* nonzero: eta = 0 */
    uint32_t stream_id;
    uint64_t seed;
    uint64_t frame0;              /* image n uses frame index frame0 + n */
} dp_pix_soft_desc;

/* Bytes of the per-cell buffer `pre` (and of the backward's workspace): 4 * B * C * (G_R,0 G_C,0 + G_R,1 G_C,1).
 * Host only.  Errors: INVALID_ARG, UNSUPPORTED (grid > 128), PAD_TOO_LARGE. */
DPPIX_API int dp_pix_soft_sizes(const dp_pix_soft_desc *d, uint64_t *pre_bytes);

/* Forward.  x, w, y: device f32, dense planar as in the desc.  pre (device, dp_pix_soft_sizes bytes,
 * caller-owned) receives the unclipped noisy cell means, per image grid 0's [C][G_R,0][G_C,0] block then
 * grid 1's; the backward needs it.  Asynchronous on cuda_stream.  Errors: as dp_pix_soft_sizes, CUDA. */
DPPIX_API int dp_pix_soft_forward(const dp_pix_soft_desc *d, const float *x, const float *w, float *y, float *pre,
                                  void *cuda_stream);

/* Backward of L with dL/dy = gy, the noise held constant:
 *   dw(p) = sum_ch gy(p) (P~_{b0}(p) - P~_{b1}(p));
 *   dx(q) = sum_j sum over the cells c whose (mirror-padded) samples read q, once per such sample, of
 *           [0 < pre_c < R] / b_j^2 * sum_{p in c inside the image} gy(p) w_j(p),   w_0 = w, w_1 = 1 - w.
 * w, gy, pre: inputs (pre from dp_pix_soft_forward with the same desc); dx [B][C][H][W], dw [B][1][H][W]:
 * outputs.  d_ws: dp_pix_soft_sizes bytes of scratch, needed unless both grids are powers of two in
 * 4..128 with H a multiple of the larger, W a multiple of 128 and 16-byte aligned buffers (NULL is then
 * allowed).  Asynchronous.  Errors: as dp_pix_soft_sizes, INVALID_ARG (missing buffer), CUDA. */
DPPIX_API int dp_pix_soft_backward(const dp_pix_soft_desc *d, const float *w, const float *gy, const float *pre,
                                   float *dx, float *dw, float *d_ws, void *cuda_stream);

/*
 * dp_pix_release without a workspace argument, for callers that cannot allocate device memory: code
 * running while a CUDA graph is captured (cudaMalloc is not allowed there), plug-ins whose host framework
 * owns every device allocation and passes in only inputs and outputs, and real-time loops that must not
 * enter an allocator.  The paper has no counterpart; this is a deployment convenience.
 *   Arguments, results and errors are those of dp_pix_release; the workspace is a 16 MiB array built into
 *   the library (each GPU that loads the library holds it until the process exits).  A call whose frames
 *   need more (n_frames * sizes.workspace_per_frame > 16 MiB) is rejected with DP_PIX_E_BUFFER_TOO_SMALL
 *   and a message; nothing is launched.  This entry point calls no cudaMalloc, cudaFree or other allocating
 *   routine.
 *   The first call on a device looks up that device's address of the array (cudaGetSymbolAddress); make
 *   that first call before any stream capture.
 *   Every call shares the one array and it keeps the last call's contents (the kernels overwrite every
 *   byte they read, so nothing needs clearing).  Calls whose work overlaps on the GPU (different streams,
 *   or host threads without ordering) race on the array: order them on one stream.
 */
DPPIX_API int dp_pix_release_noalloc(dp_pix_plan_t plan, const void *d_frames, int64_t frame_stride,
                                     const void *d_region_src, int64_t src_pitch, int64_t src_frame_stride,
                                     uint32_t n_frames, uint32_t stream_id, uint64_t frame_idx0, void *d_records,
                                     int64_t record_stride, void *cuda_stream);

/*
 * Copies one record's used bytes (header total_bytes, <= capacity) from device memory to `dst` (host if
 * dst_is_host, else device) and writes that count to *written.  Synchronizes on cuda_stream to read the
 * header.  Errors: BAD_RECORD, BUFFER_TOO_SMALL (cap < total_bytes), CUDA.
 */
DPPIX_API int dp_pix_store(const void *d_record, void *dst, uint64_t cap, uint64_t *written, int dst_is_host,
                 void *cuda_stream);

/*
 * Batched dp_pix_store for n records d_records + i*record_stride (device) into host memory
 * h_dst + i*dst_stride (pinned memory makes the copies asynchronous to the host until the final sync):
 * one strided device->host read of the n headers, then one copy of each record's used bytes.  written[i]
 * (host array, may be NULL) receives record i's size.  Synchronizes on cuda_stream.  Errors: BAD_RECORD,
 * BUFFER_TOO_SMALL (a record larger than dst_stride), CUDA.
 */
DPPIX_API int dp_pix_store_batch(const void *d_records, int64_t record_stride, uint32_t n, void *h_dst,
                                 int64_t dst_stride, uint64_t *written, void *cuda_stream);

/*
 * Rebuilds the pixelized frames from their records alone (Sec. VI-F: the stored metadata suffice;
 * Alg. 2 steps 10-11): every pixel of a cell takes the cell's stored value; the padding is cropped.
 * Geometry is read from each record's header on the device, so no plan and no host sync are needed.
 *   d_records:   n_records records, record_stride bytes apart (>= 512, multiple of 16); record_stride is
 *                also each record's capacity: a header whose sections reach past it is rejected.
 *   d_out:       image i at d_out + i*out_frame_stride; rows out_pitch bytes apart; out_type DP_PIX_OUT_*.
 *   max_M, max_N, max_C: caller's bound on the records' geometry (checked on the device; a record beyond
 *                it, or a malformed one, is skipped and flags DP_PIX_E_DEVICE in the status word).
 */
DPPIX_API int dp_pix_reconstruct(const void *d_records, int64_t record_stride, uint32_t n_records, void *d_out,
                       int64_t out_frame_stride, int64_t out_pitch, int out_type, int32_t max_M, int32_t max_N,
                       int32_t max_C, void *cuda_stream);

/*
 * Diagnostic: for i < n, runs Philox4x32-10 on counter h_ctr-style d_ctr[4i..4i+3] and key (seed mod 2^32,
 * seed >> 32), writes the four words to d_words[4i..] (may be NULL) and the Laplace(0, sigma) draws of
 * the four words to d_eta[4i..] (may be NULL) with the release path's sampler.
 */
DPPIX_API int dp_pix_debug_noise(uint64_t seed, const uint32_t *d_ctr, uint64_t n, uint32_t *d_words, float *d_eta,
                       float sigma, void *cuda_stream);

/* ---- utility metrics and edge masks ------------------------------------------------------------------- */
/*
 * Edge-based simple/complex pixel mask (Sec. VI-A: region masks from an edge detector such as the Sobel
 * operator).  For each pixel: I = sum of its C samples; Gx, Gy = the 3 x 3 Sobel responses of I (Gx: right
 * column minus left column with row weights 1, 2, 1; Gy: bottom row minus top row with column weights
 * 1, 2, 1), the frame mirrored at its four borders by pad_mode (DP_PIX_PAD_REFLECT: edge sample not
 * repeated; DP_PIX_PAD_SYMMETRIC: repeated).  mask = 1 (simple) if Gx^2 + Gy^2 < tau, else 0 (complex):
 * exact integers, so tau is a threshold on the squared gradient in channel-sum units.  The mask is the
 * input of a DP_PIX_SRC_MASK_U8 release.
 *   d_frames: n_frames frames of M x N x C u8, rows row_pitch bytes apart, frames frame_stride apart.
 *   d_mask:   n_frames u8 masks of M x N, rows mask_pitch apart, frames mask_frame_stride apart.
 * Caller-owned device buffers; asynchronous on cuda_stream; n_frames = 0 does nothing.  Errors: INVALID_ARG
 * (M or N < 2, C outside 1..4, bad pad_mode, pitches or strides too small, NULL), UNSUPPORTED (M or N >
 * 2^24), CUDA.
 */
DPPIX_API int dp_pix_sobel_mask(const void *d_frames, int32_t M, int32_t N, int32_t C, int64_t row_pitch,
                                int64_t frame_stride, uint32_t n_frames, int32_t pad_mode, uint32_t tau, void *d_mask,
                                int64_t mask_pitch, int64_t mask_frame_stride, void *cuda_stream);

/* Per-frame utility of a release (Sec. VII-A, VII-B: MSE and SSIM of the released frame against the
 * original).  Written by dp_pix_utility in device memory. */
typedef struct dp_pix_utility_t {
    uint64_t sse;                 /* exact sum of squared sample differences */
    uint64_t windows;             /* 7 x 7 windows per channel: (M - 6)(N - 6) */
    double ssim_sum;              /* sum of the window SSIM values over windows and channels */
    double mse;                   /* sse / (M N C) */
    double ssim;                  /* ssim_sum / (windows C) */
} dp_pix_utility_t;

/*
 * MSE and SSIM of n_frames image pairs (x: original, y: release), M x N x C u8.  SSIM is Wang et al.'s
 * structural similarity (IEEE TIP 2004) with the defaults of the toolkit the paper used: every 7 x 7
 * window inside the image, uniform weights, sample variances and covariance (1/48 normalisation),
 * C1 = (0.01 * 255)^2, C2 = (0.03 * 255)^2, the mean over windows and channels.  Window sums are exact
 * integers; each window's value is rounded once (fp32) and summed in fp64.
 *   d_out: n_frames entries of dp_pix_utility_t (device memory, 8-byte aligned), zeroed by this call.
 * Caller-owned device buffers; asynchronous on cuda_stream; n_frames = 0 does nothing.  Errors: INVALID_ARG
 * (M or N < 7, C outside 1..4, pitches or strides too small, NULL, misaligned d_out), UNSUPPORTED (M or N >
 * 2^24), CUDA.
 */
DPPIX_API int dp_pix_utility(const void *d_x, const void *d_y, int32_t M, int32_t N, int32_t C, int64_t pitch_x,
                             int64_t pitch_y, int64_t frame_stride_x, int64_t frame_stride_y, uint32_t n_frames,
                             dp_pix_utility_t *d_out, void *cuda_stream);

/* Synchronizes cuda_stream and returns DP_PIX_OK, or the first device-side error code recorded since the
 * last call (then clears it).  *detail (may be NULL) receives a kernel-specific detail word. */
DPPIX_API int dp_pix_status(void *cuda_stream, uint32_t *detail);

/* Thread-local, NUL-terminated message of the last failed call on this thread ("" if none). */
DPPIX_API const char *dp_pix_last_error(void);

/* Library version as 10000*major + 100*minor + patch. */
DPPIX_API int dp_pix_version(void);

/* ---- launch accounting ------------------------------------------------------------------------------- */
/* Every kernel launch the library makes is counted per kernel name.  With timing enabled (1) each
 * launch is bracketed by CUDA events on its stream and the elapsed times are summed when
 * dp_pix_prof_read() is called (which synchronizes those events).  Host-side bookkeeping only. */
typedef struct dp_pix_prof_entry {
    char name[48];
    uint64_t launches;
    double total_ms;              /* only while timing was enabled */
} dp_pix_prof_entry;

DPPIX_API int dp_pix_prof_enable(int timing);
/* Fills up to `cap` entries, returns the number of distinct kernels (>= 0) or a negative error. */
DPPIX_API int dp_pix_prof_read(dp_pix_prof_entry *out, int cap);
DPPIX_API int dp_pix_prof_reset(void);

#ifdef __cplusplus
}
#endif
#endif /* DPPIX_H */
