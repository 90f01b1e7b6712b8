// common.cuh -- internal types and device helpers of libdppix (region-adaptive DP pixelization).
//
// Plain-old-data structs passed by value to every kernel, the counter-based generator, the Laplace
// sampler and the mirror-padding index.  Nothing here allocates; nothing here is shared with the oracle.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "dppix.h"

namespace dppix {

constexpr int kMaxK = DP_PIX_MAX_REGIONS;
constexpr int kMaxT = 128;
constexpr int kMaxTileBytes = 49152;     // T*T*C limit (one staged tile)
constexpr int kMaxRankTiles = 16384;     // VARIANCE: tiles of one frame ranked in shared memory
constexpr int kFinalizeSmemTiles = 200000;  // frames up to this many tiles finalise their map in shared memory
constexpr int kMaxFrameTiles = 1 << 25;      // tiles of one frame (larger maps are finalised from global memory)
constexpr uint32_t kWaitTries = 1u << 22;     // default tries of a bounded mbarrier wait
constexpr int kMaxSplit = 16;                 // frame chunks of a pipelined release + reconstruction
constexpr int kHeaderBytes = DP_PIX_RECORD_HEADER_BYTES;

// Geometry and constants of a plan (Alg. 2 steps 1-3, Alg. 3 steps 1-2, Eq. 11).
struct Geom {
    int32_t M, N, C, K, T, GR, GC, PR, PC;
    int32_t pad_mode, source, dtype, noise_free;
    int32_t es;                       // record element bytes
    int64_t pitch;                    // frame row pitch
    int32_t grid[kMaxK];
    int32_t cells_side[kMaxK];        // T / b_r
    float sigma_f[kMaxK];
    float b2_f[kMaxK];                // b_r^2 as float (exact)
    float inv_b2_f[kMaxK];            // 1 / b_r^2 when b_r is a power of two (exact), else 0
    double sigma[kMaxK];
    double eps[kMaxK];
    double R, m;
    float R_f;
    float matte_thr;
    uint64_t seed;
    uint32_t ntiles;
    int32_t g;                        // gcd of the grids (variance path granularity)
    int32_t var_onepass;              // VARIANCE with 4 <= g <= 16: g-cell sums kept, image read once
    int32_t b_min;
    int32_t idx_bits;                 // bits for the tile index in a packed rank key
    int32_t val_bits;                 // bits of a packed (key, tile index) value
    uint64_t rowidx_offset, map_offset, payload_offset, record_cap;
    // workspace layout, per frame
    uint64_t ws_per_frame, ws_tileoff, ws_tilelist, ws_keys, ws_gsum;
    int32_t gx_cells, gy_cells;       // g-image: (GR*T/g) rows of (GC*T/g) g-cells, C u16 sums each
    int32_t gpitch;                   // u16 values per g-image row: gx_cells * C rounded up to 16 bytes
    // launch shapes
    int32_t seg_tiles;                // tiles per staged segment of a tile row
    int32_t seg_per_row;              // ceil(GC / seg_tiles)
    int32_t seg_rowstride;            // bytes per staged row (multiple of 16)
    int32_t vbands;                   // max bands of a staged tile = T / b_min (or T / g for stats)
    int32_t fused_px, fused_threads;  // launch shape of the fused release + reconstruction (tunable)
    int32_t split;                    // frame chunks of a fused call's pipeline (tunable)
    int32_t fused_cap;                // blocks per SM of the fused kernel inside that pipeline (0: occupancy)
    uint32_t wait_tries;              // tries of a bounded mbarrier wait before it gives up (tunable)
    uint32_t test_short_tx;           // test knob: bytes announced beyond what a CTA's first item delivers
    uint32_t test_shrink;             // test knob: bytes taken off the records extent the checked build sees
    // release work units (k_release): a b_r x b_r cell is summed by 2^rel_lp[r] adjacent lanes (row parts);
    // a tile of region r is rel_units[r] units, a multiple of rel_pmax (the largest part count)
    int32_t rel_lp[kMaxK];
    int32_t rel_units[kMaxK];
    int32_t rel_pmax;
    uint32_t rkey[20];                // Philox key of each of the 10 rounds, (lo, hi) pairs (from the seed)
};

// Row parts of one b x b cell of C-channel u8 samples in the release: the smallest power of two P (at most
// min(b, 32)) that keeps ceil(b/P) * b * C bytes per part within a budget, so that work units are similar.
constexpr int kRelPartBytes = 384;
constexpr int kRelMinUnits = 64;  // work units an item of one region should at least hold

// Tiles per classification item of a batch (source rows of at least 256 bytes, at most 16 tiles); es is the
// source element size (1: u8 mask, 4: f32 matte).
__host__ __device__ inline int cls_seg_tiles(int T, int es) {
    const int S = (256 + T * es - 1) / (T * es);
    return S < 1 ? 1 : (S > 16 ? 16 : S);
}
__host__ __device__ inline int rel_parts(int b, int C) {
    int P = 1;
    while (2 * P <= b && P < 32 && ((b + P - 1) / P) * b * C > kRelPartBytes) P *= 2;
    return P;
}

// Per-call arguments of a release.
struct CallArgs {
    const uint8_t *frames;
    int64_t frame_stride;
    const uint8_t *src;
    int64_t src_pitch, src_frame_stride;
    uint32_t n_frames;
    uint32_t stream_id;
    uint64_t frame_idx0;
    uint8_t *records;
    int64_t record_stride;
    uint8_t *ws;
    int32_t vec;                      // widest safe global load for frame rows: 16, 4 or 1 bytes
    int32_t *status;                  // device status word
    const dp_pix_frame_key *keys;     // per-frame (stream id, frame index), or NULL: stream_id, frame_idx0 + f
    // extents of the call's buffers from frames / records / ws (what the bounds-checked build checks against)
    uint64_t frames_bytes, records_bytes, ws_bytes;
};

// Noise key of frame f of a call: its stream id and frame index.
__device__ __forceinline__ uint32_t key_stream(const CallArgs &a, uint32_t f) {
    return a.keys ? a.keys[f].stream_id : a.stream_id;
}
__device__ __forceinline__ uint64_t key_frame(const CallArgs &a, uint32_t f) {
    return a.keys ? a.keys[f].frame_idx : a.frame_idx0 + f;
}

// One image of a ragged batch: its own geometry and call arguments, as a single-image release would get
// them, plus where its work items start in each phase's flattened work list.
struct BatchEntry {
    Geom g;
    CallArgs a;
    uint8_t *out;                     // reconstruction target (NULL: none)
    int64_t out_pitch;
    uint64_t rec_cap;                 // bytes of the image's record buffer
    uint32_t base[4];                 // first item: [0] classify rows, [1] finalize, [2] release items, [3] rebuild
    uint32_t pad_;
};

struct BatchShared {
    Geom g;
    CallArgs a;
};

// Image owning global item `item` of phase `phase` (tab sorted by base[phase]); every thread of the block
// computes it.
__device__ __forceinline__ int batch_find(const BatchEntry *tab, uint32_t n, uint32_t item, int phase) {
    int lo = 0, hi = (int)n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].base[phase] <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Copies image i's geometry and arguments into shared memory (whole block; barriers on both sides).
__device__ __forceinline__ void batch_load(const BatchEntry *tab, int i, BatchShared &bs) {
    static_assert(sizeof(BatchShared) % 4 == 0, "word copy");
    __syncthreads();
    const uint32_t *src = reinterpret_cast<const uint32_t *>(&tab[i].g);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&bs);
    for (int k = threadIdx.x; k < (int)(sizeof(BatchShared) / 4); k += blockDim.x) dst[k] = src[k];
    __syncthreads();
}

// ---------------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32->64 multiplies with the
// published multipliers, the key bumped by the published Weyl constants between rounds.
// ---------------------------------------------------------------------------------------------------
__device__ __forceinline__ void philox_round(uint4 &c, uint2 &k) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int round = 0; round < 10; ++round) philox_round(c, k);
    return c;
}

// Philox-4x32-10 for counters that differ only in their first word: philox_prep does the first round's
// work on the other three words once, philox_finish completes one counter (same words as philox4x32_10).
struct PhiloxPrep {
    uint32_t x1, y1, zxor;  // round-1 outputs that do not depend on the first word; c3 ^ k.y
    uint2 k1;               // the key after round 1
};

__device__ __forceinline__ PhiloxPrep philox_prep(uint32_t c1, uint32_t c2, uint32_t c3, uint2 k) {
    PhiloxPrep p;
    p.x1 = __umulhi(0xCD9E8D57u, c2) ^ c1 ^ k.x;
    p.y1 = 0xCD9E8D57u * c2;
    p.zxor = c3 ^ k.y;
    p.k1 = make_uint2(k.x + 0x9E3779B9u, k.y + 0xBB67AE85u);
    return p;
}

__device__ __forceinline__ uint4 philox_finish(const PhiloxPrep &p, uint32_t c0) {
    uint4 c = make_uint4(p.x1, p.y1, __umulhi(0xD2511F53u, c0) ^ p.zxor, 0xD2511F53u * c0);
    uint2 k = p.k1;
#pragma unroll
    for (int round = 1; round < 10; ++round) philox_round(c, k);
    return c;
}

// philox_finish with the round keys read from the plan (rk[2r], rk[2r + 1]: the key of round r), the products
// as one 64-bit multiply each (measured 1.4 % faster in the fused emission than philox_finish).
__device__ __forceinline__ uint4 philox_finish_rk(const PhiloxPrep &p, uint32_t c0, const uint32_t *rk) {
    uint4 c = make_uint4(p.x1, p.y1, __umulhi(0xD2511F53u, c0) ^ p.zxor, 0xD2511F53u * c0);
#pragma unroll
    for (int round = 1; round < 10; ++round) {
        const uint64_t p0 = (uint64_t)c.x * 0xD2511F53u, p1 = (uint64_t)c.z * 0xCD9E8D57u;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * round], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * round + 1], (uint32_t)p0);
    }
    return c;
}

__device__ __forceinline__ uint32_t word_of(const uint4 &w, int i) {
    return i == 0 ? w.x : (i == 1 ? w.y : (i == 2 ? w.z : w.w));
}

// Counter of the noise draw of one cell: (cell index in the frame's padded b_r-grid, r | stream << 8,
// frame mod 2^32, frame >> 32); key (seed mod 2^32, seed >> 32).  Output word ch is channel ch.
__device__ __forceinline__ uint4 cell_noise_words(uint64_t seed, uint32_t cell_idx, uint32_t region,
                                                  uint32_t stream_id, uint64_t frame) {
    return philox4x32_10(make_uint4(cell_idx, region | (stream_id << 8), (uint32_t)frame, (uint32_t)(frame >> 32)),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// Laplace(0, sigma) by the inverse CDF at u = (x + 1/2) / 2^32 (Eq. 9).  With k = x (lower half) or
// k = 2^32-1-x (upper half, sign flipped), ln(2u) or ln(2(1-u)) is ln t, t = (k + 1/2) / 2^31 in (0, 1).
// ln t is evaluated without a branch, so that the lanes of a warp never split; both halves are computed
// and one is selected:
//  - t < 1/sqrt(2): ln 2 * __log2f(t).  |ln t| > 0.34 there, so the intrinsic's documented error (absolute
//    2^-22 on [1/2, 2], 2 ulp elsewhere) stays a relative error below 1e-6;
//  - t >= 1/sqrt(2): y = t - 1 = -(j + 1/2) / 2^31 from the exact integer j = 2^31-1-k, so nothing cancels
//    near t = 1, and ln(1 + y) = 2 atanh(s), s = y / (2 + y), |s| <= 0.172, from the odd series of atanh
//    (Abramowitz & Stegun 4.5.64 with 4.1.27) truncated after s^11 (relative truncation error < 3e-9).
__device__ __forceinline__ float laplace_from_word(uint32_t x, float sigma) {
    const bool upper = (x >> 31) != 0u;
    const uint32_t k = upper ? ~x : x;    // [0, 2^31)
    const bool low = k <= 1518500249u;     // t < 1/sqrt(2)
    const float t = fmaf(__uint2float_rn(k), 0x1p-31f, 0x1p-32f);
    const float ln_low = 0.693147180559945309f * __log2f(t);
    const uint32_t j = 0x7FFFFFFFu - k;
    const float y = -fmaf(__uint2float_rn(j), 0x1p-31f, 0x1p-32f);
    const float sr = __fdividef(y, 2.0f + y);
    const float z = sr * sr;
    float poly = fmaf(z, 1.0f / 11.0f, 1.0f / 9.0f);
    poly = fmaf(z, poly, 1.0f / 7.0f);
    poly = fmaf(z, poly, 1.0f / 5.0f);
    poly = fmaf(z, poly, 1.0f / 3.0f);
    const float ln_high = 2.0f * fmaf(sr * z, poly, sr);  // ln(1 + y)
    const float lnt = low ? ln_low : ln_high;
    return upper ? -sigma * lnt : sigma * lnt;
}

// Clipped noisy mean (Sec. IV-D; Alg. 2 steps 6-9): v = min(max(S / b^2 + eta, 0), R).
__device__ __forceinline__ float noisy_mean(uint32_t S, float b2, float inv_b2, float eta, float R) {
    // a power-of-two b^2 has an exact reciprocal, and then the product is the correctly rounded quotient
    float mu;
    if (inv_b2 != 0.0f)
        mu = __fmul_rn(__uint2float_rn(S), inv_b2);
    else
        mu = __fdiv_rn(__uint2float_rn(S), b2);
    const float v = __fadd_rn(mu, eta);
    return fminf(fmaxf(v, 0.0f), R);
}

// Noise, clip and store of one cell's C channels (Alg. 3 steps 9-10 and 15-17) from its Philox words;
// sigma, b^2 and 1/b^2 (0 when not exact) of its region.  ov (optional) receives the value a
// reconstruction reads back from the stored element (Sec. VI-F).
// emit_values with the plan's record type, noise switch and clip bound passed as values (callers whose Geom
// sits in shared memory keep them in registers across the record stores).
__device__ __forceinline__ void emit_values_s(int dtype, bool noise_free, float R_f, int C, uint8_t *dst,
                                              const uint32_t *S, uint4 words, float sigma, float b2, float inv_b2,
                                              float *ov) {
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
        if (ch >= C) break;
        if (dtype == DP_PIX_REC_SUM_U32) {
            reinterpret_cast<uint32_t *>(dst)[ch] = S[ch];
            if (ov) ov[ch] = __fdiv_rn(__uint2float_rn(S[ch]), b2);
        } else {
            const float eta = noise_free ? 0.0f : laplace_from_word(word_of(words, ch), sigma);
            const float v = noisy_mean(S[ch], b2, inv_b2, eta, R_f);
            if (dtype == DP_PIX_REC_F32) {
                reinterpret_cast<float *>(dst)[ch] = v;
                if (ov) ov[ch] = v;
            } else {
                const uint32_t q = __float2uint_rn(v);
                dst[ch] = (uint8_t)q;
                if (ov) ov[ch] = (float)q;
            }
        }
    }
}

__device__ __forceinline__ void emit_values(const Geom &g, int C, uint8_t *dst, const uint32_t *S, uint4 words,
                                            float sigma, float b2, float inv_b2, float *ov) {
    emit_values_s(g.dtype, g.noise_free != 0, g.R_f, C, dst, S, words, sigma, b2, inv_b2, ov);
}

// Mirror padding by index: padded index p >= n maps back into [0, n) (Alg. 2 step 4).  Without padding
// (DP_PIX_PAD_NONE) the sample past the edge is not used, and any index inside the frame is returned.
__device__ __forceinline__ int reflect_idx(int p, int n, int pad_mode) {
    if (p < n) return p;
    if (pad_mode == DP_PIX_PAD_NONE) return n - 1;
    return pad_mode == DP_PIX_PAD_REFLECT ? 2 * (n - 1) - p : 2 * n - 1 - p;
}

__device__ __forceinline__ uint64_t align16_u64(uint64_t x) { return (x + 15ull) & ~15ull; }

// Device status word (st[0] = first error code, st[1] = detail), cleared by dp_pix_status().  Kernels get
// its address as an argument; it lives in api.cu.
__device__ __forceinline__ void raise_status(int32_t *st, int32_t code, uint32_t detail) {
    if (st != nullptr && atomicCAS(reinterpret_cast<int *>(st), 0, code) == 0) st[1] = (int32_t)detail;
}

// Bounds-checked build (compiled with DPPIX_CHECKED, libdppix_checked.so): the release, fused, statistics,
// reconstruction and batch kernels check their global accesses of these kinds against the extent of the
// buffer they belong to; an access outside is skipped and raises DP_PIX_E_DEVICE with detail 0x600 | site.
// In the normal build chk() is a constant true and costs nothing.
enum ChkSite : uint32_t { kChkRecord = 1, kChkFrame = 2, kChkWorkspace = 3, kChkOutput = 4 };
#ifdef DPPIX_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
__device__ __forceinline__ bool chk(const void *p, uint64_t n, const void *base, uint64_t extent, int32_t *status,
                                    uint32_t site) {
    if (!kChecked) return true;
    const uintptr_t x = reinterpret_cast<uintptr_t>(p), b = reinterpret_cast<uintptr_t>(base);
    if (x >= b && x - b <= extent && n <= extent - (x - b)) return true;
    raise_status(status, DP_PIX_E_DEVICE, 0x600u | site);
    return false;
}

// Launchers (one per kernel file); return cudaError_t of the launch.
cudaError_t launch_classify(const Geom &g, const CallArgs &a, cudaStream_t s);
cudaError_t launch_finalize_labels(const Geom &g, const CallArgs &a, cudaStream_t s);
cudaError_t launch_finalize_map(const Geom &g, const CallArgs &a, cudaStream_t s);
cudaError_t launch_release(const Geom &g, const CallArgs &a, cudaStream_t s);
cudaError_t launch_tile_stats(const Geom &g, const CallArgs &a, cudaStream_t s);
cudaError_t launch_tile_stats_fast(const Geom &g, const CallArgs &a, cudaStream_t s);  // NotSupported: no instance
cudaError_t launch_rank(const Geom &g, const CallArgs &a, cudaStream_t s);
cudaError_t launch_emit(const Geom &g, const CallArgs &a, cudaStream_t s);
cudaError_t launch_emit_recon(const Geom &g, const CallArgs &a, uint8_t *out, int64_t out_frame_stride,
                              int64_t out_pitch, int out_type, int out_align, int max_per_sm,
                              cudaStream_t s);  // NotSupported: fall back; max_per_sm 0: occupancy limit
cudaError_t launch_reconstruct(const uint8_t *records, int64_t record_stride, uint32_t n, uint8_t *out,
                               int64_t out_frame_stride, int64_t out_pitch, int out_type, int max_M, int max_N,
                               int max_C, int out_align, int32_t *status, cudaStream_t s);
cudaError_t launch_batch_classify(const BatchEntry *tab, uint32_t n_img, uint32_t items, int T, int matte,
                                  cudaStream_t s);
cudaError_t launch_batch_finalize(const BatchEntry *tab, uint32_t n_img, uint32_t max_tiles, cudaStream_t s);
cudaError_t launch_batch_release(const BatchEntry *tab, uint32_t n_img, uint32_t items, int T, int C, int S,
                                 cudaStream_t s);
size_t release_smem(int T, int C, int S);  // dynamic shared memory of the release kernels for S-tile segments
// Whole-warps-per-tile batch release (S-tile segments sharing 8 warps); 0 smem: S does not apply.
size_t batch_tiles_smem(int T, int C, int S);
cudaError_t launch_batch_tiles(const BatchEntry *tab, uint32_t n_img, uint32_t items, int T, int C, int S,
                               cudaStream_t s);
// Streaming batch kernels (k_batch_stream.cu): classification of (image, tile row) items, and the release (with
// the u8 reconstruction when `recon`) of (image, tile row, segment of S tiles) items.
struct BatchStreamShape {
    int S, NB, vpitch, csq, cellv_off, edge_off, edge_pitch, smem, recon_ok;  // S = 0: the streaming release does not apply
};
bool batch_classify_stream_ok(int T, int matte);
cudaError_t launch_batch_classify_stream(const BatchEntry *tab, uint32_t n_img, uint32_t items, int matte,
                                         uint32_t max_gc, cudaStream_t s);
BatchStreamShape batch_release_stream_shape(int T, int C, int b_min, int max_seg);
cudaError_t launch_batch_release_stream(const BatchEntry *tab, uint32_t n_img, uint32_t items, int C,
                                        const BatchStreamShape &bs, int recon, cudaStream_t s);
cudaError_t launch_batch_reconstruct(const BatchEntry *tab, uint32_t n_img, uint32_t items, int out_type, int max_C,
                                     int out_align, int32_t *status, cudaStream_t s);
cudaError_t launch_debug_noise(uint64_t seed, const uint32_t *ctr, uint64_t n, uint32_t *words, float *eta,
                               float sigma, cudaStream_t s);
cudaError_t launch_keys_advance(dp_pix_frame_key *keys, uint32_t n, uint64_t delta, cudaStream_t s);

// An NVTX range for the duration of a library call (host side; profilers such as Nsight show the calls on
// the timeline and can filter kernels by them).  Costs a branch when no profiler is attached.
struct ApiRange {
    explicit ApiRange(const char *name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
    ApiRange(const ApiRange &) = delete;
    ApiRange &operator=(const ApiRange &) = delete;
};
#define DPPIX_RANGE() ::dppix::ApiRange dppix_api_range_(__func__)

// Host-side launch accounting (api.cu).
void prof_begin(const char *name, cudaStream_t s);
void prof_end(const char *name, cudaStream_t s);
int sm_count();
int32_t *status_word();  // device address of the status word on the current device (nullptr on failure)
cudaStream_t *side_streams(int n);  // n (<= 8) non-blocking streams of the current device, or nullptr
int launch_prep(const void *kernel, int threads, size_t smem);  // blocks per SM (cached); raises the smem limit
}  // namespace dppix
struct dp_pix_plan_s;
namespace dppix {
uint64_t plan_ws_per_frame(const dp_pix_plan_s *plan);  // workspace bytes per frame of a plan (0 for NULL)
int set_last_error(int code, const char *msg);          // sets this thread's dp_pix_last_error(), returns code
void clear_last_error();                               // empties this thread's dp_pix_last_error()
int plan_geometry(const dp_pix_desc *d, Geom &g);       // dp_pix_plan's validation and geometry (host)
void set_release_units(Geom &g);                        // release work units for the plan's segment width
int cuda_device_ok();                                   // DP_PIX_OK, or DP_PIX_E_CUDA with the message set

}  // namespace dppix
