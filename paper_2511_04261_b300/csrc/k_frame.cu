// k_frame.cu -- per-frame kernels: region-map finalisation and variance-quantile ranking.
//
// One CTA per frame.  Given the frame's u8 tile -> region map, the CTA counts tiles per region, lays out
// the region-major payload (Table IV: mu'_G then mu'_Gs, generalised to K regions), writes each tile's
// payload byte offset to the workspace, writes the tile-row index and the 512-byte header into the
// record.  The rank kernel first builds the map from the per-tile variance keys (exact integers) by a
// bitonic sort of (key, tile index) in shared memory.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace dppix {

namespace {

constexpr int kFrameThreads = 1024;

// Exclusive scan of kMaxK counters per thread across the block.  warp_tot: smem [32][kMaxK].
__device__ void block_excl_scan_k(uint32_t (&v)[kMaxK], uint32_t (&excl)[kMaxK], uint32_t (&total)[kMaxK],
                                  uint32_t (*warp_tot)[kMaxK]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
    uint32_t incl[kMaxK];
#pragma unroll
    for (int r = 0; r < kMaxK; ++r) incl[r] = v[r];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
        for (int r = 0; r < kMaxK; ++r) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl[r], off);
            if (lane >= off) incl[r] += t;
        }
    }
    if (lane == 31) {
#pragma unroll
        for (int r = 0; r < kMaxK; ++r) warp_tot[warp][r] = incl[r];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int r = 0; r < kMaxK; ++r) {
            uint32_t x = lane < nwarps ? warp_tot[lane][r] : 0u;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, x, off);
                if (lane >= off) x += t;
            }
            if (lane < nwarps) warp_tot[lane][r] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kMaxK; ++r) {
        const uint32_t base = warp > 0 ? warp_tot[warp - 1][r] : 0u;
        excl[r] = base + incl[r] - v[r];
        total[r] = warp_tot[nwarps - 1][r];
    }
    __syncthreads();
}

struct FinalizeSmem {
    uint32_t warp_tot[32][kMaxK];
    uint64_t roff[kMaxK];
    uint64_t tile_bytes[kMaxK];
    uint32_t count[kMaxK];
    uint32_t tstart[kMaxK];  // first position of region r's tiles in the region-ordered tile list
    dp_pix_record_header hdr;
};

// Lays out the record of frame f from the map in shared memory (see file comment); also writes the
// workspace's per-tile payload offsets and the tile ids in record order (region-major, row-major).
__device__ void finalize_frame(const Geom &g, const CallArgs &a, uint32_t f, const uint8_t *map_s, bool write_map,
                               FinalizeSmem &sm) {
    const uint32_t n = g.ntiles;
    const uint32_t chunk = (n + blockDim.x - 1) / blockDim.x;
    const uint32_t c0 = min(n, threadIdx.x * chunk), c1 = min(n, c0 + chunk);
    uint32_t cnt[kMaxK], excl[kMaxK], total[kMaxK];
#pragma unroll
    for (int r = 0; r < kMaxK; ++r) cnt[r] = 0;
    for (uint32_t i = c0; i < c1; ++i) {
        const uint32_t r = map_s[i];
#pragma unroll
        for (int q = 0; q < kMaxK; ++q) cnt[q] += (r == (uint32_t)q);
    }
    block_excl_scan_k(cnt, excl, total, sm.warp_tot);

    uint8_t *rec = a.records + (uint64_t)f * (uint64_t)a.record_stride;
    if (threadIdx.x == 0) {
        uint64_t off = g.payload_offset;
        uint32_t tacc = 0;
        for (int r = 0; r < g.K; ++r) {
            const uint64_t cs = (uint64_t)g.cells_side[r];
            sm.tile_bytes[r] = cs * cs * (uint64_t)g.C * (uint64_t)g.es;
            sm.roff[r] = off;
            sm.count[r] = total[r];
            sm.tstart[r] = tacc;
            tacc += total[r];
            off = align16_u64(off + (uint64_t)total[r] * sm.tile_bytes[r]);
        }
        dp_pix_record_header &h = sm.hdr;
        memset(&h, 0, sizeof(h));
        h.magic[0] = 'D'; h.magic[1] = 'P'; h.magic[2] = 'P'; h.magic[3] = 'X';
        h.version = 1;
        h.header_bytes = kHeaderBytes;
        h.flags = g.noise_free ? 1u : 0u;
        h.M = g.M; h.N = g.N; h.C = g.C; h.T = g.T; h.K = g.K; h.GR = g.GR; h.GC = g.GC;
        if (key_stream(a, f) >= (1u << 24)) raise_status(a.status, DP_PIX_E_DEVICE, 0x400u | (f & 0xFFu));
        h.pad_mode = g.pad_mode; h.record_dtype = g.dtype; h.region_source = g.source; h.stream_id = key_stream(a, f);
        h.seed = g.seed;
        h.frame_idx = key_frame(a, f);
        h.value_range = g.R; h.m = g.m;
        h.total_bytes = off;
        h.map_offset = g.map_offset;
        for (int r = 0; r < g.K; ++r) {
            h.grid[r] = g.grid[r];
            h.eps[r] = g.eps[r];
            h.sigma[r] = g.sigma[r];
            h.count[r] = total[r];
            h.region_offset[r] = sm.roff[r];
        }
        h.rowidx_offset = g.rowidx_offset;
        h.payload_offset = g.payload_offset;
    }
    __syncthreads();
    // header out: 32 x 16 bytes
    if (threadIdx.x < kHeaderBytes / 16)
        reinterpret_cast<uint4 *>(rec)[threadIdx.x] = reinterpret_cast<const uint4 *>(&sm.hdr)[threadIdx.x];
    // per-tile offsets and tile-row index
    uint32_t *tileoff = reinterpret_cast<uint32_t *>(a.ws + (uint64_t)f * g.ws_per_frame + g.ws_tileoff);
    uint32_t *rowidx = reinterpret_cast<uint32_t *>(rec + g.rowidx_offset);
    uint32_t *tilelist = reinterpret_cast<uint32_t *>(a.ws + (uint64_t)f * g.ws_per_frame + g.ws_tilelist);
    uint32_t run[kMaxK];
#pragma unroll
    for (int r = 0; r < kMaxK; ++r) run[r] = excl[r];
    for (uint32_t i = c0; i < c1; ++i) {
        if (i % (uint32_t)g.GC == 0) {
            const uint32_t ty = i / (uint32_t)g.GC;
#pragma unroll
            for (int r = 0; r < kMaxK; ++r)
                if (r < g.K) rowidx[ty * g.K + r] = run[r];
        }
        const uint32_t r = map_s[i];
        uint32_t ri = 0;
#pragma unroll
        for (int q = 0; q < kMaxK; ++q)
            if (r == (uint32_t)q) { ri = run[q]; run[q] = ri + 1; }
        tileoff[i] = (uint32_t)(sm.roff[r] + (uint64_t)ri * sm.tile_bytes[r]);
        tilelist[sm.tstart[r] + ri] = i;  // tiles in record (payload) order
    }
    if (write_map) {
        uint8_t *map = rec + g.map_offset;
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) map[i] = map_s[i];
    }
    // zero the alignment gaps so that a record is a deterministic byte string
    const uint64_t row_end = g.rowidx_offset + (uint64_t)g.GR * g.K * 4;
    for (uint64_t i = row_end + threadIdx.x; i < g.map_offset; i += blockDim.x) rec[i] = 0;
    for (uint64_t i = g.map_offset + n + threadIdx.x; i < g.payload_offset; i += blockDim.x) rec[i] = 0;
    if (threadIdx.x < (unsigned)g.K) {
        const int r = threadIdx.x;
        const uint64_t end = sm.roff[r] + (uint64_t)sm.count[r] * sm.tile_bytes[r];
        for (uint64_t i = end; i < align16_u64(end); ++i) rec[i] = 0;
    }
}

// Map given by the caller (tile labels) or already written into the record by k_classify.
__global__ void __launch_bounds__(kFrameThreads) k_finalize(const Geom g, const CallArgs a, int from_labels) {
    extern __shared__ __align__(16) uint8_t dyn[];
    FinalizeSmem &sm = *reinterpret_cast<FinalizeSmem *>(dyn);
    uint8_t *map_s = dyn + sizeof(FinalizeSmem);
    const uint32_t f = blockIdx.x;
    const uint8_t *src = from_labels ? a.src + (uint64_t)f * (uint64_t)a.src_frame_stride
                                     : a.records + (uint64_t)f * (uint64_t)a.record_stride + g.map_offset;
    for (uint32_t i = threadIdx.x; i < g.ntiles; i += blockDim.x) {
        uint8_t r = src[i];
        if (r >= (uint32_t)g.K) {
            raise_status(a.status, DP_PIX_E_DEVICE, 0x100u | r);
            r = 0;
        }
        map_s[i] = r;
    }
    __syncthreads();
    finalize_frame(g, a, f, map_s, from_labels != 0, sm);
}

// Batch: one CTA per image (map written by k_batch_classify, or caller labels).
__global__ void __launch_bounds__(kFrameThreads) k_batch_finalize(const BatchEntry *tab, uint32_t n_img) {
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ BatchShared bs;
    FinalizeSmem &sm = *reinterpret_cast<FinalizeSmem *>(dyn);
    uint8_t *map_s = dyn + sizeof(FinalizeSmem);
    for (uint32_t i = blockIdx.x; i < n_img; i += gridDim.x) {
        batch_load(tab, (int)i, bs);
        const Geom &g = bs.g;
        const CallArgs &a = bs.a;
        const bool from_labels = g.source == DP_PIX_SRC_TILE_LABELS;
        const uint8_t *src = from_labels ? a.src : a.records + g.map_offset;
        for (uint32_t t = threadIdx.x; t < g.ntiles; t += blockDim.x) {
            uint8_t r = src[t];
            if (r >= (uint32_t)g.K) {
                raise_status(a.status, DP_PIX_E_DEVICE, 0x100u | r);
                r = 0;
            }
            map_s[t] = r;
        }
        __syncthreads();
        finalize_frame(g, a, 0u, map_s, from_labels, sm);
        __syncthreads();
    }
}

// VARIANCE classes: tiles ranked by (key, index) ascending get class q = floor(K * rank / n).  Only the
// K - 1 class boundaries matter: the tile of rank ceil(q n / K) starts class q.  Each boundary value is
// found exactly by a radix select over the unique packed values key << idx_bits | index (8-bit digits from
// the top); a tile's class is then the number of boundaries not above its value.
__global__ void __launch_bounds__(kFrameThreads) k_rank(const Geom g, const CallArgs a) {
    extern __shared__ __align__(16) uint8_t dyn[];
    FinalizeSmem &sm = *reinterpret_cast<FinalizeSmem *>(dyn);
    const uint32_t f = blockIdx.x, n = g.ntiles;
    uint64_t *vals = reinterpret_cast<uint64_t *>(dyn + sizeof(FinalizeSmem));
    uint8_t *map_s = reinterpret_cast<uint8_t *>(vals + n);
    __shared__ uint32_t hist[kMaxK - 1][256];
    __shared__ uint64_t prefix[kMaxK - 1];
    __shared__ uint32_t target[kMaxK - 1];
    const int Q = g.K - 1;
    const uint64_t *keys = reinterpret_cast<const uint64_t *>(a.ws + (uint64_t)f * g.ws_per_frame + g.ws_keys);
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) vals[i] = (keys[i] << g.idx_bits) | (uint64_t)i;
    if ((int)threadIdx.x < Q) {
        prefix[threadIdx.x] = 0ull;
        target[threadIdx.x] = (uint32_t)(((uint64_t)(threadIdx.x + 1) * n + g.K - 1) / g.K);  // 0-based rank
    }
    __syncthreads();
    const int passes = Q > 0 ? (g.val_bits + 7) / 8 : 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * (passes - 1 - pass);
        for (int i = threadIdx.x; i < Q * 256; i += blockDim.x) hist[i >> 8][i & 255] = 0u;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
            const uint64_t v = vals[i];
            const uint64_t hi = shift + 8 >= 64 ? 0ull : v >> (shift + 8);
            const uint32_t d = (uint32_t)(v >> shift) & 255u;
            for (int q = 0; q < Q; ++q)
                if (hi == prefix[q]) atomicAdd(&hist[q][d], 1u);
        }
        __syncthreads();
        if (warp < Q) {  // warp q finds the digit bucket that holds its target rank
            uint32_t c[8], sum = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                c[j] = hist[warp][8 * lane + j];
                sum += c[j];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += t;
            }
            const uint32_t excl = incl - sum, t = target[warp];
            if (excl <= t && t < incl) {
                uint32_t acc = excl;
                int j = 0;
                while (j < 7 && acc + c[j] <= t) acc += c[j++];
                prefix[warp] = (prefix[warp] << 8) | (uint64_t)(8 * lane + j);
                target[warp] = t - acc;
            }
        }
        __syncthreads();
    }
    const uint64_t mask = (1ull << g.idx_bits) - 1ull;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint64_t v = vals[i];
        int cls = 0;
        for (int q = 0; q < Q; ++q) cls += v >= prefix[q] ? 1 : 0;
        map_s[v & mask] = (uint8_t)cls;
    }
    __syncthreads();
    finalize_frame(g, a, f, map_s, true, sm);
}

}  // namespace

cudaError_t launch_finalize_labels(const Geom &g, const CallArgs &a, cudaStream_t s) {
    const size_t smem = sizeof(FinalizeSmem) + g.ntiles;
    launch_prep(reinterpret_cast<const void *>(k_finalize), kFrameThreads, smem);
    prof_begin("k_finalize", s);
    k_finalize<<<a.n_frames, kFrameThreads, smem, s>>>(g, a, 1);
    prof_end("k_finalize", s);
    return cudaGetLastError();
}

cudaError_t launch_finalize_map(const Geom &g, const CallArgs &a, cudaStream_t s) {
    const size_t smem = sizeof(FinalizeSmem) + g.ntiles;
    launch_prep(reinterpret_cast<const void *>(k_finalize), kFrameThreads, smem);
    prof_begin("k_finalize", s);
    k_finalize<<<a.n_frames, kFrameThreads, smem, s>>>(g, a, 0);
    prof_end("k_finalize", s);
    return cudaGetLastError();
}

cudaError_t launch_batch_finalize(const BatchEntry *tab, uint32_t n_img, uint32_t max_tiles, cudaStream_t s) {
    const size_t smem = sizeof(FinalizeSmem) + max_tiles;
    launch_prep(reinterpret_cast<const void *>(k_batch_finalize), kFrameThreads, smem);
    const int grid = (int)std::min<uint32_t>(n_img, (uint32_t)sm_count());
    prof_begin("k_batch_finalize", s);
    k_batch_finalize<<<grid, kFrameThreads, smem, s>>>(tab, n_img);
    prof_end("k_batch_finalize", s);
    return cudaGetLastError();
}

cudaError_t launch_rank(const Geom &g, const CallArgs &a, cudaStream_t s) {
    const size_t smem = sizeof(FinalizeSmem) + (size_t)g.ntiles * 8 + g.ntiles;
    launch_prep(reinterpret_cast<const void *>(k_rank), kFrameThreads, smem);
    prof_begin("k_rank", s);
    k_rank<<<a.n_frames, kFrameThreads, smem, s>>>(g, a);
    prof_end("k_rank", s);
    return cudaGetLastError();
}

}  // namespace dppix
