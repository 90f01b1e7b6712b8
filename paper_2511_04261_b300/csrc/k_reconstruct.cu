// k_reconstruct.cu -- rebuild pixelized frames from their records alone (Sec. VI-F; Alg. 2 steps 10-11).
//
// Geometry comes from each record's header on the device, so one launch serves any mix of records.
// Work item = (record, tile row, segment of tiles).  Every pixel of a cell takes the cell's stored value
// (u8 output rounds half to even); rows and columns past M, N (the padding) are cropped.
//
// Fast path (records with the launch's channel count): the segment -- a whole tile row when it fits -- has
// its cell values converted once into shared memory; each thread owns 16-byte columns of the output rows and
// assembles its vector from the cells it covers.  With 16-byte aligned rows the same vector is stored to
// every row of the current cell band before it is rebuilt; rows of any other alignment get their aligned
// middle in 16-byte chunks built per row and their head and tail one element at a time.
// Generic path (anything else): the CTA builds each distinct output row in shared memory and copies it out
// with the widest aligned stores.
#include <algorithm>

#include "seg_write.cuh"

namespace dppix {
namespace {

constexpr int kThreads = 256;
constexpr int kRowBytes = 2048;     // generic path: shared-memory row pattern
constexpr int kStageBytes = 24576;  // fast path: staged cell values of one segment
constexpr int kMaxSegPx = kSegMaxPx;
constexpr int kMaxSegTiles = kSegMaxTiles;
// Bytes of one row-pattern buffer of the u8 writer for rows of any alignment (C channels).
__host__ __device__ constexpr int pat_stride(int C) { return 16 * (kMaxSegPx * C / 16 + 1); }

// Dynamic shared memory of the fast path: stage | colinfo | two row patterns (u8 rows of any alignment).
__host__ __device__ constexpr size_t fast_smem(int out_f32, int fast_c, int out_align) {
    return (size_t)kStageBytes + colinfo_words(kMaxSegPx) * 4 +
           (!out_f32 && fast_c > 0 && out_align != 16 ? 2 * (size_t)pat_stride(fast_c) : 0);
}

struct RecGeom {
    int32_t ok, fast;
    int32_t M, N, C, T, K, GR, GC, dtype, es, SR, nseg;
    int32_t grid[kMaxK];
    uint32_t count[kMaxK];
    uint64_t map_offset, rowidx_offset;
    uint64_t region_offset[kMaxK];
};

__device__ __forceinline__ int gcd_i(int a, int b) {
    while (b) {
        const int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Checks a record header (a shared-memory copy): geometry within the caller's bounds, and every section
// (tile-row index, map, region payloads) inside total_bytes <= cap, so that no later read leaves the
// record.  Chooses the fast path when the record has fast_C channels, output rows are 16-byte aligned,
// and a segment's cell values fit the staging buffer.
__device__ bool read_header(const dp_pix_record_header *h, uint64_t cap, int max_M, int max_N, int max_C, RecGeom &rg,
                            int oes, int fast_C, int out_align) {
    if (h->magic[0] != 'D' || h->magic[1] != 'P' || h->magic[2] != 'P' || h->magic[3] != 'X' || h->version != 1)
        return false;
    rg.M = (int)h->M; rg.N = (int)h->N; rg.C = (int)h->C; rg.T = (int)h->T; rg.K = (int)h->K;
    rg.GR = (int)h->GR; rg.GC = (int)h->GC; rg.dtype = (int)h->record_dtype;
    if (rg.M < 1 || rg.N < 1 || rg.M > max_M || rg.N > max_N || rg.C < 1 || rg.C > max_C || rg.C > 4) return false;
    if (rg.T < 1 || rg.T > kMaxT || rg.K < 1 || rg.K > kMaxK || rg.dtype < 0 || rg.dtype > 2) return false;
    if (rg.GR != (rg.M + rg.T - 1) / rg.T || rg.GC != (rg.N + rg.T - 1) / rg.T) return false;
    const uint64_t total = h->total_bytes;
    if (total > cap) return false;
    rg.es = rg.dtype == DP_PIX_REC_U8 ? 1 : 4;
    int bmin = rg.T;
    for (int r = 0; r < rg.K; ++r) {
        rg.grid[r] = (int)h->grid[r];
        rg.count[r] = h->count[r];
        rg.region_offset[r] = h->region_offset[r];
        if (rg.grid[r] < 1 || rg.T % rg.grid[r] != 0) return false;
        const uint64_t cs = (uint64_t)(rg.T / rg.grid[r]);
        if (rg.region_offset[r] > total || (uint64_t)rg.count[r] * cs * cs * rg.C * rg.es > total - rg.region_offset[r])
            return false;
        bmin = rg.grid[r] < bmin ? rg.grid[r] : bmin;
    }
    rg.map_offset = h->map_offset;
    rg.rowidx_offset = h->rowidx_offset;
    const uint64_t ntiles = (uint64_t)rg.GR * rg.GC;
    if (rg.map_offset > total || ntiles > total - rg.map_offset) return false;
    if (rg.rowidx_offset > total || (uint64_t)rg.GR * rg.K * 4 > total - rg.rowidx_offset || rg.rowidx_offset % 4)
        return false;
    rg.fast = 0;
    const int trb = rg.T * rg.C * oes;  // bytes of one tile row of output
    if (rg.C == fast_C && (out_align == 16 || oes == 1 || out_align >= 4) && trb >= 16) {
        // S tiles per segment, S a multiple of s0 so that segment starts stay 16-byte aligned, and as many
        // tiles as the staging buffers take (a whole tile row of a 1080p frame)
        const int s0 = 16 / gcd_i(trb, 16);
        const int csmax = rg.T / bmin;
        const int vb = oes == 4 ? 16 : 4;  // staged bytes per cell
        int S = min(kMaxSegTiles, ((rg.GC + s0 - 1) / s0) * s0) / s0 * s0;
        while (S > 0 && ((int64_t)S * csmax * csmax * vb > kStageBytes || S * rg.T > kMaxSegPx)) S -= s0;
        if (S > 0) {
            rg.fast = 1;
            rg.SR = S;
        }
    }
    if (!rg.fast) {
        const int sr = kRowBytes / trb;
        rg.SR = sr < 1 ? 1 : (sr > 16 ? 16 : sr);
    }
    rg.nseg = (rg.GC + rg.SR - 1) / rg.SR;
    return true;
}

// Stored value of one (cell, channel) as the output element's float.
__device__ __forceinline__ float record_value(const uint8_t *src, int dtype, int b) {
    if (dtype == DP_PIX_REC_F32) return *reinterpret_cast<const float *>(src);
    if (dtype == DP_PIX_REC_U8) return (float)*src;
    return __fdiv_rn(__uint2float_rn(*reinterpret_cast<const uint32_t *>(src)), (float)(b * b));
}


// Tile table of the segment [tx0, tx0 + ns) of tile row ty: region, grid, payload offset.  The number of
// region-r tiles before the segment comes from the record's tile-row index plus a block-parallel count
// over the map row, so no thread walks the row alone.
__device__ void seg_tile_info(const uint8_t *rec, const RecGeom &rg, int ty, int tx0, int ns, uint32_t rec_i,
                              int32_t *status, SegTiles &st, uint32_t *cnt_s) {
    const uint8_t *maprow = rec + rg.map_offset + (uint64_t)ty * rg.GC;
    if (threadIdx.x < kMaxK) cnt_s[threadIdx.x] = 0u;
    if (threadIdx.x < ns) {
        const int r = maprow[tx0 + threadIdx.x];
        st.reg[threadIdx.x] = r < rg.K ? r : 0;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < tx0; x += blockDim.x) {
        const int r = maprow[x];
        if (r < rg.K) atomicAdd(&cnt_s[r], 1u);
    }
    __syncthreads();
    if (threadIdx.x < ns) {
        const int t = threadIdx.x;
        const int r = st.reg[t];
        uint32_t before = reinterpret_cast<const uint32_t *>(rec + rg.rowidx_offset)[ty * rg.K + r] + cnt_s[r];
        for (int x = 0; x < t; ++x) before += (st.reg[x] == r);  // the segment's region ids, in shared memory
        int b = rg.grid[r], cs = rg.T / b;
        uint64_t off = rg.region_offset[r] + (uint64_t)before * (uint64_t)(cs * cs * rg.C * rg.es);
        if (before >= rg.count[r]) {  // inconsistent index: read the header instead of leaving the record
            raise_status(status, DP_PIX_E_DEVICE, 0x300u | (rec_i & 0xFFu));
            b = rg.T;
            cs = 1;
            off = 0;
        }
        st.b[t] = b;
        st.cs[t] = cs;
        st.off[t] = off;
    }
    __syncthreads();
}

template <int C, int kOutF32>
__device__ void fast_item(const uint8_t *rec, const RecGeom &rg, uint32_t rec_i, int ty, int sg, uint8_t *obase,
                          int64_t out_pitch, int out_align, uint8_t *stage, uint32_t *colinfo, uint8_t *pat,
                          SegTiles &st, uint32_t *cnt_s, int32_t *status) {
    constexpr int oes = kOutF32 ? 4 : 1;
    const int T = rg.T;
    const int tx0 = sg * rg.SR;
    const int ns = min(rg.SR, rg.GC - tx0);
    seg_tile_info(rec, rg, ty, tx0, ns, rec_i, status, st, cnt_s);
    seg_prefix_colinfo(st, ns, T, colinfo, threadIdx.x, blockDim.x);
    if (!kOutF32 && out_align != 16) seg_row_groups(st, ns, T, threadIdx.x);
    __syncthreads();
    // cell values of the segment, converted once
    const int ncell = st.base[ns];
    for (int e = threadIdx.x; e < ncell; e += blockDim.x) {
        int lo = 0, hi = ns - 1;  // last tile with base <= e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (st.base[mid] <= e) lo = mid; else hi = mid - 1;
        }
        const int t = lo;
        const int c = e - st.base[t];
        const uint8_t *src = rec + st.off[t] + (uint64_t)c * C * rg.es;
        if (kOutF32) {
            float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ch = 0; ch < C; ++ch) v[ch] = record_value(src + ch * rg.es, rg.dtype, st.b[t]);
            reinterpret_cast<float4 *>(stage)[e] = make_float4(v[0], v[1], v[2], v[3]);
        } else {
            uint32_t pk = 0;
#pragma unroll
            for (int ch = 0; ch < C; ++ch) pk |= to_u8(record_value(src + ch * rg.es, rg.dtype, st.b[t])) << (8 * ch);
            reinterpret_cast<uint32_t *>(stage)[e] = pk;
        }
    }
    __syncthreads();
    // write phase: no barrier until the next item
    const int x0 = tx0 * T;
    uint8_t *orow0 = obase + (int64_t)(ty * T) * out_pitch + (int64_t)x0 * C * oes;
    if (out_align == 16)
        seg_write_rows<C, kOutF32>(st, colinfo, stage, ns, T, min(ns * T, rg.N - x0), min(T, rg.M - ty * T), orow0,
                                   out_pitch, threadIdx.x, blockDim.x, obase,
                                   (uint64_t)(rg.M - 1) * (uint64_t)out_pitch + (uint64_t)rg.N * C * oes, status);
    else if (!kOutF32)
        seg_write_rows_pat<C>(st, colinfo, stage, ns, T, min(ns * T, rg.N - x0), min(T, rg.M - ty * T), orow0,
                              out_pitch, pat, pat_stride(C), threadIdx.x, blockDim.x, obase,
                              (uint64_t)(rg.M - 1) * (uint64_t)out_pitch + (uint64_t)rg.N * C, status);
    else
        seg_write_rows_any<C, kOutF32>(st, colinfo, stage, ns, T, min(ns * T, rg.N - x0), min(T, rg.M - ty * T),
                                       orow0, out_pitch, threadIdx.x, blockDim.x);
    __syncthreads();
}

// ---- generic path ------------------------------------------------------------------------------------
template <int kOutF32>
__device__ void generic_item(const uint8_t *rec, const RecGeom &rg, uint32_t rec_i, int ty, int sg, uint8_t *obase,
                             int64_t out_pitch, int out_align, uint8_t *rowpat, SegTiles &st, uint32_t *cnt_s,
                             int32_t *status) {
    constexpr int oes = kOutF32 ? 4 : 1;
    const int T = rg.T, C = rg.C, es = rg.es;
    const int tx0 = sg * rg.SR;
    const int ns = min(rg.SR, rg.GC - tx0);
    seg_tile_info(rec, rg, ty, tx0, ns, rec_i, status, st, cnt_s);
    const int x0 = tx0 * T;
    const int vpx = min(ns * T, rg.N - x0);
    const int row_bytes = vpx * C * oes;
    uint8_t *orow0 = obase + (uint64_t)x0 * C * oes;
    // widest unit that keeps every row segment start aligned
    int U = out_align;
    while (U > 1 && (((int64_t)rg.SR * T * C * oes) % U != 0)) U >>= 1;
    if (U == 2) U = 1;  // copies move 16, 8, 4 or 1 bytes
    const int nu = row_bytes / U;
    const int tail0 = nu * U;
    const int jmax = min(T, rg.M - ty * T);
    int j = 0;
    while (j < jmax) {
        // next row where some tile enters a new cell band
        int jn = jmax;
        for (int t = 0; t < ns; ++t) {
            const int nb = (j / st.b[t] + 1) * st.b[t];
            jn = min(jn, nb);
        }
        // build the row pattern of rows [j, jn)
        const int elems = ns * T * C;
        for (int e = threadIdx.x; e < elems; e += blockDim.x) {
            const int t = e / (T * C);
            const int rem = e - t * (T * C);
            const int px = rem / C, ch = rem - px * C;
            const int b = st.b[t], cs = st.cs[t];
            const int cell = (j / b) * cs + px / b;
            const float v = record_value(rec + st.off[t] + ((uint64_t)cell * C + ch) * es, rg.dtype, b);
            if (kOutF32)
                reinterpret_cast<float *>(rowpat)[e] = v;
            else
                rowpat[e] = (uint8_t)to_u8(v);
        }
        __syncthreads();
        const int rows = jn - j;
        const int per_row = nu + (row_bytes - tail0);
        for (int q = threadIdx.x; q < rows * per_row; q += blockDim.x) {
            const int rr = q / per_row, u = q - rr * per_row;
            uint8_t *orow = orow0 + (int64_t)(ty * T + j + rr) * out_pitch;
            if (u < nu) {
                const int o = u * U;
                if (U == 16)
                    *reinterpret_cast<uint4 *>(orow + o) = *reinterpret_cast<const uint4 *>(rowpat + o);
                else if (U == 8)
                    *reinterpret_cast<uint2 *>(orow + o) = *reinterpret_cast<const uint2 *>(rowpat + o);
                else if (U == 4)
                    *reinterpret_cast<uint32_t *>(orow + o) = *reinterpret_cast<const uint32_t *>(rowpat + o);
                else
                    orow[o] = rowpat[o];
            } else {
                const int o = tail0 + (u - nu);
                orow[o] = rowpat[o];
            }
        }
        __syncthreads();
        j = jn;
    }
}

// kFastC: channel count served by the fast path in this launch (0: generic only).
// CTAs are dealt to records: with n <= gridDim records each record gets gridDim / n CTAs that split its
// work items into contiguous runs; with more records than CTAs, CTA c takes records c, c + gridDim, ...
// Each CTA parses a record header once (one parallel 512-byte copy into shared memory).
template <int kOutF32, int kFastC>
__global__ void __launch_bounds__(kThreads)
    k_reconstruct(const uint8_t *records, int64_t record_stride, uint32_t n, uint8_t *out, int64_t out_frame_stride,
                  int64_t out_pitch, int max_M, int max_N, int max_C, int out_align, int32_t *status) {
    extern __shared__ __align__(16) uint8_t dyn[];  // fast path: stage | colinfo | two row patterns
    __shared__ __align__(16) uint8_t rowpat[kRowBytes];
    __shared__ __align__(16) dp_pix_record_header hdr_s;
    __shared__ RecGeom rg;
    __shared__ SegTiles st;
    __shared__ uint32_t cnt_s[kMaxK];
    constexpr int oes = kOutF32 ? 4 : 1;
    uint8_t *stage = dyn;
    uint32_t *colinfo = reinterpret_cast<uint32_t *>(dyn + kStageBytes);
    uint8_t *pat = dyn + kStageBytes + colinfo_words(kMaxSegPx) * 4;
    const uint32_t G = gridDim.x;
    const uint32_t per_rec = n <= G ? G / n : 1u;  // CTAs per record
    const uint32_t slots = n <= G ? n : G;         // records handled concurrently
    if (blockIdx.x >= per_rec * slots) return;     // spare CTAs (whole block)
    const uint32_t sub = blockIdx.x / slots, slot = blockIdx.x % slots;
    for (uint32_t i = slot; i < n; i += slots) {
        const uint8_t *rec = records + (uint64_t)i * (uint64_t)record_stride;
        if (threadIdx.x < kHeaderBytes / 16)
            reinterpret_cast<uint4 *>(&hdr_s)[threadIdx.x] = reinterpret_cast<const uint4 *>(rec)[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) {
            rg.ok = read_header(&hdr_s, (uint64_t)record_stride, max_M, max_N, max_C, rg, oes, kFastC, out_align) ? 1
                                                                                                                  : 0;
            if (!rg.ok && sub == 0) raise_status(status, DP_PIX_E_DEVICE, 0x200u | (i & 0xFFu));
        }
        __syncthreads();
        if (rg.ok) {
            const uint64_t items = (uint64_t)rg.GR * rg.nseg;
            const uint64_t chunk = (items + per_rec - 1) / per_rec;
            const uint64_t k0 = (uint64_t)sub * chunk, k1 = min(items, k0 + chunk);
            uint8_t *obase = out + (uint64_t)i * (uint64_t)out_frame_stride;
            for (uint64_t k = k0; k < k1; ++k) {
                const int ty = (int)(k / rg.nseg), sg = (int)(k - (uint64_t)ty * rg.nseg);
                if (kFastC > 0 && rg.fast)
                    fast_item<(kFastC > 0 ? kFastC : 1), kOutF32>(rec, rg, i, ty, sg, obase, out_pitch, out_align, stage, colinfo,
                                                                   pat, st, cnt_s, status);
                else
                    generic_item<kOutF32>(rec, rg, i, ty, sg, obase, out_pitch, out_align, rowpat, st, cnt_s, status);
            }
        }
        __syncthreads();
    }
}

// Batch: one item per (image, tile row), image i owning [base[3], base[3] + GR); the record and the output of
// each image come from the batch table, and its header is parsed when a CTA moves to a new image.
// Tile rows per chunk: 1.  Images are in largest-first order and a tile row's work grows with the image width,
// so single rows dealt round-robin balance the CTAs best (256-portrait batch: 1.71 ms, against 2.00 and 2.85 ms
// with chunks of 4 and 16 rows).
constexpr uint32_t kRecChunk = 1;
template <int kOutF32, int kFastC>
__global__ void __launch_bounds__(kThreads)
    k_batch_reconstruct(const BatchEntry *tab, uint32_t n_img, uint32_t items, int max_C, int out_align,
                        int32_t *status) {
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ __align__(16) uint8_t rowpat[kRowBytes];
    __shared__ __align__(16) dp_pix_record_header hdr_s;
    __shared__ RecGeom rg;
    __shared__ SegTiles st;
    __shared__ uint32_t cnt_s[kMaxK];
    constexpr int oes = kOutF32 ? 4 : 1;
    uint8_t *stage = dyn;
    uint32_t *colinfo = reinterpret_cast<uint32_t *>(dyn + kStageBytes);
    uint8_t *pat = dyn + kStageBytes + colinfo_words(kMaxSegPx) * 4;
    // chunks of q consecutive tile rows dealt round-robin; a CTA parses a header only when its image changes
    const uint32_t share = (items + gridDim.x - 1) / gridDim.x;
    const uint32_t q = share < kRecChunk ? (share ? share : 1u) : kRecChunk;
    auto next_item = [&](uint32_t it) -> uint32_t {
        const uint64_t n = (it + 1) % q ? (uint64_t)it + 1 : (uint64_t)it + 1 + (uint64_t)(gridDim.x - 1) * q;
        return n < items ? (uint32_t)n : items;
    };
    int cur = -1;
    uint32_t lo = 0, hi = 0;  // items of image cur
    for (uint32_t item = (uint64_t)blockIdx.x * q < items ? blockIdx.x * q : items; item < items;
         item = next_item(item)) {
        const int i = (cur >= 0 && item >= lo && item < hi) ? cur : batch_find(tab, n_img, item, 3);
        const BatchEntry &e = tab[i];
        const uint8_t *rec = e.a.records;
        if (i != cur) {
            __syncthreads();
            if (threadIdx.x < kHeaderBytes / 16)
                reinterpret_cast<uint4 *>(&hdr_s)[threadIdx.x] = reinterpret_cast<const uint4 *>(rec)[threadIdx.x];
            __syncthreads();
            if (threadIdx.x == 0) {
                rg.ok = read_header(&hdr_s, e.rec_cap, e.g.M, e.g.N, max_C, rg, oes, kFastC, out_align) ? 1 : 0;
                if (!rg.ok) raise_status(status, DP_PIX_E_DEVICE, 0x300u | ((uint32_t)i & 0xFFu));
            }
            __syncthreads();
            cur = i;
            lo = e.base[3];
            hi = i + 1 < (int)n_img ? tab[i + 1].base[3] : items;
        }
        if (!rg.ok || e.out == nullptr) continue;
        const int ty = (int)(item - e.base[3]);
        if (ty >= rg.GR) continue;
        for (int sg = 0; sg < rg.nseg; ++sg) {
            if (kFastC > 0 && rg.fast)
                fast_item<(kFastC > 0 ? kFastC : 1), kOutF32>(rec, rg, (uint32_t)i, ty, sg, e.out, e.out_pitch, out_align, stage,
                                                               colinfo, pat, st, cnt_s, status);
            else
                generic_item<kOutF32>(rec, rg, (uint32_t)i, ty, sg, e.out, e.out_pitch, out_align, rowpat, st, cnt_s,
                                      status);
        }
    }
}

template <int kOutF32, int kFastC>
cudaError_t launch_brc(const BatchEntry *tab, uint32_t n_img, uint32_t items, int max_C, int out_align,
                       int32_t *status, cudaStream_t s) {
    const size_t smem = fast_smem(kOutF32, kFastC, out_align);
    auto kern = k_batch_reconstruct<kOutF32, kFastC>;
    const int per_sm = launch_prep(reinterpret_cast<const void *>(kern), kThreads, smem);
    const int grid = (int)std::min<uint64_t>(items, (uint64_t)per_sm * sm_count());
    const char *name = kOutF32 ? "k_batch_reconstruct_f32" : "k_batch_reconstruct_u8";
    prof_begin(name, s);
    kern<<<grid, kThreads, smem, s>>>(tab, n_img, items, max_C, out_align, status);
    prof_end(name, s);
    return cudaGetLastError();
}

// Adds delta to the frame index of each of n keys (stream ids unchanged).
__global__ void k_keys_advance(dp_pix_frame_key *keys, uint32_t n, uint64_t delta) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) keys[i].frame_idx += delta;
}

__global__ void k_debug_noise(uint64_t seed, const uint32_t *ctr, uint64_t n, uint32_t *words, float *eta, float sigma) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
        const uint4 w = philox4x32_10(c, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
        if (words) {
            words[4 * i] = w.x; words[4 * i + 1] = w.y; words[4 * i + 2] = w.z; words[4 * i + 3] = w.w;
        }
        if (eta) {
            eta[4 * i] = laplace_from_word(w.x, sigma);
            eta[4 * i + 1] = laplace_from_word(w.y, sigma);
            eta[4 * i + 2] = laplace_from_word(w.z, sigma);
            eta[4 * i + 3] = laplace_from_word(w.w, sigma);
        }
    }
}

template <int kOutF32, int kFastC>
cudaError_t launch_rc(const uint8_t *records, int64_t record_stride, uint32_t n, uint8_t *out, int64_t out_frame_stride,
                      int64_t out_pitch, int max_M, int max_N, int max_C, int out_align, int32_t *status,
                      cudaStream_t s) {
    const size_t smem = fast_smem(kOutF32, kFastC, out_align);
    auto kern = k_reconstruct<kOutF32, kFastC>;
    const int per_sm = launch_prep(reinterpret_cast<const void *>(kern), kThreads, smem);
    const int grid = per_sm * sm_count();
    const char *name = kOutF32 ? "k_reconstruct_f32" : "k_reconstruct_u8";
    prof_begin(name, s);
    kern<<<grid, kThreads, smem, s>>>(records, record_stride, n, out, out_frame_stride, out_pitch, max_M, max_N, max_C,
                                      out_align, status);
    prof_end(name, s);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_batch_reconstruct(const BatchEntry *tab, uint32_t n_img, uint32_t items, int out_type, int max_C,
                                     int out_align, int32_t *status, cudaStream_t s) {
    const int fc = max_C;  // the fast path serves any row alignment (16-byte rows reuse vectors per band)
#define DPPIX_BRC(F, FC) return launch_brc<F, FC>(tab, n_img, items, max_C, out_align, status, s)
    if (out_type == DP_PIX_OUT_F32) {
        switch (fc) {
            case 1: DPPIX_BRC(1, 1);
            case 2: DPPIX_BRC(1, 2);
            case 3: DPPIX_BRC(1, 3);
            case 4: DPPIX_BRC(1, 4);
            default: DPPIX_BRC(1, 0);
        }
    }
    switch (fc) {
        case 1: DPPIX_BRC(0, 1);
        case 2: DPPIX_BRC(0, 2);
        case 3: DPPIX_BRC(0, 3);
        case 4: DPPIX_BRC(0, 4);
        default: DPPIX_BRC(0, 0);
    }
#undef DPPIX_BRC
}

cudaError_t launch_reconstruct(const uint8_t *records, int64_t record_stride, uint32_t n, uint8_t *out,
                               int64_t out_frame_stride, int64_t out_pitch, int out_type, int max_M, int max_N,
                               int max_C, int out_align, int32_t *status, cudaStream_t s) {
    const int fc = max_C;  // the fast path serves any row alignment (16-byte rows reuse vectors per band)
#define DPPIX_RC(F, FC) \
    return launch_rc<F, FC>(records, record_stride, n, out, out_frame_stride, out_pitch, max_M, max_N, max_C, out_align, \
                            status, s)
    if (out_type == DP_PIX_OUT_F32) {
        switch (fc) {
            case 1: DPPIX_RC(1, 1);
            case 2: DPPIX_RC(1, 2);
            case 3: DPPIX_RC(1, 3);
            case 4: DPPIX_RC(1, 4);
            default: DPPIX_RC(1, 0);
        }
    }
    switch (fc) {
        case 1: DPPIX_RC(0, 1);
        case 2: DPPIX_RC(0, 2);
        case 3: DPPIX_RC(0, 3);
        case 4: DPPIX_RC(0, 4);
        default: DPPIX_RC(0, 0);
    }
#undef DPPIX_RC
}

cudaError_t launch_keys_advance(dp_pix_frame_key *keys, uint32_t n, uint64_t delta, cudaStream_t s) {
    const uint32_t blocks = std::min<uint32_t>((n + 255) / 256, 1024);
    prof_begin("k_keys_advance", s);
    k_keys_advance<<<blocks, 256, 0, s>>>(keys, n, delta);
    prof_end("k_keys_advance", s);
    return cudaGetLastError();
}

cudaError_t launch_debug_noise(uint64_t seed, const uint32_t *ctr, uint64_t n, uint32_t *words, float *eta,
                               float sigma, cudaStream_t s) {
    const uint64_t blocks = (n + 255) / 256;
    const int grid = (int)(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096);
    prof_begin("k_debug_noise", s);
    k_debug_noise<<<grid, 256, 0, s>>>(seed, ctr, n, words, eta, sigma);
    prof_end("k_debug_noise", s);
    return cudaGetLastError();
}

}  // namespace dppix
