// k_release.cu -- the streaming kernels of the release path.
//
// The kernels work on "segments": one tile row (T image rows) times `seg_tiles` consecutive tiles of one
// frame, with the mirror padding of the last tile row/column resolved by index (Alg. 2 step 4, Alg. 3
// step 3; the padded image is never materialised).
//  - k_release / k_batch_release: exact u32 sums of each tile's b_r x b_r cells (Eq. 2; Alg. 2 step 6;
//    Alg. 3 steps 8 and 14) from the staged segment, Laplace noise from the in-register Philox, clip, the
//    record payload (Alg. 3 steps 9-10 and 15-17);
//  - k_tile_stats: per-tile S, Q for the variance classes and, when the grids share a divisor g >= 4, the
//    g x g cell sums from which any b_r-cell sum is later assembled (image read once): column sums over
//    each band's rows in 16-bit SIMD lanes, then per-(cell, channel) sums over the band's columns;
//  - k_emit: g-cell sums -> b_r-cell sums -> noise -> record;
//  - k_emit_recon: k_emit and the reconstruction fused.
#include <algorithm>

#include "seg_write.cuh"

namespace dppix {
namespace {

constexpr int kThreads = 256;
constexpr int kRelThreads = 256;  // threads of the release kernels' item loop

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Stage rows ty*T .. ty*T+T-1 (mirrored past M) and pixel columns [x0, x0 + ns*T) (mirrored past N) of
// frame f into raw[j * rowstride + byte], then barrier.
__device__ void stage_segment(const Geom &g, const CallArgs &a, uint32_t f, int ty, int tx0, int ns, uint8_t *raw) {
    const int T = g.T, C = g.C, rs = g.seg_rowstride;
    const int x0 = tx0 * T;
    const int W = ns * T;
    const int xv = min(W, g.N - x0);  // in-image columns of the segment (>= 1)
    const int vb = xv * C;
    const uint8_t *fbase = a.frames + (uint64_t)f * (uint64_t)a.frame_stride + (int64_t)x0 * C;
    const int tid = threadIdx.x, nt = blockDim.x;
    int done = 0;  // bytes per row covered by vector copies
    if (a.vec == 16) {
        const int nv = vb >> 4;
        for (int idx = tid; idx < T * nv; idx += nt) {
            const int j = idx / nv, v = idx - j * nv;
            const int sy = reflect_idx(ty * T + j, g.M, g.pad_mode);
            cp_async16(raw + j * rs + 16 * v, fbase + (int64_t)sy * g.pitch + 16 * v);
        }
        done = nv << 4;
    } else {
        // rows not 16-byte aligned: each thread takes 4 consecutive staged chunks of a row (the last one may be
        // partial), loads the aligned 16-byte granules that hold them (all in flight together) and cuts the
        // chunks out with funnel shifts.  Only granules holding a byte of the row are read, so no load leaves
        // the allocation.
        const int nvt = (vb + 15) >> 4, tb = vb & 15;
        const int ng = (nvt + 3) >> 2;
        for (int idx = tid; idx < T * ng; idx += nt) {
            const int j = idx / ng, v0 = 4 * (idx - j * ng);
            const int cnt = min(4, nvt - v0);
            const int last_bytes = (v0 + cnt == nvt && tb) ? tb : 16;  // bytes of the group's last chunk
            const int sy = reflect_idx(ty * T + j, g.M, g.pad_mode);
            const uintptr_t addr = reinterpret_cast<uintptr_t>(fbase + (int64_t)sy * g.pitch) + 16u * (uint32_t)v0;
            const int o = (int)(addr & 15u);
            const uint4 *ga = reinterpret_cast<const uint4 *>(addr - (uintptr_t)o);
            uint4 x[5];
#pragma unroll
            for (int q = 0; q < 5; ++q)
                x[q] = (q < cnt || (q == cnt && o + last_bytes > 16)) ? __ldg(ga + q) : make_uint4(0u, 0u, 0u, 0u);
            const int qw = o >> 2, sh = 8 * (o & 3);
            uint8_t *dst = raw + j * rs + 16 * v0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (q >= cnt) break;
                const uint32_t w[8] = {x[q].x, x[q].y, x[q].z, x[q].w, x[q + 1].x, x[q + 1].y, x[q + 1].z, x[q + 1].w};
                uint32_t r[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    // words qw+k and qw+k+1 of the 32-byte window, selected without dynamic register indexing
                    uint32_t lo = w[k], hi = w[k + 1];
                    if (qw == 1) { lo = w[k + 1]; hi = w[k + 2]; }
                    if (qw == 2) { lo = w[k + 2]; hi = w[k + 3]; }
                    if (qw == 3) { lo = w[k + 3]; hi = w[k + 4]; }
                    r[k] = __funnelshift_r(lo, hi, sh);
                }
                if (q < cnt - 1 || last_bytes == 16) {
                    reinterpret_cast<uint4 *>(dst)[q] = make_uint4(r[0], r[1], r[2], r[3]);
                } else {
                    for (int bb = 0; bb < last_bytes; ++bb) dst[16 * q + bb] = (uint8_t)(r[bb >> 2] >> (8 * (bb & 3)));
                }
            }
        }
        done = vb;
    }
    const int tail = vb - done;
    if (tail > 0) {
        for (int idx = tid; idx < T * tail; idx += nt) {
            const int j = idx / tail, k = done + (idx - j * tail);
            const int sy = reflect_idx(ty * T + j, g.M, g.pad_mode);
            raw[j * rs + k] = fbase[(int64_t)sy * g.pitch + k];
        }
    }
    const int pb = (W - xv) * C;  // mirrored bytes past the right edge
    if (pb > 0) {
        const uint8_t *fb0 = a.frames + (uint64_t)f * (uint64_t)a.frame_stride;
        for (int idx = tid; idx < T * pb; idx += nt) {
            const int j = idx / pb, k = idx - j * pb;
            const int px = xv + k / C, ch = k - (k / C) * C;
            const int sy = reflect_idx(ty * T + j, g.M, g.pad_mode);
            const int sx = reflect_idx(x0 + px, g.N, g.pad_mode);
            raw[j * rs + px * C + ch] = fb0[(int64_t)sy * g.pitch + (int64_t)sx * C + ch];
        }
    }
    cp_async_wait_all();
    __syncthreads();
}

__device__ __forceinline__ void emit_cell(const Geom &g, const CallArgs &a, uint8_t *dst, const uint32_t *S, int r,
                                          uint32_t cell_idx, uint64_t frame, uint32_t sid, float *ov = nullptr) {
    uint4 words = make_uint4(0, 0, 0, 0);
    if (!g.noise_free && g.dtype != DP_PIX_REC_SUM_U32)
        words = cell_noise_words(g.seed, cell_idx, (uint32_t)r, sid, frame);
    emit_values(g, g.C, dst, S, words, g.sigma_f[r], g.b2_f[r], g.inv_b2_f[r], ov);
}

// ------------------------------------------------------------------------------------------------------
// k_release / k_batch_release: staged segment -> exact cell sums of each tile's own grid -> noise -> clip
// -> record (Alg. 3 steps 8-10 and 14-17).
//
// Staging: every row of an item is copied as the aligned 16-byte granules that hold its bytes (cp.async,
// whatever the row's alignment), and the row's offset inside its first granule is kept; consumers realign
// words with a funnel shift.  The item's map bytes and payload offsets come with the same asynchronous
// copies, so preparing an item waits on nothing.  Items are double-buffered: the next item's copies are in
// flight while the current one is summed.  Each CTA takes chunks of consecutive items, dealt round-robin.  Work units are
// (tile, cell, row part): a b_r x b_r cell is split into 2^rel_lp[r] row parts when its bytes exceed a
// budget, so that units do similar work; the parts of a cell sit on adjacent, aligned lanes and add their
// partial sums with shuffles.  A row part's sums use dp4a with compile-time channel masks on realigned words.
// ------------------------------------------------------------------------------------------------------
constexpr int kRelSegMax = 16;   // tiles per staged segment

struct RelItem {
    int32_t ns, tx0, xv, padb, ty, mapoff;
    uint32_t f;
    uint32_t mapw[6];                // aligned words holding the segment's map bytes (from byte mapoff)
    uint32_t tileoff[kRelSegMax];    // payload offsets of the segment's tiles
    int32_t rowbase[kMaxT];          // staged byte of each row's first pixel (row * stride + granule offset)
};

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Bulk (TMA) copies into shared memory completing on an mbarrier, and the mbarrier operations they need.
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_complete_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.complete_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar)) : "memory");
}
// Waits for the phase of the given parity to complete; gives up (false) after `tries` tries (try_wait itself
// blocks for a bounded time), so that a copy that never lands cannot hang the GPU.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t tries = kWaitTries) {
    for (uint32_t it = 0; it < tries; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(smem_u32(bar)), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Bytes per staged row of an item of S tiles: room for the 15-byte granule offset and the word reads
// that run up to 7 bytes past a row's last byte.
__host__ __device__ __forceinline__ int rel_rowstride(int S, int T, int C) { return (S * T * C + 15) / 16 * 16 + 32; }

// x / d for 0 <= x < 2^14, 1 <= d <= 128 from an approximate reciprocal: the product is at most one short.
__device__ __forceinline__ int udiv_small(int x, int d, float inv) {
    int q = __float2int_rz(__int2float_rn(x) * inv);
    if (x - q * d >= d) ++q;
    return q;
}

// Issues one bulk copy per row j < T of image rows ty*T + j (mirrored past M) of `base` (rows `pitch` bytes
// apart), bytes [0, vb) of each, as the aligned 16-byte granules that hold them, into raw + j * rs;
// rowbase[j] receives the staged position of byte 0.  Thread j copies row j: the warps with warp*32 < T
// call this (whole warps).  Each warp announces its rows' bytes to the mbarrier before copying.  In the
// bounds-checked build a row whose bytes leave [ext, ext + ext_bytes) is not copied (and raises the error).
__device__ __forceinline__ void stage_rows(const uint8_t *base, int64_t pitch, int M, int pad_mode, int ty, int T, int vb,
                                           int rs, uint8_t *raw, int32_t *rowbase, uint64_t *bar,
                                           const uint8_t *ext = nullptr, uint64_t ext_bytes = 0,
                                           int32_t *status = nullptr) {
    const int j = threadIdx.x, lane = threadIdx.x & 31;
    uint32_t bytes = 0;
    const uint8_t *ga = nullptr;
    if (j < T) {
        const int sy = reflect_idx(ty * T + j, M, pad_mode);
        const uintptr_t addr = reinterpret_cast<uintptr_t>(base + (int64_t)sy * pitch);
        const int o = (int)(addr & 15u);
        ga = reinterpret_cast<const uint8_t *>(addr - (uintptr_t)o);
        const bool in = ext == nullptr ||
                        chk(reinterpret_cast<const uint8_t *>(addr), (uint64_t)vb, ext, ext_bytes, status, kChkFrame);
        bytes = in ? 16u * (uint32_t)((o + vb + 15) >> 4) : 0u;
        rowbase[j] = j * rs + o;
    }
    const uint32_t wsum = __reduce_add_sync(0xffffffffu, bytes);
    if (lane == 0) mbar_expect_tx(bar, wsum);
    __syncwarp();
    if (j < T && bytes > 0) bulk_g2s(raw + j * rs, ga, bytes, bar);
}

// Prepares item (f, ty, sg) into `it` and issues the copies of its map bytes, payload offsets and rows
// (whole block; no barrier: the caller's barrier after cp.async.wait publishes `it`).
__device__ __forceinline__ void rel_prepare(const Geom &g, const CallArgs &a, uint32_t f, uint32_t rowitem, RelItem &it,
                                            uint8_t *raw, uint64_t *bar) {
    const int T = g.T;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (warp * 32 >= max(T, 64)) return;  // the copies need warps 0 and 1 and one thread per row
    const int C = g.C, S = g.seg_tiles;
    const int rs = rel_rowstride(S, T, C);
    const int ty = (int)(rowitem / (uint32_t)g.seg_per_row);
    const int tx0 = ((int)rowitem - ty * g.seg_per_row) * S;
    const int ns = min(S, g.GC - tx0);
    const int x0 = tx0 * T;
    const int xv = min(ns * T, g.N - x0);
    if (warp == 0) {
        const uintptr_t msrc = reinterpret_cast<uintptr_t>(a.records + (uint64_t)f * (uint64_t)a.record_stride +
                                                           g.map_offset + (uint64_t)ty * g.GC + tx0);
        const int mo = (int)(msrc & 3u);
        if (lane == 0) {
            it.ns = ns;
            it.tx0 = tx0;
            it.xv = xv;
            it.padb = (ns * T - xv) * C;
            it.ty = ty;
            it.mapoff = mo;
            it.f = f;
        }
        if (lane < ((mo + ns + 3) >> 2)) cp_async4(&it.mapw[lane], reinterpret_cast<const void *>(msrc - mo + 4u * lane));
    } else if (warp == 1 && lane < ns) {
        const uint32_t *toff = reinterpret_cast<const uint32_t *>(a.ws + (uint64_t)f * g.ws_per_frame + g.ws_tileoff);
        cp_async4(&it.tileoff[lane], toff + ty * g.GC + tx0 + lane);
    }
    if (warp * 32 < T)
        stage_rows(a.frames + (uint64_t)f * (uint64_t)a.frame_stride + (int64_t)x0 * C, g.pitch, g.M, g.pad_mode, ty, T,
                   xv * C, rs, raw, it.rowbase, bar, a.frames, a.frames_bytes, a.status);
}

// dp4a mask of channel ch for a word whose first byte is byte 4k of a cell row (C interleaved channels).
template <int C>
__device__ __forceinline__ constexpr uint32_t chan_mask(int k, int ch) {
    return C == 1 ? 0x01010101u
         : C == 2 ? (ch == 0 ? 0x00010001u : 0x01000100u)
         : C == 4 ? (1u << (8 * ch))
         : /* C == 3: byte i of word k is channel (4k + i) mod 3 */
           ((((4 * k + 0) % 3 == ch) ? 0x00000001u : 0u) | (((4 * k + 1) % 3 == ch) ? 0x00000100u : 0u) |
            (((4 * k + 2) % 3 == ch) ? 0x00010000u : 0u) | (((4 * k + 3) % 3 == ch) ? 0x01000000u : 0u));
}

template <int C, int KP>
__device__ __forceinline__ void acc_word(uint32_t w, uint32_t *S) {
#pragma unroll
    for (int ch = 0; ch < C; ++ch) S[ch] = __dp4a(w, chan_mask<C>(KP, ch), S[ch]);
}

// Channel sums of `nbytes` bytes starting at staged byte rowbase[j] + L0, over rows j in [r0, r1).
template <int C>
__device__ __forceinline__ void rows_sum(const uint8_t *raw, const int32_t *rowbase, int r0, int r1, int L0,
                                         int nbytes, uint32_t *S) {
    constexpr int PER = (C == 3) ? 3 : 1;  // words per mask period
    const int nw = (nbytes + 3) >> 2;
    const int nfull = nbytes >> 2;
    const uint32_t tail = (nbytes & 3) ? (1u << (8 * (nbytes & 3))) - 1u : 0xFFFFFFFFu;
    for (int j = r0; j < r1; ++j) {
        const int addr = rowbase[j] + L0;
        const uint32_t *w = reinterpret_cast<const uint32_t *>(raw + (addr & ~3));
        const uint32_t sh = 8u * (uint32_t)(addr & 3);
        uint32_t lo = w[0];
        int k = 0;
        for (; k + PER <= nfull; k += PER) {
#pragma unroll
            for (int kk = 0; kk < PER; ++kk) {
                const uint32_t hi = w[k + kk + 1];
                const uint32_t x = __funnelshift_r(lo, hi, sh);
                lo = hi;
                if (kk == 0) acc_word<C, 0>(x, S);
                if (kk == 1) acc_word<C, 1>(x, S);
                if (kk == 2) acc_word<C, 2>(x, S);
            }
        }
        // the rest: fewer than PER full words and the partial word, in mask order
#pragma unroll
        for (int kk = 0; kk < PER + 1; ++kk) {
            if (k + kk >= nw) break;
            const uint32_t hi = w[k + kk + 1];
            uint32_t x = __funnelshift_r(lo, hi, sh);
            lo = hi;
            if (k + kk == nw - 1) x &= tail;
            if (kk % PER == 0) acc_word<C, 0>(x, S);
            if (kk % PER == 1) acc_word<C, 1>(x, S);
            if (kk % PER == 2) acc_word<C, 2>(x, S);
        }
    }
}

// rows_sum for cells of at most 4 NWO bytes per row, straight-line: each row reads the NWO + 1 words under its
// bytes, realigns NWO words, masks the bytes past nbytes and adds them with the channel masks of their word
// position (the cell's first byte is channel 0).
template <int C, int NWO>
__device__ __forceinline__ void rows_sum_fixed(const uint8_t *raw, const int32_t *rowbase, int r0, int r1, int L0,
                                               int nbytes, uint32_t *S) {
    uint32_t m[NWO];
#pragma unroll
    for (int q = 0; q < NWO; ++q) {
        const int keep = nbytes - 4 * q;
        m[q] = keep >= 4 ? 0xFFFFFFFFu : (keep <= 0 ? 0u : (1u << (8 * keep)) - 1u);
    }
    for (int j = r0; j < r1; ++j) {
        const int addr = rowbase[j] + L0;
        const uint32_t *w = reinterpret_cast<const uint32_t *>(raw + (addr & ~3));
        const uint32_t sh = 8u * (uint32_t)(addr & 3);
        uint32_t in[NWO + 1];
#pragma unroll
        for (int q = 0; q <= NWO; ++q) in[q] = w[q];
#pragma unroll
        for (int q = 0; q < NWO; ++q) {
            const uint32_t x = __funnelshift_r(in[q], in[q + 1], sh) & m[q];
#pragma unroll
            for (int ch = 0; ch < C; ++ch) S[ch] = __dp4a(x, chan_mask<C>(q % (C == 3 ? 3 : 1), ch), S[ch]);
        }
    }
}

// Sums of a cell's rows, straight-line for cells of up to 32 bytes per row (cell_bytes = b C, the same for all
// lanes of a warp), the general loop otherwise.
template <int C>
__device__ __forceinline__ void cell_rows_sum(const uint8_t *raw, const int32_t *rowbase, int r0, int r1, int L0,
                                              int nbytes, int cell_bytes, uint32_t *S) {
    switch ((cell_bytes + 3) >> 2) {
        case 1:
        case 2: rows_sum_fixed<C, 2>(raw, rowbase, r0, r1, L0, nbytes, S); break;
        case 3: rows_sum_fixed<C, 3>(raw, rowbase, r0, r1, L0, nbytes, S); break;
        case 4: rows_sum_fixed<C, 4>(raw, rowbase, r0, r1, L0, nbytes, S); break;
        case 5: rows_sum_fixed<C, 5>(raw, rowbase, r0, r1, L0, nbytes, S); break;
        case 6: rows_sum_fixed<C, 6>(raw, rowbase, r0, r1, L0, nbytes, S); break;
        case 7:
        case 8: rows_sum_fixed<C, 8>(raw, rowbase, r0, r1, L0, nbytes, S); break;
        default: rows_sum<C>(raw, rowbase, r0, r1, L0, nbytes, S); break;
    }
}

// Sums, noise and record of the staged item `it` (whole block).
template <int C>
__device__ __forceinline__ void rel_compute(const Geom &g, const CallArgs &a, const RelItem &it, uint8_t *raw) {
    const int T = g.T;
    const bool strict = g.pad_mode == DP_PIX_PAD_NONE;  // no padding: edge cells keep their samples in the frame
    const int hv = strict ? min(T, g.M - it.ty * T) : T;  // rows of the item inside the frame
    if (it.padb > 0 && !strict) {
        // mirrored columns past the right edge, copied next to the row's last in-image byte
        const uint8_t *fb0 = a.frames + (uint64_t)it.f * (uint64_t)a.frame_stride;
        const int x0 = it.tx0 * T, pb = it.padb;
        for (int idx = threadIdx.x; idx < T * pb; idx += blockDim.x) {
            const int j = idx / pb, k = idx - j * pb;
            const int px = it.xv + k / C, ch = k - (k / C) * C;
            const int sy = reflect_idx(it.ty * T + j, g.M, g.pad_mode);
            const int sx = reflect_idx(x0 + px, g.N, g.pad_mode);
            const uint8_t *src = fb0 + (int64_t)sy * g.pitch + (int64_t)sx * C + ch;
            if (chk(src, 1, a.frames, a.frames_bytes, a.status, kChkFrame)) raw[it.rowbase[j] + it.xv * C + k] = *src;
        }
        fence_proxy_async();  // these generic writes precede the bulk copies that later refill the buffer
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int ns = it.ns, pmax = g.rel_pmax;
    const uint8_t *mapb = reinterpret_cast<const uint8_t *>(it.mapw) + it.mapoff;
    int total = 0;
    for (int t = 0; t < ns; ++t) {
        int r = mapb[t];
        if (r >= g.K) r = 0;
        total += g.rel_units[r];
    }
    uint8_t *rec = a.records + (uint64_t)it.f * (uint64_t)a.record_stride;
    const uint64_t frame = key_frame(a, it.f);
    const uint32_t sid = key_stream(a, it.f);
    for (int u = threadIdx.x; u - lane < total; u += blockDim.x) {
        uint32_t S[4] = {0u, 0u, 0u, 0u};
        int t = 0, r = 0, lp = 0, cell = 0, part = 0;
        bool valid = false;
        if (u < total) {
            int start = 0;
            for (;; ++t) {
                r = mapb[t];
                if (r >= g.K) r = 0;
                const int cnt = g.rel_units[r];
                if (u < start + cnt || t + 1 == ns) break;
                start += cnt;
            }
            const int lu = u - start;
            const int cs = g.cells_side[r], b = g.grid[r];
            lp = g.rel_lp[r];
            part = lu & ((1 << lp) - 1);
            cell = lu >> lp;
            if (cell < cs * cs) {
                valid = true;
                const int cy = udiv_small(cell, cs, __fdividef(1.0f, (float)cs)), cx = cell - cy * cs;
                const int rpp = (b + (1 << lp) - 1) >> lp;
                const int r0 = cy * b + part * rpp;
                int r1 = min(r0 + rpp, (cy + 1) * b);
                int nbytes = b * C;
                if (strict) {
                    r1 = min(r1, hv);
                    nbytes = max(0, min(b, g.N - (it.tx0 + t) * T - cx * b)) * C;
                }
                if (r0 < r1 && nbytes > 0) rows_sum<C>(raw, it.rowbase, r0, r1, (t * T + cx * b) * C, nbytes, S);
            } else {
                lp = 0;
            }
        }
        // the 2^lp lanes of a cell are adjacent and aligned: butterfly over the offsets below 2^lp
        for (int o = 1; o < pmax; o <<= 1) {
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                const uint32_t v = __shfl_xor_sync(0xffffffffu, S[ch], o);
                if (o < (1 << lp)) S[ch] += v;
            }
        }
        if (valid && part == 0) {
            const int cs = g.cells_side[r];
            const int cy = udiv_small(cell, cs, __fdividef(1.0f, (float)cs)), cx = cell - cy * cs;
            const uint32_t cell_idx =
                (uint32_t)(it.ty * cs + cy) * (uint32_t)(g.GC * cs) + (uint32_t)((it.tx0 + t) * cs + cx);
            uint8_t *dst = rec + it.tileoff[t] + (uint64_t)cell * C * g.es;
            float sigma = g.sigma_f[r], b2 = g.b2_f[r], ib2 = g.inv_b2_f[r];
            int n = 1;
            if (strict) {
                // Alg. 1's partial cell: mean over its h x w samples in the frame, noise scale R m / (h w eps_r)
                const int b = g.grid[r];
                const int h = max(0, min(b, hv - cy * b));
                const int w = max(0, min(b, g.N - (it.tx0 + t) * T - cx * b));
                n = h * w;
                if (n > 0 && n < b * b) {
                    b2 = (float)n;
                    ib2 = 0.0f;
                    sigma = __fdiv_rn(g.sigma_f[r] * g.b2_f[r], (float)n);
                }
            }
            if (!chk(dst, (uint64_t)C * g.es, a.records, a.records_bytes, a.status, kChkRecord)) {
                // bounds-checked build: a write outside the records is skipped
            } else if (n == 0) {  // wholly outside the frame: no sample, stored as 0
#pragma unroll
                for (int ch = 0; ch < C; ++ch) {
                    if (g.es == 4) reinterpret_cast<uint32_t *>(dst)[ch] = 0u;
                    else dst[ch] = 0;
                }
            } else {
                uint4 words = make_uint4(0, 0, 0, 0);
                if (!g.noise_free && g.dtype != DP_PIX_REC_SUM_U32)
                    words = cell_noise_words(g.seed, cell_idx, (uint32_t)r, sid, frame);
                emit_values(g, C, dst, S, words, sigma, b2, ib2, nullptr);
            }
        }
    }
}

// The items of a CTA: chunks of q consecutive items dealt round-robin over the CTAs, q = kRelChunk or, for
// launches with fewer items, an equal share.  Each CTA's items increase, so an image changes at most once per
// chunk, while concurrently running CTAs read neighbouring chunks (measured on the 256-portrait batch: release
// 2.56 ms with one contiguous share per CTA, 2.22 / 2.21 / 2.18 ms with chunks of 8 / 16 / 32 items).
constexpr uint32_t kRelChunk = 32;
struct RelSeq {
    uint32_t items, q;
    __device__ __forceinline__ RelSeq(uint32_t n) : items(n) {
        const uint32_t share = (n + gridDim.x - 1) / gridDim.x;
        q = share < kRelChunk ? share : kRelChunk;
        if (q == 0) q = 1;
    }
    __device__ __forceinline__ uint32_t first() const {
        const uint64_t f = (uint64_t)blockIdx.x * q;
        return f < items ? (uint32_t)f : items;
    }
    __device__ __forceinline__ uint32_t next(uint32_t item) const {
        const uint64_t n = (item + 1) % q ? (uint64_t)item + 1 : (uint64_t)item + 1 + (uint64_t)(gridDim.x - 1) * q;
        return n < items ? (uint32_t)n : items;
    }
};

// The double-buffered item loop of both release kernels: prepare(item, nb) stages an item into buffer nb
// (rows by bulk copies completing on bars[nb], its tables by cp.async), compute(nb) consumes buffer nb.
// The mbarrier of a buffer completes one phase per item: thread 0 arrives once every warp has announced
// the item's bytes.  A wait gives up after `tries` tries, raises DP_PIX_E_TIMEOUT and ends the CTA once
// this item's and the next item's copies have landed (those waits are bounded too).  short_tx > 0 (a test
// of this path) announces that many bytes more than the CTA's first item delivers, so its phase cannot
// complete and the wait runs out; the phantom bytes are then retired, so the drain still sees every copy
// land and none is in flight when the CTA ends.
template <class Prep, class Comp>
__device__ __forceinline__ void rel_loop(const RelSeq &seq, uint64_t *bars, int32_t *status, Prep prepare,
                                         Comp compute, uint32_t tries = kWaitTries, uint32_t short_tx = 0) {
    const uint32_t i0 = seq.first(), items = seq.items;
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    int buf = 0;
    uint32_t ph0 = 0, ph1 = 0;
    if (threadIdx.x == 0 && i0 < items && short_tx) mbar_expect_tx(&bars[0], short_tx);
    if (i0 < items) prepare(i0, 0);
    cp_async_commit();
    __syncthreads();
    if (threadIdx.x == 0 && i0 < items) mbar_arrive(&bars[0]);
    for (uint32_t item = i0; item < items;) {
        const uint32_t nitem = seq.next(item);
        const bool next = nitem < items;
        if (next) prepare(nitem, buf ^ 1);
        cp_async_commit();
        cp_async_wait_1();
        // warp 0 waits for the copies; the barrier releases the other warps (which do not spin meanwhile) and
        // orders the landed bytes before their reads
        const bool ok = threadIdx.x < 32 ? mbar_wait(&bars[buf], buf ? ph1 : ph0, tries) : true;
        const int fail = __syncthreads_or(!ok);
        if (threadIdx.x == 0 && next) mbar_arrive(&bars[buf ^ 1]);
        if (fail) {
            if (threadIdx.x == 0) {
                raise_status(status, DP_PIX_E_TIMEOUT, 0x500u);
                if (short_tx && item == i0) mbar_complete_tx(&bars[buf], short_tx);
            }
            (void)mbar_wait(&bars[buf], buf ? ph1 : ph0);                // this item's copies, bounded
            if (next) (void)mbar_wait(&bars[buf ^ 1], buf ? ph0 : ph1);  // the next item's copies, bounded
            cp_async_wait_all();
            return;
        }
        if (buf) ph1 ^= 1u; else ph0 ^= 1u;
        compute(buf);
        __syncthreads();
        buf ^= 1;
        item = nitem;
    }
    cp_async_wait_all();
}

template <int C>
__global__ void __launch_bounds__(kRelThreads) k_release(const Geom g, const CallArgs a) {
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ RelItem it[2];
    __shared__ uint64_t bars[2];
    const int buf_bytes = g.T * rel_rowstride(g.seg_tiles, g.T, C);
    const RelSeq seq(a.n_frames * (uint32_t)g.GR * (uint32_t)g.seg_per_row);
    const uint32_t per_frame = (uint32_t)g.GR * (uint32_t)g.seg_per_row;
    auto prepare = [&](uint32_t item, int nb) {
        const uint32_t f = item / per_frame;
        rel_prepare(g, a, f, item - f * per_frame, it[nb], dyn + nb * buf_bytes, &bars[nb]);
    };
    auto compute = [&](int nb) { rel_compute<C>(g, a, it[nb], dyn + nb * buf_bytes); };
    rel_loop(seq, bars, a.status, prepare, compute, g.wait_tries, g.test_short_tx);
}

// Batch: items = (tile row, segment) of every image, image i owning [base[2], base[2] + GR * seg_per_row).
template <int C>
__global__ void __launch_bounds__(kRelThreads) k_batch_release(const BatchEntry *tab, uint32_t n_img, uint32_t items,
                                                            int buf_bytes) {
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ RelItem it[2];
    __shared__ BatchShared bs[2];
    __shared__ uint64_t bars[2];
    const RelSeq seq(items);
    int cur0 = -1, cur1 = -1;        // image whose geometry bs[0], bs[1] hold
    int img = -1;                    // image of the last prepared item, owning items [img_lo, img_hi)
    uint32_t img_lo = 0, img_hi = 0;
    auto prepare = [&](uint32_t item, int nb) {
        if (img < 0 || item >= img_hi) {  // items increase: the image changes at most once per chunk
            const int i = batch_find(tab, n_img, item, 2);
            img = i;
            img_lo = tab[i].base[2];
            img_hi = i + 1 < (int)n_img ? tab[i + 1].base[2] : items;
        }
        int &cur = nb ? cur1 : cur0;
        if (cur != img) {
            batch_load(tab, img, bs[nb]);
            cur = img;
        }
        rel_prepare(bs[nb].g, bs[nb].a, 0u, item - img_lo, it[nb], dyn + nb * buf_bytes, &bars[nb]);
    };
    auto compute = [&](int nb) { rel_compute<C>(bs[nb].g, bs[nb].a, it[nb], dyn + nb * buf_bytes); };
    rel_loop(seq, bars, tab[0].a.status, prepare, compute);
}

// ------------------------------------------------------------------------------------------------------
// k_batch_tiles: the batch release with whole warps per tile.  Items and their staging are k_batch_release's
// ((image, tile row, segment of S tiles), rows by bulk copies, double-buffered); the CTA's 8 warps are dealt
// out W = 8 / S to a tile.  The W warps of a tile take its cells in rounds of 32 W lanes, lane = (cell, row
// part): a tile of few cells splits each cell into 2^lp row parts on adjacent lanes (added by a butterfly),
// so that no lane searches a unit list and all lanes of a warp share one region and one cell width (the
// straight-line row sums of cell_rows_sum apply to the whole warp).
// ------------------------------------------------------------------------------------------------------
constexpr int kTilesThreads = 256;  // 8 warps

template <int C>
__device__ __forceinline__ void tiles_compute(const Geom &g, const CallArgs &a, const RelItem &it, uint8_t *raw) {
    const int T = g.T, S = g.seg_tiles;
    const bool strict = g.pad_mode == DP_PIX_PAD_NONE;  // no padding: edge cells keep their samples in the frame
    const int hv = strict ? min(T, g.M - it.ty * T) : T;  // rows of the item inside the frame
    if (it.padb > 0 && !strict) {
        // mirrored columns past the right edge, copied next to the row's last in-image byte
        const uint8_t *fb0 = a.frames;
        const int x0 = it.tx0 * T, pb = it.padb;
        for (int idx = threadIdx.x; idx < T * pb; idx += blockDim.x) {
            const int j = idx / pb, k = idx - j * pb;
            const int px = it.xv + k / C, ch = k - (k / C) * C;
            const int sy = reflect_idx(it.ty * T + j, g.M, g.pad_mode);
            const int sx = reflect_idx(x0 + px, g.N, g.pad_mode);
            const uint8_t *src = fb0 + (int64_t)sy * g.pitch + (int64_t)sx * C + ch;
            if (chk(src, 1, a.frames, a.frames_bytes, a.status, kChkFrame)) raw[it.rowbase[j] + it.xv * C + k] = *src;
        }
        fence_proxy_async();  // these generic writes precede the bulk copies that later refill the buffer
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ns = it.ns;
    const uint8_t *mapb = reinterpret_cast<const uint8_t *>(it.mapw) + it.mapoff;
    const int W = (kTilesThreads / 32) / S;  // warps per tile
    const int t = warp / W, wl = warp - t * W;
    if (t >= ns) return;
    int r = mapb[t];
    if (r >= g.K) r = 0;
    const int b = g.grid[r], cs = g.cells_side[r], ncell = cs * cs;
    int lp = 0;
    while ((ncell << (lp + 1)) <= 32 * W && (2 << lp) <= b && lp < 5) ++lp;
    const int units = ncell << lp, rpp = (b + (1 << lp) - 1) >> lp;
    const float inv_cs = __fdividef(1.0f, (float)cs);
    const int tx = it.tx0 + t;
    const int wt = strict ? max(0, min(T, g.N - tx * T)) : T;  // columns of the tile inside the frame
    uint8_t *rec = a.records + it.tileoff[t];
    const uint64_t frame = key_frame(a, 0);
    const uint32_t sid = key_stream(a, 0);
    const bool noisy = !g.noise_free && g.dtype != DP_PIX_REC_SUM_U32;
    for (int u0 = 32 * wl; u0 < units; u0 += 32 * W) {  // warp-uniform rounds
        const int u = u0 + lane;
        const bool valid = u < units;
        const int cell = u >> lp, part = u & ((1 << lp) - 1);
        const int cy = valid ? udiv_small(cell, cs, inv_cs) : 0, cx = cell - cy * cs;
        uint32_t Sm[4] = {0u, 0u, 0u, 0u};
        if (valid) {
            const int r0 = cy * b + part * rpp;
            int r1 = min(r0 + rpp, (cy + 1) * b);
            int nbytes = b * C;
            if (strict) {
                r1 = min(r1, hv);
                nbytes = max(0, min(b, wt - cx * b)) * C;
            }
            if (r0 < r1 && nbytes > 0)
                cell_rows_sum<C>(raw, it.rowbase, r0, r1, (t * T + cx * b) * C, nbytes, b * C, Sm);
        }
        for (int o = 1; o < (1 << lp); o <<= 1) {  // the 2^lp lanes of a cell are adjacent and aligned
#pragma unroll
            for (int ch = 0; ch < C; ++ch) Sm[ch] += __shfl_xor_sync(0xffffffffu, Sm[ch], o);
        }
        if (!valid || part != 0) continue;
        const uint32_t cell_idx = (uint32_t)(it.ty * cs + cy) * (uint32_t)(g.GC * cs) + (uint32_t)(tx * cs + cx);
        uint8_t *dst = rec + (uint64_t)cell * C * g.es;
        float sigma = g.sigma_f[r], b2 = g.b2_f[r], ib2 = g.inv_b2_f[r];
        int n = 1;
        if (strict) {
            // Alg. 1's partial cell: mean over its h x w samples in the frame, noise scale R m / (h w eps_r)
            const int h = max(0, min(b, hv - cy * b));
            const int w = max(0, min(b, wt - cx * b));
            n = h * w;
            if (n > 0 && n < b * b) {
                b2 = (float)n;
                ib2 = 0.0f;
                sigma = __fdiv_rn(g.sigma_f[r] * g.b2_f[r], (float)n);
            }
        }
        if (!chk(dst, (uint64_t)C * g.es, a.records, a.records_bytes, a.status, kChkRecord)) {
            // bounds-checked build: a write outside the record is skipped
        } else if (n == 0) {  // wholly outside the frame: no sample, stored as 0
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                if (g.es == 4) reinterpret_cast<uint32_t *>(dst)[ch] = 0u;
                else dst[ch] = 0;
            }
        } else {
            const uint4 words = noisy ? cell_noise_words(g.seed, cell_idx, (uint32_t)r, sid, frame)
                                      : make_uint4(0u, 0u, 0u, 0u);
            emit_values(g, C, dst, Sm, words, sigma, b2, ib2, nullptr);
        }
    }
}

template <int C>
__global__ void __launch_bounds__(kTilesThreads, 4) k_batch_tiles(const BatchEntry *tab, uint32_t n_img,
                                                                 uint32_t items, int buf_bytes) {
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ RelItem it[2];
    __shared__ BatchShared bs[2];
    __shared__ uint64_t bars[2];
    const RelSeq seq(items);
    int cur0 = -1, cur1 = -1;        // image whose geometry bs[0], bs[1] hold
    int img = -1;                    // image of the last prepared item, owning items [img_lo, img_hi)
    uint32_t img_lo = 0, img_hi = 0;
    auto prepare = [&](uint32_t item, int nb) {
        if (img < 0 || item >= img_hi) {  // items increase: the image changes at most once per chunk
            const int i = batch_find(tab, n_img, item, 2);
            img = i;
            img_lo = tab[i].base[2];
            img_hi = i + 1 < (int)n_img ? tab[i + 1].base[2] : items;
        }
        int &cur = nb ? cur1 : cur0;
        if (cur != img) {
            batch_load(tab, img, bs[nb]);
            cur = img;
        }
        rel_prepare(bs[nb].g, bs[nb].a, 0u, item - img_lo, it[nb], dyn + nb * buf_bytes, &bars[nb]);
    };
    auto compute = [&](int nb) { tiles_compute<C>(bs[nb].g, bs[nb].a, it[nb], dyn + nb * buf_bytes); };
    rel_loop(seq, bars, tab[0].a.status, prepare, compute);
}

// ------------------------------------------------------------------------------------------------------
// k_batch_classify: tile classification of every image of a batch from its u8 mask or f32 matte (Alg. 3
// steps 5-6), over (image, tile row, segment of cls_seg_tiles tiles) items with the release's staging loop:
// each item's T source rows arrive by bulk copies, then one thread per (column, row half) counts the simple
// samples of its column (mask: nonzero; matte: alpha < thr), mirrored columns past the right edge taken
// from their staged source column.  A tile is simple (region 0) iff 2 * #simple > T^2, a tie going to
// complex (region 1).
// ------------------------------------------------------------------------------------------------------
struct ClsItem {
    int32_t ns, tx0, xv, ty;
    uint32_t cnt[kRelSegMax];
    int32_t rowbase[kMaxT];
};

template <bool kMatte>
__device__ __forceinline__ void cls_compute(const Geom &g, const CallArgs &a, const ClsItem &it, uint8_t *raw,
                                            uint32_t *cnt_s) {
    constexpr int es = kMatte ? 4 : 1;
    const int T = g.T, ns = it.ns, ncols = ns * T;
    const int x0 = it.tx0 * T;
    const bool strict = g.pad_mode == DP_PIX_PAD_NONE;  // only the pixels inside the frame count
    const int hv = strict ? min(T, g.M - it.ty * T) : T;
    const int rsplit = max(1, (int)blockDim.x / ncols);
    const int rows_per = (T + rsplit - 1) / rsplit;
    for (int u = threadIdx.x; u < ncols * rsplit; u += blockDim.x) {
        const int part = u / ncols, c = u - part * ncols;
        const int j0 = part * rows_per, j1 = min(hv, j0 + rows_per);
        if (strict && c >= it.xv) continue;
        const int x = x0 + c;
        int sc = c;  // staged column of the sample
        bool global = false;
        if (c >= it.xv) {
            const int sx = reflect_idx(x, g.N, g.pad_mode);
            sc = sx - x0;
            global = sc < 0;
        }
        uint32_t n = 0;
        if (!global) {
#pragma unroll 4
            for (int j = j0; j < j1; ++j) {
                const uint8_t *p = raw + it.rowbase[j] + sc * es;
                if (kMatte)
                    n += !(*reinterpret_cast<const float *>(p) >= g.matte_thr) ? 1u : 0u;
                else
                    n += *p != 0 ? 1u : 0u;
            }
        } else {
            const int sx = reflect_idx(x, g.N, g.pad_mode);
            for (int j = j0; j < j1; ++j) {
                const int sy = reflect_idx(it.ty * T + j, g.M, g.pad_mode);
                const uint8_t *p = a.src + (int64_t)sy * a.src_pitch + (int64_t)sx * es;
                if (kMatte)
                    n += !(*reinterpret_cast<const float *>(p) >= g.matte_thr) ? 1u : 0u;
                else
                    n += *p != 0 ? 1u : 0u;
            }
        }
        atomicAdd(&cnt_s[c / T], n);
    }
    __syncthreads();
    if ((int)threadIdx.x < ns) {
        uint8_t *map = a.records + g.map_offset + (uint64_t)it.ty * g.GC + it.tx0;
        const int wv = strict ? min(T, g.N - (it.tx0 + (int)threadIdx.x) * T) : T;
        map[threadIdx.x] = (2u * cnt_s[threadIdx.x] > (uint32_t)hv * (uint32_t)wv) ? 0 : 1;
        cnt_s[threadIdx.x] = 0u;  // ready for the next item
    }
}

template <bool kMatte>
__global__ void __launch_bounds__(kThreads) k_batch_classify(const BatchEntry *tab, uint32_t n_img, uint32_t items,
                                                             int buf_bytes) {
    constexpr int es = kMatte ? 4 : 1;
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ ClsItem it[2];
    __shared__ BatchShared bs[2];
    __shared__ uint64_t bars[2];
    __shared__ uint32_t cnt_s[kRelSegMax];
    if (threadIdx.x < kRelSegMax) cnt_s[threadIdx.x] = 0u;
    const RelSeq seq(items);
    int cur0 = -1, cur1 = -1;
    int img = -1;
    uint32_t img_lo = 0, img_hi = 0;
    auto prepare = [&](uint32_t item, int nb) {
        if (img < 0 || item >= img_hi) {  // items increase: the image changes at most once per chunk
            const int i = batch_find(tab, n_img, item, 0);
            img = i;
            img_lo = tab[i].base[0];
            img_hi = i + 1 < (int)n_img ? tab[i + 1].base[0] : items;
        }
        int &cur = nb ? cur1 : cur0;
        if (cur != img) {
            batch_load(tab, img, bs[nb]);
            cur = img;
        }
        const Geom &g = bs[nb].g;
        const int T = g.T;
        if ((int)(threadIdx.x & ~31u) >= T) return;  // whole warps: the rows' copies start with a warp reduction
        const int S = cls_seg_tiles(T, es);
        const int spr = (g.GC + S - 1) / S;
        const uint32_t rowitem = item - img_lo;
        const int ty = (int)(rowitem / (uint32_t)spr);
        const int tx0 = ((int)rowitem - ty * spr) * S;
        const int ns = min(S, g.GC - tx0);
        const int x0 = tx0 * T;
        const int xv = min(ns * T, g.N - x0);
        ClsItem &c = it[nb];
        if (threadIdx.x == 0) {
            c.ns = ns;
            c.tx0 = tx0;
            c.xv = xv;
            c.ty = ty;
        }
        stage_rows(bs[nb].a.src + (int64_t)x0 * es, bs[nb].a.src_pitch, g.M, g.pad_mode, ty, T, xv * es,
                   rel_rowstride(S, T, es), dyn + nb * buf_bytes, c.rowbase, &bars[nb]);
    };
    auto compute = [&](int nb) { cls_compute<kMatte>(bs[nb].g, bs[nb].a, it[nb], dyn + nb * buf_bytes, cnt_s); };
    rel_loop(seq, bars, tab[0].a.status, prepare, compute);
}

// ------------------------------------------------------------------------------------------------------
// k_tile_stats: per tile S = sum x, Q = sum x^2 over the C*T*T padded samples -> key = n*Q - S^2 (exact);
// with `gsum`, also the g x g cell sums (u16) of every tile into the workspace.
// ------------------------------------------------------------------------------------------------------
template <bool kGsum>
__global__ void __launch_bounds__(kThreads) k_tile_stats(const Geom g, const CallArgs a) {
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ uint32_t S_s[16];
    __shared__ unsigned long long Q_s[16];
    const int T = g.T, C = g.C, TC = T * C, rs = g.seg_rowstride;
    uint8_t *raw = dyn;
    uint16_t *V = reinterpret_cast<uint16_t *>(dyn + (size_t)T * rs);
    const int gg = kGsum ? g.g : T;          // band height
    const int bands = T / gg;
    const int wcs = TC >> 2;                 // word columns (TC % 4 == 0 required on this path)
    const int per_tile = ((bands * wcs + 31) / 32) * 32;  // warp-aligned items per tile
    const int gcs = T / g.g;                 // g-cells per tile side
    const uint32_t items = a.n_frames * (uint32_t)g.GR * (uint32_t)g.seg_per_row;
    const int lane = threadIdx.x & 31;
    for (uint32_t item = blockIdx.x; item < items; item += gridDim.x) {
        const uint32_t sg = item % g.seg_per_row;
        const uint32_t fr = item / g.seg_per_row;
        const int ty = (int)(fr % g.GR);
        const uint32_t f = fr / g.GR;
        const int tx0 = (int)sg * g.seg_tiles;
        const int ns = min(g.seg_tiles, g.GC - tx0);
        if (threadIdx.x < 16) {
            S_s[threadIdx.x] = 0u;
            Q_s[threadIdx.x] = 0ull;
        }
        stage_segment(g, a, f, ty, tx0, ns, raw);

        const int totalA = ns * per_tile;
        for (int it = threadIdx.x; it - lane < totalA; it += blockDim.x) {
            // all lanes of a warp share one tile (per_tile is a multiple of 32)
            const int t = it / per_tile;
            const int rem = it - t * per_tile;
            uint32_t s = 0, q = 0;
            if (it < totalA && rem < bands * wcs) {
                const int band = rem / wcs, wc = rem - band * wcs;
                const uint32_t *src = reinterpret_cast<const uint32_t *>(raw + band * gg * rs + t * TC + 4 * wc);
                const int step = rs >> 2;
                uint32_t lo = 0, hi = 0;
                for (int i = 0; i < gg; ++i) {
                    const uint32_t w = src[i * step];
                    q = __dp4a(w, w, q);
                    s = __dp4a(w, 0x01010101u, s);
                    if (kGsum) {
                        lo += __byte_perm(w, 0u, 0x4240);
                        hi += __byte_perm(w, 0u, 0x4341);
                    }
                }
                if (kGsum) {
                    uint32_t *vdst = reinterpret_cast<uint32_t *>(V + ((size_t)(t * bands + band) * TC)) + 2 * wc;
                    vdst[0] = __byte_perm(lo, hi, 0x5410);
                    vdst[1] = __byte_perm(lo, hi, 0x7632);
                }
            }
            const uint32_t sw = __reduce_add_sync(0xffffffffu, s);
            unsigned long long qw = q;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) qw += __shfl_xor_sync(0xffffffffu, qw, off);
            if (lane == 0 && t < ns) {
                atomicAdd(&S_s[t], sw);
                atomicAdd(&Q_s[t], qw);
            }
        }
        __syncthreads();

        const uint32_t tile0 = (uint32_t)ty * g.GC + tx0;
        if (kGsum) {
            uint16_t *gimg = reinterpret_cast<uint16_t *>(a.ws + (uint64_t)f * g.ws_per_frame + g.ws_gsum);
            const int cells = gcs * gcs;
            for (int it = threadIdx.x; it < ns * cells; it += blockDim.x) {
                const int t = it / cells, cell = it - t * cells;
                const int cy = cell / gcs, cx = cell - cy * gcs;
                const uint16_t *vrow = V + (size_t)(t * bands + cy) * TC + cx * g.g * C;
                uint32_t S[4] = {0u, 0u, 0u, 0u};
                for (int i = 0; i < g.g; ++i) {
#pragma unroll
                    for (int ch = 0; ch < 4; ++ch)
                        if (ch < C) S[ch] += vrow[i * C + ch];
                }
                // g-image position of g-cell (cy, cx) of tile (ty, tx0 + t)
                uint16_t *dst = gimg + (size_t)(ty * gcs + cy) * g.gpitch + ((size_t)(tx0 + t) * gcs + cx) * C;
#pragma unroll
                for (int ch = 0; ch < 4; ++ch)
                    if (ch < C) dst[ch] = (uint16_t)S[ch];
            }
        }
        if (threadIdx.x < ns) {
            const int t = threadIdx.x;
            const unsigned long long n = (unsigned long long)TC * (unsigned long long)T;
            const unsigned long long S = S_s[t];
            uint64_t *keys = reinterpret_cast<uint64_t *>(a.ws + (uint64_t)f * g.ws_per_frame + g.ws_keys);
            keys[tile0 + t] = n * Q_s[t] - S * S;
        }
        __syncthreads();
    }
}

// Sum of an nb x nb block of g-cells (C u16 channel sums each; rows rowvals values apart) into S[0..C).
// With nb even and 4-byte alignment a pair of g-cells is C whole words whose halves map to compile-time
// channels, so each row is read with C * nb / 2 word loads that can all be in flight together.
template <int C>
__device__ __forceinline__ void gblock_sum(const uint16_t *p0, size_t rowvals, int nb, uint32_t *S) {
    const bool pairs = (nb % 2 == 0) && (reinterpret_cast<uintptr_t>(p0) & 3) == 0 && (rowvals & 1) == 0;
    for (int yy = 0; yy < nb; ++yy) {
        const uint16_t *p = p0 + (size_t)yy * rowvals;
        if (pairs) {
            const uint32_t *w = reinterpret_cast<const uint32_t *>(p);
#pragma unroll 4
            for (int pr = 0; pr < nb / 2; ++pr) {
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    const uint32_t x = w[pr * C + k];
                    S[(2 * k) % C] += x & 0xFFFFu;
                    S[(2 * k + 1) % C] += x >> 16;
                }
            }
        } else {
            for (int xx = 0; xx < nb; ++xx) {
#pragma unroll
                for (int ch = 0; ch < C; ++ch) S[ch] += p[xx * C + ch];
            }
        }
    }
}

// gblock_sum for a compile-time block width NB (g-cells per side): fully unrolled loads and adds.
template <int C, int NB>
__device__ __forceinline__ void gblock_sum_n(const uint16_t *p0, size_t rowvals, uint32_t *S) {
#pragma unroll
    for (int yy = 0; yy < NB; ++yy) {
        const uint16_t *p = p0 + (size_t)yy * rowvals;
#pragma unroll
        for (int xx = 0; xx < NB; ++xx)
#pragma unroll
            for (int ch = 0; ch < C; ++ch) S[ch] += p[xx * C + ch];
    }
}

// Block sum dispatched on the block width: unrolled for 1, 2, 4 and 8 g-cells, the generic loop otherwise.
// (Work items hand a warp cells of one grid size, so the branch is uniform across the warp.)
template <int C>
__device__ __forceinline__ void gblock_sum_any(const uint16_t *p0, size_t rowvals, int nb, uint32_t *S) {
    switch (nb) {
        case 1: gblock_sum_n<C, 1>(p0, rowvals, S); break;
        case 2: gblock_sum_n<C, 2>(p0, rowvals, S); break;
        case 4: gblock_sum_n<C, 4>(p0, rowvals, S); break;
        case 8: gblock_sum_n<C, 8>(p0, rowvals, S); break;
        default: gblock_sum<C>(p0, rowvals, nb, S); break;
    }
}

// ------------------------------------------------------------------------------------------------------
// k_emit: walks each record's payload in order, one thread per cell.  Element e of the payload lies in the
// region whose cumulative cell count passes e; the region-ordered tile list gives its tile, and the cell
// sum is assembled from the tile's (b_r/g)^2 g-cell sums in the g-image.  Consecutive threads therefore
// write consecutive record bytes and share one region, so a warp's lanes do equal work.
// ------------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_emit(const Geom g, const CallArgs a) {
    __shared__ uint32_t cstart[kMaxK + 1], tstart[kMaxK + 1];
    __shared__ uint64_t roff[kMaxK];
    const uint32_t f = blockIdx.y;
    uint8_t *rec = a.records + (uint64_t)f * (uint64_t)a.record_stride;
    if (threadIdx.x == 0) {
        const dp_pix_record_header *h = reinterpret_cast<const dp_pix_record_header *>(rec);
        uint32_t c = 0, t = 0;
        for (int r = 0; r < g.K; ++r) {
            const uint32_t n = min(h->count[r], g.ntiles);
            cstart[r] = c;
            tstart[r] = t;
            roff[r] = h->region_offset[r];
            c += n * (uint32_t)(g.cells_side[r] * g.cells_side[r]);
            t += n;
        }
        cstart[g.K] = c;
        tstart[g.K] = t;
    }
    __syncthreads();
    const uint32_t total = tstart[g.K] <= g.ntiles ? cstart[g.K] : 0u;
    const uint8_t *wsf = a.ws + (uint64_t)f * g.ws_per_frame;
    const uint32_t *tilelist = reinterpret_cast<const uint32_t *>(wsf + g.ws_tilelist);
    const uint16_t *gimg = reinterpret_cast<const uint16_t *>(wsf + g.ws_gsum);
    const int C = g.C, gcs = g.T / g.g;
    const size_t rowvals = (size_t)g.gpitch;
    const uint64_t frame = key_frame(a, f);
    const uint32_t sid = key_stream(a, f);
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        int r = 0;
        while (r + 1 < g.K && e >= cstart[r + 1]) ++r;
        const uint32_t local = e - cstart[r];
        const int cs = g.cells_side[r];
        const bool p2 = (cs & (cs - 1)) == 0;
        const int lcs = __ffs(cs) - 1;
        const uint32_t cells = (uint32_t)(cs * cs);
        const uint32_t k = p2 ? local >> (2 * lcs) : local / cells;
        const int c = (int)(local - k * cells);
        const int cy = p2 ? c >> lcs : c / cs, cx = c - cy * cs;
        const uint32_t tile = tilelist[tstart[r] + k];
        const uint32_t ty = tile / (uint32_t)g.GC, tx = tile - ty * (uint32_t)g.GC;
        const int nb = g.grid[r] / g.g;
        const uint16_t *p0 = gimg + ((size_t)(ty * gcs + cy * nb)) * rowvals + ((size_t)tx * gcs + (size_t)cx * nb) * C;
        uint32_t S[4] = {0u, 0u, 0u, 0u};
        switch (C) {
            case 1: gblock_sum_any<1>(p0, rowvals, nb, S); break;
            case 2: gblock_sum_any<2>(p0, rowvals, nb, S); break;
            case 3: gblock_sum_any<3>(p0, rowvals, nb, S); break;
            default: gblock_sum_any<4>(p0, rowvals, nb, S); break;
        }
        const uint32_t cell_idx = (ty * cs + cy) * (uint32_t)(g.GC * cs) + tx * cs + cx;
        uint8_t *dst = rec + roff[r] + (uint64_t)local * C * g.es;
        if (chk(dst, (uint64_t)C * g.es, a.records, a.records_bytes, a.status, kChkRecord))
            emit_cell(g, a, dst, S, r, cell_idx, frame, sid);
    }
}

template <typename K>
int grid_for(K kernel, size_t smem, uint32_t items, int threads = kThreads) {
    const int per_sm = launch_prep(reinterpret_cast<const void *>(kernel), threads, smem);
    const uint64_t cap = (uint64_t)per_sm * (uint64_t)sm_count();
    return (int)(items < cap ? items : cap);
}

// ------------------------------------------------------------------------------------------------------
// k_emit_recon: the emit and the reconstruction fused, for one (frame, tile-row segment) per item.
//  A. the segment's tile table (map byte, payload offset) and its block of the g-image (T/g rows of
//     ns*T/g g-cells) are fetched together with 16-byte loads into shared memory -- one round trip;
//  B. one thread per cell: the b_r-cell sum from the shared g-cells, noise, clip, the record element,
//     and the value a reconstruction would read back (Sec. VI-F) staged in shared memory;
//  C. the segment's output rows are written from the stage (seg_write.cuh) -- the record is never read back.
// Shared memory: g-cells [T/g][gseg_bytes] | stage | colinfo, sized by the launcher.
// ------------------------------------------------------------------------------------------------------
struct FusedShape {
    int seg;            // tiles per item
    int gseg_bytes;     // bytes per g-image row of a segment (multiple of 16)
    int stage_off, colinfo_off, smem;
};

template <int C, int kOutF32, int kThr>
__global__ void __launch_bounds__(kThr, 2048 / kThr / 2)
    k_emit_recon(const Geom g, const CallArgs a, uint8_t *out, int64_t out_frame_stride, int64_t out_pitch,
                 const FusedShape fs) {
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ SegTiles st;
    __shared__ uint8_t rlist[kSegMaxTiles];
    __shared__ int32_t rtile[kMaxK], rcell[kMaxK + 1], rcs[kMaxK], rnb[kMaxK], rlcs[kMaxK];
    constexpr int oes = kOutF32 ? 4 : 1;
    uint8_t *gseg = dyn;
    uint8_t *stage = dyn + fs.stage_off;
    uint32_t *colinfo = reinterpret_cast<uint32_t *>(dyn + fs.colinfo_off);
    const int T = g.T, gcs = T / g.g, seg = fs.seg;
    const int gsv = fs.gseg_bytes >> 1;  // u16 values per shared g-image row
    const uint32_t nseg = (uint32_t)((g.GC + seg - 1) / seg);
    const uint32_t items = a.n_frames * (uint32_t)g.GR * nseg;
    // the g-cells of an item's segment (T/g rows of ns*T/g g-cells) are copied into gseg with cp.async; the
    // copies for the next item are issued as soon as this item's cells are done, so that they arrive while
    // its rows are written
    auto fetch_gseg = [&](uint32_t it) {
        const uint32_t fr_ = it / nseg;
        const int ty_ = (int)(fr_ % g.GR), tx0_ = (int)(it % nseg) * seg;
        const int ns_ = min(seg, g.GC - tx0_);
        const uint8_t *wsf_ = a.ws + (uint64_t)(fr_ / g.GR) * g.ws_per_frame;
        const int nvec = (ns_ * gcs * C * 2 + 15) >> 4;  // 16-byte chunks per row (the row pitch covers the last)
        const uint8_t *src0 = wsf_ + g.ws_gsum + ((size_t)ty_ * gcs * g.gpitch + (size_t)tx0_ * gcs * C) * 2;
        for (int i = threadIdx.x; i < gcs * nvec; i += kThr) {
            const int row = i / nvec, v = i - row * nvec;
            cp_async16(gseg + row * fs.gseg_bytes + v * 16, src0 + (size_t)row * g.gpitch * 2 + 16 * v);
        }
    };
    if (blockIdx.x < items) fetch_gseg(blockIdx.x);
    for (uint32_t item = blockIdx.x; item < items; item += gridDim.x) {
        const uint32_t sg = item % nseg, fr = item / nseg;
        const int ty = (int)(fr % g.GR);
        const uint32_t f = fr / g.GR;
        const int tx0 = (int)sg * seg;
        const int ns = min(seg, g.GC - tx0);
        uint8_t *rec = a.records + (uint64_t)f * (uint64_t)a.record_stride;
        const uint8_t *wsf = a.ws + (uint64_t)f * g.ws_per_frame;
        // ---- A: tile table; the g-cells were fetched ahead ----
        if ((int)threadIdx.x < ns) {
            const int t = threadIdx.x;
            const uint32_t tile = (uint32_t)ty * g.GC + tx0 + t;
            int r = rec[g.map_offset + tile];
            if (r >= g.K) r = 0;
            st.reg[t] = r;
            st.b[t] = g.grid[r];
            st.cs[t] = g.cells_side[r];
            st.off[t] = reinterpret_cast<const uint32_t *>(wsf + g.ws_tileoff)[tile];
        }
        cp_async_wait_all();  // this thread's copies of the item's g-cells; the barrier publishes everyone's
        __syncthreads();
        seg_prefix_colinfo(st, ns, T, colinfo, threadIdx.x, kThr);  // warp 0 and all threads
        if (threadIdx.x >= 32 && threadIdx.x < 64) {
            // warp 1: the segment's tiles grouped by region (tile order kept), with region cell bases, so that
            // the cell loop below hands a warp cells of one grid size (equal work per lane)
            const int l = threadIdx.x - 32;
            const int r0 = l < ns ? st.reg[l] : -1, r1 = l + 32 < ns ? st.reg[l + 32] : -1;
            const unsigned lt = (1u << l) - 1u;
            int tb = 0, cb = 0;
            for (int r = 0; r < g.K; ++r) {
                const unsigned m0 = __ballot_sync(0xffffffffu, r0 == r), m1 = __ballot_sync(0xffffffffu, r1 == r);
                const int n0 = __popc(m0), n = n0 + __popc(m1);
                if (r0 == r) rlist[tb + __popc(m0 & lt)] = (uint8_t)l;
                if (r1 == r) rlist[tb + n0 + __popc(m1 & lt)] = (uint8_t)(l + 32);
                const int cs = g.cells_side[r];
                if (l == 0) {
                    rtile[r] = tb;
                    rcell[r] = cb;
                    rcs[r] = cs;
                    rnb[r] = g.grid[r] / g.g;
                    rlcs[r] = (cs & (cs - 1)) == 0 ? __ffs(cs) - 1 : -1;
                }
                tb += n;
                cb += n * cs * cs;
            }
            if (l == 0) rcell[g.K] = cb;
        }
        __syncthreads();
        // ---- B: cells, region by region ----
        const uint64_t frame = key_frame(a, f);
        const uint32_t sid = key_stream(a, f);
        const bool noisy = !g.noise_free && g.dtype != DP_PIX_REC_SUM_U32;
        const uint16_t *gs16 = reinterpret_cast<const uint16_t *>(gseg);
        for (int r = 0; r < g.K; ++r) {
            const int e0 = rcell[r], e1 = rcell[r + 1];
            if (e0 >= e1) continue;
            const int cs = rcs[r], lcs = rlcs[r], nb = rnb[r], tb = rtile[r];
            const uint32_t crow = (uint32_t)(g.GC * cs);  // cells per row of the frame's padded b_r-grid
            const float sigma = g.sigma_f[r], b2 = g.b2_f[r], inv_b2 = g.inv_b2_f[r];
            const PhiloxPrep pp = philox_prep((uint32_t)r | (sid << 8), (uint32_t)frame, (uint32_t)(frame >> 32),
                                              make_uint2((uint32_t)g.seed, (uint32_t)(g.seed >> 32)));
            // the item's cells go round robin over the threads (cell e to thread e mod kThr) across regions,
            // so that a region's few large cells do not all land on the first warp
            int e = e0 + (int)(((uint32_t)threadIdx.x + (uint32_t)kThr - (uint32_t)e0 % (uint32_t)kThr) % (uint32_t)kThr);
            for (; e < e1; e += kThr) {
                const int local = e - e0;
                int k, c, cy, cx;
                if (lcs >= 0) {  // power-of-two cells per tile side: shifts and masks (uniform across the warp)
                    k = local >> (2 * lcs);
                    c = local & ((1 << (2 * lcs)) - 1);
                    cy = c >> lcs;
                    cx = c & (cs - 1);
                } else {
                    k = local / (cs * cs);
                    c = local - k * cs * cs;
                    cy = c / cs;
                    cx = c - cy * cs;
                }
                const int t = rlist[tb + k];
                const int tx = tx0 + t;
                uint32_t S[4] = {0u, 0u, 0u, 0u};
                gblock_sum_any<C>(gs16 + (size_t)(cy * nb) * gsv + (size_t)(t * gcs + cx * nb) * C, (size_t)gsv, nb, S);
                const uint32_t cell_idx = (uint32_t)(ty * cs + cy) * crow + (uint32_t)(tx * cs + cx);
                float ov[4] = {0.f, 0.f, 0.f, 0.f};
                const uint4 words = noisy ? philox_finish_rk(pp, cell_idx, g.rkey) : make_uint4(0, 0, 0, 0);
                uint8_t *dst = rec + st.off[t] + (uint64_t)c * C * g.es;
                if (chk(dst, (uint64_t)C * g.es, a.records, a.records_bytes, a.status, kChkRecord))
                    emit_values(g, C, dst, S, words, sigma, b2, inv_b2, ov);
                const int si = st.base[t] + c;  // the stage keeps segment order for the row writer
                if (kOutF32) {
                    reinterpret_cast<float4 *>(stage)[si] = make_float4(ov[0], ov[1], ov[2], ov[3]);
                } else {
                    uint32_t pk = 0;
#pragma unroll
                    for (int ch = 0; ch < C; ++ch) pk |= to_u8(ov[ch]) << (8 * ch);
                    reinterpret_cast<uint32_t *>(stage)[si] = pk;
                }
            }
        }
        __syncthreads();
        if (item + gridDim.x < items) fetch_gseg(item + gridDim.x);  // gseg is free once the cells are done
        // ---- C: output rows ----
        const int x0 = tx0 * T;
        uint8_t *oframe = out + (uint64_t)f * (uint64_t)out_frame_stride;
        seg_write_rows<C, kOutF32>(st, colinfo, stage, ns, T, min(ns * T, g.N - x0), min(T, g.M - ty * T),
                                   oframe + (int64_t)(ty * T) * out_pitch + (int64_t)x0 * C * oes, out_pitch,
                                   threadIdx.x, kThr, oframe,
                                   (uint64_t)(g.M - 1) * (uint64_t)out_pitch + (uint64_t)g.N * C * oes, a.status);
        __syncthreads();
    }
}

template <int C, int kOutF32, int kThr>
cudaError_t launch_er(const Geom &g, const CallArgs &a, uint8_t *out, int64_t ofs, int64_t op, const FusedShape &fs,
                      int max_per_sm, cudaStream_t s) {
    auto kern = k_emit_recon<C, kOutF32, kThr>;

    const uint32_t items = a.n_frames * (uint32_t)g.GR * (uint32_t)((g.GC + fs.seg - 1) / fs.seg);
    int per_sm = launch_prep(reinterpret_cast<const void *>(kern), kThr, fs.smem);
    if (max_per_sm > 0 && max_per_sm < per_sm) per_sm = max_per_sm;
    const uint64_t cap = (uint64_t)per_sm * (uint64_t)sm_count();
    const int grid = (int)(items < cap ? items : cap);
    const char *name = kOutF32 ? "k_emit_recon_f32" : "k_emit_recon_u8";
    prof_begin(name, s);
    kern<<<grid, kThr, fs.smem, s>>>(g, a, out, ofs, op, fs);
    prof_end(name, s);
    return cudaGetLastError();
}

size_t seg_smem(const Geom &g, int bands_per_tile) {
    return (size_t)g.T * g.seg_rowstride + (size_t)g.seg_tiles * bands_per_tile * g.T * g.C * 2;
}


}  // namespace

cudaError_t launch_release(const Geom &g, const CallArgs &a, cudaStream_t s) {
    if (g.seg_tiles > kRelSegMax) return cudaErrorInvalidValue;
    const int buf_bytes = g.T * rel_rowstride(g.seg_tiles, g.T, g.C);
    const size_t smem = 2 * (size_t)buf_bytes;
    const uint32_t items = a.n_frames * (uint32_t)g.GR * (uint32_t)g.seg_per_row;
    prof_begin("k_release", s);
    switch (g.C) {
        case 1: k_release<1><<<grid_for(k_release<1>, smem, items, kRelThreads), kRelThreads, smem, s>>>(g, a); break;
        case 2: k_release<2><<<grid_for(k_release<2>, smem, items, kRelThreads), kRelThreads, smem, s>>>(g, a); break;
        case 3: k_release<3><<<grid_for(k_release<3>, smem, items, kRelThreads), kRelThreads, smem, s>>>(g, a); break;
        default: k_release<4><<<grid_for(k_release<4>, smem, items, kRelThreads), kRelThreads, smem, s>>>(g, a); break;
    }
    prof_end("k_release", s);
    return cudaGetLastError();
}

size_t release_smem(int T, int C, int S) { return 2 * (size_t)T * (size_t)rel_rowstride(S, T, C); }

cudaError_t launch_batch_release(const BatchEntry *tab, uint32_t n_img, uint32_t items, int T, int C, int S,
                                 cudaStream_t s) {
    if (S > kRelSegMax) return cudaErrorInvalidValue;
    const int buf_bytes = T * rel_rowstride(S, T, C);
    const size_t smem = 2 * (size_t)buf_bytes;
    prof_begin("k_batch_release", s);
    switch (C) {
        case 1: k_batch_release<1><<<grid_for(k_batch_release<1>, smem, items, kRelThreads), kRelThreads, smem, s>>>(tab, n_img, items, buf_bytes); break;
        case 2: k_batch_release<2><<<grid_for(k_batch_release<2>, smem, items, kRelThreads), kRelThreads, smem, s>>>(tab, n_img, items, buf_bytes); break;
        case 3: k_batch_release<3><<<grid_for(k_batch_release<3>, smem, items, kRelThreads), kRelThreads, smem, s>>>(tab, n_img, items, buf_bytes); break;
        default: k_batch_release<4><<<grid_for(k_batch_release<4>, smem, items, kRelThreads), kRelThreads, smem, s>>>(tab, n_img, items, buf_bytes); break;
    }
    prof_end("k_batch_release", s);
    return cudaGetLastError();
}

// Dynamic shared memory of the whole-warps-per-tile batch release for segments of S tiles (S divides the CTA's
// 8 warps): two buffers of T staged rows.  0: S does not apply (not 1, 2, 4 or 8, or past 200 KB).
size_t batch_tiles_smem(int T, int C, int S) {
    if ((S != 1 && S != 2 && S != 4 && S != 8) || T > kTilesThreads || S > kRelSegMax) return 0;
    const size_t smem = 2 * (size_t)T * (size_t)rel_rowstride(S, T, C);
    return smem <= 200 * 1024 ? smem : 0;
}

cudaError_t launch_batch_tiles(const BatchEntry *tab, uint32_t n_img, uint32_t items, int T, int C, int S,
                               cudaStream_t s) {
    const size_t smem = batch_tiles_smem(T, C, S);
    if (smem == 0) return cudaErrorInvalidValue;
    const int buf_bytes = T * rel_rowstride(S, T, C);
    const void *kern = nullptr;
    switch (C) {
        case 1: kern = reinterpret_cast<const void *>(k_batch_tiles<1>); break;
        case 2: kern = reinterpret_cast<const void *>(k_batch_tiles<2>); break;
        case 3: kern = reinterpret_cast<const void *>(k_batch_tiles<3>); break;
        case 4: kern = reinterpret_cast<const void *>(k_batch_tiles<4>); break;
        default: return cudaErrorInvalidValue;
    }
    const int per_sm = launch_prep(kern, kTilesThreads, smem);
    const uint64_t cap = (uint64_t)per_sm * (uint64_t)sm_count();
    const int grid = (int)(items < cap ? items : cap);
    prof_begin("k_batch_tiles", s);
    if (grid > 0) {
        void *args[] = {(void *)&tab, (void *)&n_img, (void *)&items, (void *)&buf_bytes};
        const cudaError_t e = cudaLaunchKernel(kern, dim3(grid), dim3(kTilesThreads), args, smem, s);
        if (e != cudaSuccess) {
            prof_end("k_batch_tiles", s);
            return e;
        }
    }
    prof_end("k_batch_tiles", s);
    return cudaGetLastError();
}

cudaError_t launch_batch_classify(const BatchEntry *tab, uint32_t n_img, uint32_t items, int T, int matte,
                                  cudaStream_t s) {
    const int es = matte ? 4 : 1;
    const int S = cls_seg_tiles(T, es);
    const int buf_bytes = T * rel_rowstride(S, T, es);
    const size_t smem = 2 * (size_t)buf_bytes;
    prof_begin("k_batch_classify", s);
    if (matte)
        k_batch_classify<true><<<grid_for(k_batch_classify<true>, smem, items), kThreads, smem, s>>>(tab, n_img, items,
                                                                                                      buf_bytes);
    else
        k_batch_classify<false><<<grid_for(k_batch_classify<false>, smem, items), kThreads, smem, s>>>(tab, n_img, items,
                                                                                                        buf_bytes);
    prof_end("k_batch_classify", s);
    return cudaGetLastError();
}

cudaError_t launch_tile_stats(const Geom &g, const CallArgs &a, cudaStream_t s) {
    const uint32_t items = a.n_frames * (uint32_t)g.GR * (uint32_t)g.seg_per_row;
    const cudaError_t fe = launch_tile_stats_fast(g, a, s);
    if (fe != cudaErrorNotSupported) return fe;
    if (g.var_onepass) {
        const size_t smem = seg_smem(g, g.T / g.g);
        const int grid = grid_for(k_tile_stats<true>, smem, items);
        prof_begin("k_tile_stats_gsum", s);
        k_tile_stats<true><<<grid, kThreads, smem, s>>>(g, a);
        prof_end("k_tile_stats_gsum", s);
    } else {
        const size_t smem = seg_smem(g, 0);
        const int grid = grid_for(k_tile_stats<false>, smem, items);
        prof_begin("k_tile_stats", s);
        k_tile_stats<false><<<grid, kThreads, smem, s>>>(g, a);
        prof_end("k_tile_stats", s);
    }
    return cudaGetLastError();
}

int gcd_int(int a, int b) {
    while (b) {
        const int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Fused emit + reconstruction when the output layout allows the vectorised write (16-byte aligned rows)
// and a segment fits shared memory; cudaErrorNotSupported (nothing launched) otherwise.  The segment is
// the largest whole number of tiles with at most fused_px pixel columns whose output bytes and g-image
// bytes both start on 16-byte boundaries.
cudaError_t launch_emit_recon(const Geom &g, const CallArgs &a, uint8_t *out, int64_t out_frame_stride,
                              int64_t out_pitch, int out_type, int out_align, int max_per_sm, cudaStream_t s) {
    const int oes = out_type == DP_PIX_OUT_F32 ? 4 : 1;
    const int trb = g.T * g.C * oes;
    if (!g.var_onepass || out_align != 16 || trb < 16 || (reinterpret_cast<uintptr_t>(a.ws) & 15) != 0)
        return cudaErrorNotSupported;
    const int gcs = g.T / g.g;
    const int gtb = gcs * g.C * 2;  // g-image bytes of one tile in one g-row
    const int s0 = 16 / gcd_int(trb, 16), s1 = 16 / gcd_int(gtb, 16);
    const int sm = s0 / gcd_int(s0, s1) * s1;  // segment tile-count granularity
    int csmax = 1;
    for (int r = 0; r < g.K; ++r) csmax = std::max(csmax, g.cells_side[r]);
    const int vb = oes == 4 ? 16 : 4;
    int px = g.fused_px;
    // few frames (a single frame, a small batch): smaller items until the launch covers the SMs -- each item's
    // chain of load, cells and rows is shorter as well
    while (px > 256 && (uint64_t)a.n_frames * g.GR * (uint64_t)((g.GC * g.T + px - 1) / px) < (uint64_t)sm_count())
        px >>= 1;
    int seg = std::max(1, std::min(kSegMaxTiles, std::min(px, kSegMaxPx) / g.T) / sm) * sm;
    FusedShape fs{};
    for (; seg >= sm; seg -= sm) {
        if (seg > kSegMaxTiles || seg * g.T > kSegMaxPx) continue;
        fs.seg = seg;
        fs.gseg_bytes = (seg * gtb + 15) / 16 * 16;
        fs.stage_off = gcs * fs.gseg_bytes;
        fs.colinfo_off = fs.stage_off + (seg * csmax * csmax * vb + 15) / 16 * 16;
        fs.smem = fs.colinfo_off + (colinfo_words(seg * g.T) * 4 + 15) / 16 * 16;
        if (fs.smem <= 64 * 1024) break;
    }
    if (seg < sm) return cudaErrorNotSupported;
    const int thr = g.fused_threads;
#define DPPIX_ER(CC, F)                                                                        \
    switch (thr) {                                                                             \
        case 96: return launch_er<CC, F, 96>(g, a, out, out_frame_stride, out_pitch, fs, max_per_sm, s);   \
        case 192: return launch_er<CC, F, 192>(g, a, out, out_frame_stride, out_pitch, fs, max_per_sm, s); \
        case 256: return launch_er<CC, F, 256>(g, a, out, out_frame_stride, out_pitch, fs, max_per_sm, s); \
        default: return launch_er<CC, F, 128>(g, a, out, out_frame_stride, out_pitch, fs, max_per_sm, s);  \
    }
    if (oes == 4) {
        switch (g.C) {
            case 1: DPPIX_ER(1, 1);
            case 2: DPPIX_ER(2, 1);
            case 3: DPPIX_ER(3, 1);
            default: DPPIX_ER(4, 1);
        }
    }
    switch (g.C) {
        case 1: DPPIX_ER(1, 0);
        case 2: DPPIX_ER(2, 0);
        case 3: DPPIX_ER(3, 0);
        default: DPPIX_ER(4, 0);
    }
#undef DPPIX_ER
}

cudaError_t launch_emit(const Geom &g, const CallArgs &a, cudaStream_t s) {
    // one wave of resident CTAs shared out over the frames, looping over the cells (a partial second wave
    // would leave its CTAs' whole shares to the end)
    const int per_sm = launch_prep(reinterpret_cast<const void *>(k_emit), kThreads, 0);
    int per_frame = std::max(1, per_sm * sm_count() / (int)a.n_frames);
    int maxcells = 1;
    for (int r = 0; r < g.K; ++r) maxcells = std::max(maxcells, g.cells_side[r] * g.cells_side[r]);
    const int need = (int)(((uint64_t)g.ntiles * maxcells + kThreads - 1) / kThreads);
    per_frame = std::max(1, std::min(per_frame, need));
    prof_begin("k_emit", s);
    k_emit<<<dim3(per_frame, a.n_frames), kThreads, 0, s>>>(g, a);
    prof_end("k_emit", s);
    return cudaGetLastError();
}

}  // namespace dppix
