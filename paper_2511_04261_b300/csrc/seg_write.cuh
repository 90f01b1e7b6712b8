// seg_write.cuh -- shared-memory segment machinery of the reconstruction (Sec. VI-F), used by the
// stand-alone reconstruction and by the fused release + reconstruction.
//
// A segment is ns consecutive tiles of one tile row.  Its cell values sit in shared memory ("stage"),
// tile by tile in row-major cell order (st.base[t] = first cell of tile t); colinfo maps each pixel column
// of the segment to (tile, cell column).  The write loop gives each thread 16-byte columns of the output
// rows: it assembles the vector once per cell band and stores it to every row of the band.
#pragma once

#include "common.cuh"

namespace dppix {

constexpr int kSegMaxTiles = 64;    // tiles of one segment
constexpr int kSegMaxPx = 2048;     // pixel columns of one segment

// The pixel-column map (colinfo) keeps entry i at word i + i / 32: the row writers' lanes read it at strides of
// 16 / C entries (one 16-byte chunk each), which without the gap every 32 words would pile up in a few banks.
__host__ __device__ constexpr int colinfo_words(int n) { return n + (n + 31) / 32; }
__device__ __forceinline__ int cix(int i) { return i + (i >> 5); }

__device__ __forceinline__ uint32_t to_u8(float v) { return __float2uint_rn(fminf(fmaxf(v, 0.0f), 255.0f)); }

struct SegTiles {
    int32_t reg[kSegMaxTiles], b[kSegMaxTiles], cs[kSegMaxTiles], base[kSegMaxTiles + 1];
    uint64_t off[kSegMaxTiles];
    uint32_t rowgrp[2][kMaxT / 32];  // row-group starts of the pattern writer, one mask per warp of tiles
    int32_t gbase[2][kSegMaxTiles];  // pattern writer: first staged cell of each tile's band in a row group
};

// ---- vector assembly ----------------------------------------------------------------------------------
// Output element i of a 16-byte chunk whose first element is channel P of local pixel 0 belongs to local
// pixel (P + i) / C, channel (P + i) % C -- compile-time once P and C are.
template <int C>
struct FastK {
    static constexpr int NPX8 = (C - 1 + 16) / C + 1;  // pixels a u8 chunk can touch (upper bound)
    static constexpr int NPXF = (C - 1 + 4) / C + 1;   // pixels an f32 chunk can touch (upper bound)
};

// Byte-permute selector for output word K of a chunk with phase P: byte i of the word is element
// e = P + 4K + i, i.e. channel e % C of pixel e / C, which for C >= 2 is one of the two adjacent pixels
// a = (P + 4K) / C and a + 1 (selector nibbles 0-3 and 4-7).
template <int C>
__host__ __device__ constexpr uint32_t word_sel(int e0) {
    uint32_t sel = 0;
    for (int i = 0; i < 4; ++i) {
        const int pix = (e0 + i) / C - e0 / C, ch = (e0 + i) % C;
        sel |= (uint32_t)(pix * 4 + ch) << (4 * i);
    }
    return sel;
}

template <int C, int P>
__device__ __forceinline__ uint4 build_u8(const uint32_t *pv) {
    uint32_t w[4];
    if (C == 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            w[k] = __byte_perm(__byte_perm(pv[4 * k], pv[4 * k + 1], 0x0040), __byte_perm(pv[4 * k + 2], pv[4 * k + 3], 0x0040),
                               0x5410);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int a = (P + 4 * k) / C;
            w[k] = __byte_perm(pv[a], pv[a + 1], word_sel<C>(P + 4 * k));
        }
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

template <int C, int P>
__device__ __forceinline__ uint4 build_f32(const float4 *pv) {
    float o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 v = pv[(P + i) / C];
        const int ch = (P + i) % C;
        o[i] = ch == 0 ? v.x : (ch == 1 ? v.y : (ch == 2 ? v.z : v.w));
    }
    return make_uint4(__float_as_uint(o[0]), __float_as_uint(o[1]), __float_as_uint(o[2]), __float_as_uint(o[3]));
}

// C = 3 with a runtime phase and no branch: word k of the chunk draws on pixels a and a + 1 with
// a = (p + 4k) / 3, which for p in {0, 1, 2} takes at most two values per word, so each word is one byte
// permute of two selected pixels with a selected selector (neighbouring lanes have different phases).
__device__ __forceinline__ uint4 build_u8_c3(int p, const uint32_t *pv) {
    constexpr uint32_t s00 = word_sel<3>(0), s01 = word_sel<3>(1), s02 = word_sel<3>(2);
    constexpr uint32_t s10 = word_sel<3>(4), s11 = word_sel<3>(5), s12 = word_sel<3>(6);
    constexpr uint32_t s20 = word_sel<3>(8), s21 = word_sel<3>(9), s22 = word_sel<3>(10);
    constexpr uint32_t s30 = word_sel<3>(12), s31 = word_sel<3>(13), s32 = word_sel<3>(14);
    const bool p0 = p == 0, p1 = p == 1;
    const uint32_t w0 = __byte_perm(pv[0], pv[1], p0 ? s00 : (p1 ? s01 : s02));
    const uint32_t w1 = p == 2 ? __byte_perm(pv[2], pv[3], s12) : __byte_perm(pv[1], pv[2], p0 ? s10 : s11);
    const uint32_t w2 = p0 ? __byte_perm(pv[2], pv[3], s20) : __byte_perm(pv[3], pv[4], p1 ? s21 : s22);
    const uint32_t w3 = __byte_perm(pv[4], pv[5], p0 ? s30 : (p1 ? s31 : s32));
    return make_uint4(w0, w1, w2, w3);
}

template <int C>
__device__ __forceinline__ uint4 build_u8_phase(int p, const uint32_t *pv) {
    if (C == 3) return build_u8_c3(p, pv);
    if (p == 0) return build_u8<C, 0>(pv);
    if (C > 1 && p == 1) return build_u8<C, (C > 1 ? 1 : 0)>(pv);
    if (C > 2 && p == 2) return build_u8<C, (C > 2 ? 2 : 0)>(pv);
    return build_u8<C, (C > 3 ? 3 : 0)>(pv);
}

template <int C>
__device__ __forceinline__ uint4 build_f32_phase(int p, const float4 *pv) {
    if (p == 0) return build_f32<C, 0>(pv);
    if (C > 1 && p == 1) return build_f32<C, (C > 1 ? 1 : 0)>(pv);
    if (C > 2 && p == 2) return build_f32<C, (C > 2 ? 2 : 0)>(pv);
    return build_f32<C, (C > 3 ? 3 : 0)>(pv);
}

// Cell prefix st.base[0..ns] (the first warp of the group, two tiles per lane; ns <= 64) and the
// pixel-column map; needs st.b and st.cs.  The group is threads tid = 0..nthr-1 (nthr a multiple of 32,
// whole warps).  Ends without a barrier.
__device__ __forceinline__ void seg_prefix_colinfo(SegTiles &st, int ns, int T, uint32_t *colinfo, int tid, int nthr) {
    if (tid < 32) {  // exclusive prefix of the tiles' cell counts, two tiles per lane
        const int l = tid;
        const int c0 = 2 * l < ns ? st.cs[2 * l] * st.cs[2 * l] : 0;
        const int c1 = 2 * l + 1 < ns ? st.cs[2 * l + 1] * st.cs[2 * l + 1] : 0;
        int incl = c0 + c1;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, off);
            if (l >= off) incl += v;
        }
        const int excl = incl - c0 - c1;
        if (2 * l <= ns) st.base[2 * l] = excl;
        if (2 * l + 1 <= ns) st.base[2 * l + 1] = excl + c0;
        if (l == 31) st.base[ns] = incl;  // the total (ns may be 64)
    }
    // pixel column -> (tile, cell column)
    const bool tp2 = (T & (T - 1)) == 0;
    const int lt = __ffs(T) - 1;
    for (int px = tid; px < ns * T; px += nthr) {
        const int t = tp2 ? px >> lt : px / T;
        const int b = st.b[t], pt = px - t * T;
        colinfo[cix(px)] = ((uint32_t)t << 16) | (uint32_t)((b & (b - 1)) == 0 ? pt >> (__ffs(b) - 1) : pt / b);
    }
}

// Subtracts n from k until k < n; returns how many times.
__device__ __forceinline__ int wrap_count(int &k, int n) {
    int c = 0;
    while (k >= n) {
        k -= n;
        ++c;
    }
    return c;
}

// Writes the jmax output rows of a segment whose first output byte is orow0 (16-byte aligned) and
// whose rows hold vpx pixels; stage holds the segment's cell values (packed u8 or float4).  Threads
// tid = 0..nthr-1 of the group share the work.  The rows are stored with the streaming hint (st.global.cs):
// nothing reads them back here, and their lines leave L2 while this issue-bound writer runs instead of being
// written back during the next, bandwidth-bound pass (64-frame clip step: 205.1 -> 199.4 us).
template <int C, int kOutF32>
__device__ void seg_write_rows(const SegTiles &st, const uint32_t *colinfo, const uint8_t *stage, int ns, int T, int vpx,
                               int jmax, uint8_t *orow0, int64_t out_pitch, int tid, int nthr,
                               const uint8_t *img = nullptr, uint64_t img_bytes = 0, int32_t *status = nullptr) {
    // bounds-checked build: every store must fall inside the image [img, img + img_bytes) when img is given
    auto ok = [&](const uint8_t *p, int n) { return img == nullptr || chk(p, n, img, img_bytes, status, kChkOutput); };
    constexpr int oes = kOutF32 ? 4 : 1;
    // write phase: thread = (16-byte column chunk, group of rows); no barrier until the next item
    const int row_bytes = vpx * C * oes;
    const int nch = (row_bytes + 15) >> 4;
    int RG = (nthr + nch - 1) / nch;  // about one (chunk, row group) unit per thread: long row runs per set-up
    RG = RG < 1 ? 1 : (RG > jmax ? jmax : RG);
    const int rpg = (jmax + RG - 1) / RG;
    const int last_px = ns * T - 1;
    constexpr int kElems = 16 / oes;
    constexpr int NPX = kOutF32 ? FastK<C>::NPXF : FastK<C>::NPX8;
    // units (chunk k, row group grp), w = grp * nch + k; consecutive threads take consecutive chunks so that warp
    // stores are contiguous, and (k, grp) follow w without a division per unit
    int k = tid % nch, grp = tid / nch;
    for (int w = tid; w < nch * RG; w += nthr, k += nthr, grp += wrap_count(k, nch)) {
        const int j0 = grp * rpg, j1 = min(jmax, j0 + rpg);
        if (j0 >= j1) continue;
        const int o = k << 4;
        const int e0 = o / oes;  // first output element of the chunk
        const int p = e0 % C;
        const int l0 = e0 / C;   // first pixel column
        // the chunk's real pixels lie in at most two tiles (a tile row has >= 16 bytes); trailing entries past
        // them are never used by the vector builder and are pointed at the last real pixel
        const int lastp = min((e0 + kElems - 1) / C, last_px);
        const uint32_t cl = colinfo[cix(lastp)];
        const int tA = colinfo[cix(min(l0, last_px))] >> 16;
        const int tB = cl >> 16;
        int cc[NPX];
        bool inB[NPX];
#pragma unroll
        for (int l = 0; l < NPX; ++l) {
            const uint32_t v = l0 + l <= lastp ? colinfo[cix(l0 + l)] : cl;
            cc[l] = (int)(v & 0xFFFFu);
            inB[l] = (int)(v >> 16) != tA;
        }
        const int bA = st.b[tA], bB = st.b[tB], csA = st.cs[tA], csB = st.cs[tB];
        const bool full = o + 16 <= row_bytes;
        // cell bands followed incrementally: band of row j, and the row where it ends.  Every lane walks the
        // same rows (the store loop never diverges); a lane rebuilds its vector only where its band changes.
        int bandA = (bA & (bA - 1)) == 0 ? j0 >> (__ffs(bA) - 1) : j0 / bA;
        int bandB = (bB & (bB - 1)) == 0 ? j0 >> (__ffs(bB) - 1) : j0 / bB;
        int endA = (bandA + 1) * bA, endB = (bandB + 1) * bB;
        const int b0A = st.base[tA], b0B = st.base[tB];
        auto build = [&]() -> uint4 {
            const int baseA = b0A + bandA * csA, baseB = b0B + bandB * csB;
            if (kOutF32) {
                float4 pv[NPX];
#pragma unroll
                for (int l = 0; l < NPX; ++l) pv[l] = reinterpret_cast<const float4 *>(stage)[(inB[l] ? baseB : baseA) + cc[l]];
                return build_f32_phase<C>(p, pv);
            } else {
                uint32_t pv[NPX];
#pragma unroll
                for (int l = 0; l < NPX; ++l) pv[l] = reinterpret_cast<const uint32_t *>(stage)[(inB[l] ? baseB : baseA) + cc[l]];
                return build_u8_phase<C>(p, pv);
            }
        };
        uint4 vec = build();
        uint8_t *dst = orow0 + (int64_t)j0 * out_pitch + o;
        int j = j0;
        if (full && (bA & 3) == 0 && (bB & 3) == 0 && (j0 & 3) == 0) {
            // bands of multiples of 4 rows: the band check once per 4 rows
            for (; j + 4 <= j1; j += 4, dst += 4 * out_pitch) {
                if (j == endA || j == endB) {
                    if (j == endA) {
                        ++bandA;
                        endA += bA;
                    }
                    if (j == endB) {
                        ++bandB;
                        endB += bB;
                    }
                    vec = build();
                }
                if (ok(dst, 16) && ok(dst + 3 * out_pitch, 16)) {
                    __stcs(reinterpret_cast<uint4 *>(dst), vec);
                    __stcs(reinterpret_cast<uint4 *>(dst + out_pitch), vec);
                    __stcs(reinterpret_cast<uint4 *>(dst + 2 * out_pitch), vec);
                    __stcs(reinterpret_cast<uint4 *>(dst + 3 * out_pitch), vec);
                }
            }
        }
        for (; j < j1; ++j, dst += out_pitch) {
            if (j == endA || j == endB) {
                if (j == endA) {
                    ++bandA;
                    endA += bA;
                }
                if (j == endB) {
                    ++bandB;
                    endB += bB;
                }
                vec = build();
            }
            if (!ok(dst, full ? 16 : row_bytes - o)) {
                // bounds-checked build: a store outside the image is skipped
            } else if (full) {
                __stcs(reinterpret_cast<uint4 *>(dst), vec);
            } else {
                for (int i = 0; o + i < row_bytes; ++i) {
                    const uint32_t wv = i < 4 ? vec.x : (i < 8 ? vec.y : (i < 12 ? vec.z : vec.w));
                    dst[i] = (uint8_t)(wv >> (8 * (i & 3)));
                }
            }
        }
    }
}

// Writes the jmax output rows of a segment whose rows may start at any byte alignment (f32 rows at 4-byte
// alignment): per row, the aligned middle in 16-byte chunks, each assembled from the cells it covers for
// that row (rows do not share vectors, their alignments differ), and the head and tail (< 16 bytes each)
// one element at a time.
template <int C, int kOutF32>
__device__ void seg_write_rows_any(const SegTiles &st, const uint32_t *colinfo, const uint8_t *stage, int ns, int T,
                                   int vpx, int jmax, uint8_t *orow0, int64_t out_pitch, int tid, int nthr) {
    constexpr int oes = kOutF32 ? 4 : 1;
    constexpr int kElems = 16 / oes;
    constexpr int NPX = kOutF32 ? FastK<C>::NPXF : FastK<C>::NPX8;
    const int row_bytes = vpx * C * oes;
    const int last_px = ns * T - 1;
    const int maxch = (row_bytes >> 4) + 1;
    for (int w = tid; w < jmax * maxch; w += nthr) {
        const int j = w / maxch, k = w - j * maxch;
        uint8_t *row = orow0 + (int64_t)j * out_pitch;
        const int h = min((int)((16u - (uint32_t)(reinterpret_cast<uintptr_t>(row) & 15u)) & 15u), row_bytes);
        if (k >= ((row_bytes - h) >> 4)) continue;
        const int o = h + 16 * k;
        const int e0 = o / oes;
        const int p = e0 % C;
        const int l0 = e0 / C;
        const int lastp = min((e0 + kElems - 1) / C, last_px);
        const uint32_t cl = colinfo[cix(lastp)];
        const int tA = colinfo[cix(min(l0, last_px))] >> 16;
        const int tB = cl >> 16;
        const int baseA = st.base[tA] + (j / st.b[tA]) * st.cs[tA];
        const int baseB = st.base[tB] + (j / st.b[tB]) * st.cs[tB];
        uint4 vec;
        if (kOutF32) {
            float4 pv[NPX];
#pragma unroll
            for (int l = 0; l < NPX; ++l) {
                const uint32_t v = l0 + l <= lastp ? colinfo[cix(l0 + l)] : cl;
                const int idx = ((int)(v >> 16) != tA ? baseB : baseA) + (int)(v & 0xFFFFu);
                pv[l] = reinterpret_cast<const float4 *>(stage)[idx];
            }
            vec = build_f32_phase<C>(p, pv);
        } else {
            uint32_t pv[NPX];
#pragma unroll
            for (int l = 0; l < NPX; ++l) {
                const uint32_t v = l0 + l <= lastp ? colinfo[cix(l0 + l)] : cl;
                const int idx = ((int)(v >> 16) != tA ? baseB : baseA) + (int)(v & 0xFFFFu);
                pv[l] = reinterpret_cast<const uint32_t *>(stage)[idx];
            }
            vec = build_u8_phase<C>(p, pv);
        }
        *reinterpret_cast<uint4 *>(row + o) = vec;
    }
    // heads and tails: at most 2 * kElems - 2 elements per row
    constexpr int kEdge = 2 * kElems;
    for (int w = tid; w < jmax * kEdge; w += nthr) {
        const int j = w / kEdge, i = w - j * kEdge;
        uint8_t *row = orow0 + (int64_t)j * out_pitch;
        const int h = min((int)((16u - (uint32_t)(reinterpret_cast<uintptr_t>(row) & 15u)) & 15u), row_bytes);
        const int tail0 = h + (((row_bytes - h) >> 4) << 4);
        const int nh = h / oes, nt = (row_bytes - tail0) / oes;
        int e;
        if (i < nh) e = i;
        else if (i - nh < nt) e = tail0 / oes + (i - nh);
        else continue;
        const int px = e / C, ch = e - px * C;
        const uint32_t v = colinfo[cix(px)];
        const int t = (int)(v >> 16);
        const int idx = st.base[t] + (j / st.b[t]) * st.cs[t] + (int)(v & 0xFFFFu);
        if (kOutF32) {
            const float4 f = reinterpret_cast<const float4 *>(stage)[idx];
            reinterpret_cast<float *>(row)[e] = ch == 0 ? f.x : (ch == 1 ? f.y : (ch == 2 ? f.z : f.w));
        } else {
            row[e] = (uint8_t)(reinterpret_cast<const uint32_t *>(stage)[idx] >> (8 * ch));
        }
    }
}

// ---- rows of any alignment, u8 output, through row patterns --------------------------------------------
// The rows of a segment fall into groups inside which every tile stays in one cell band: a group starts at
// row j when j is a multiple of some tile's grid.  Each group's output row is built once in shared memory
// and then stored to each row of the group with 16-byte stores at that row's own byte alignment (the pattern
// read as a 32-byte window and funnel-shifted), the head and tail bytes one at a time.

// Marks the group starts of the segment's rows (bit j of rowgrp[w][j / 32], w = the warp of tiles 0..31 or
// 32..63).  Threads 0..63 of the group take part; the caller's next barrier publishes the masks.
__device__ __forceinline__ void seg_row_groups(SegTiles &st, int ns, int T, int tid) {
    if (tid < 64) {
        uint32_t m[kMaxT / 32] = {0u, 0u, 0u, 0u};
        if (tid < ns) {
            const int b = st.b[tid];
            for (int j = 0; j < T; j += b) m[j >> 5] |= 1u << (j & 31);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int q = 0; q < kMaxT / 32; ++q) m[q] |= __shfl_xor_sync(0xffffffffu, m[q], off);
        if ((tid & 31) == 0)
#pragma unroll
            for (int q = 0; q < kMaxT / 32; ++q) st.rowgrp[tid >> 5][q] = m[q];
    }
}

// First group start after row j, or jmax.
__device__ __forceinline__ int seg_next_group(const SegTiles &st, int j, int jmax) {
    for (int q = (j + 1) >> 5; q < kMaxT / 32; ++q) {
        uint32_t m = st.rowgrp[0][q] | st.rowgrp[1][q];
        if (q == ((j + 1) >> 5)) m &= ~0u << ((j + 1) & 31);
        if (m != 0u) return min(jmax, 32 * q + __ffs(m) - 1);
    }
    return jmax;
}

// Band base of tile t for the row group starting at row j, into the buffer that the group after the current
// one (which reads buffer buf) reads.
__device__ __forceinline__ void st_gbase_next(SegTiles &st, int buf, int t, int j) {
    st.gbase[buf ^ 1][t] = st.base[t] + (j / st.b[t]) * st.cs[t];
}

// Bytes h .. h + 15 of the 32 bytes lo:hi (h in 0..15).
__device__ __forceinline__ uint4 window16(const uint4 &lo, const uint4 &hi, int h) {
    const int sh = (h & 3) * 8;
    switch (h >> 2) {
        case 0: return make_uint4(__funnelshift_r(lo.x, lo.y, sh), __funnelshift_r(lo.y, lo.z, sh),
                                  __funnelshift_r(lo.z, lo.w, sh), __funnelshift_r(lo.w, hi.x, sh));
        case 1: return make_uint4(__funnelshift_r(lo.y, lo.z, sh), __funnelshift_r(lo.z, lo.w, sh),
                                  __funnelshift_r(lo.w, hi.x, sh), __funnelshift_r(hi.x, hi.y, sh));
        case 2: return make_uint4(__funnelshift_r(lo.z, lo.w, sh), __funnelshift_r(lo.w, hi.x, sh),
                                  __funnelshift_r(hi.x, hi.y, sh), __funnelshift_r(hi.y, hi.z, sh));
        default: return make_uint4(__funnelshift_r(lo.w, hi.x, sh), __funnelshift_r(hi.x, hi.y, sh),
                                   __funnelshift_r(hi.y, hi.z, sh), __funnelshift_r(hi.z, hi.w, sh));
    }
}

// Writes the jmax u8 output rows (vpx pixels each, first output byte orow0, any alignment) of a segment whose
// cell values are staged (packed u8) and whose row groups seg_row_groups marked.  pat: two pattern buffers,
// pat_stride bytes apart, each of at least 16 * (ceil(vpx C / 16) + 1) bytes (16-byte aligned).  Threads
// tid = 0..nthr-1 of the group share the work; one barrier per row group.  In the bounds-checked build every
// store must fall inside the image [img, img + img_bytes) when img is given.
template <int C>
__device__ void seg_write_rows_pat(SegTiles &st, const uint32_t *colinfo, const uint8_t *stage, int ns, int T,
                                   int vpx, int jmax, uint8_t *orow0, int64_t out_pitch, uint8_t *pat, int pat_stride,
                                   int tid, int nthr, const uint8_t *img = nullptr, uint64_t img_bytes = 0,
                                   int32_t *status = nullptr) {
    auto ok = [&](const uint8_t *p, int n) { return img == nullptr || chk(p, n, img, img_bytes, status, kChkOutput); };
    constexpr int NPX = FastK<C>::NPX8;
    const int row_bytes = vpx * C;
    const int nch = (row_bytes + 15) >> 4;
    const int last_px = ns * T - 1;
    const uint32_t *stage32 = reinterpret_cast<const uint32_t *>(stage);
    int buf = 0;
    for (int ja = 0; ja < jmax;) {
        const int jb = seg_next_group(st, ja, jmax);
        uint8_t *P = pat + buf * pat_stride;
        // each tile's band base for the next group, published by this group's barrier (the first group's
        // bands are the tiles' first ones)
        if (tid < ns && jb < jmax) st_gbase_next(st, buf, tid, jb);
        const int32_t *gb = ja == 0 ? st.base : st.gbase[buf];
        // the group's row (the band of row ja in every tile), one 16-byte chunk per thread step
        for (int k = tid; k < nch; k += nthr) {
            const int e0 = k << 4;
            const int p = e0 % C, l0 = e0 / C;
            const int lastp = min((e0 + 15) / C, last_px);
            const uint32_t cl = colinfo[cix(lastp)];
            const int tA = colinfo[cix(min(l0, last_px))] >> 16, tB = cl >> 16;
            const int baseA = gb[tA], baseB = gb[tB];
            uint32_t pv[NPX];
#pragma unroll
            for (int l = 0; l < NPX; ++l) {
                const uint32_t v = l0 + l <= lastp ? colinfo[cix(l0 + l)] : cl;
                pv[l] = stage32[((int)(v >> 16) != tA ? baseB : baseA) + (int)(v & 0xFFFFu)];
            }
            *reinterpret_cast<uint4 *>(P + 16 * k) = build_u8_phase<C>(p, pv);
        }
        __syncthreads();
        // rows ja .. jb-1: unit k < nch of a row is its k-th aligned 16-byte chunk, unit nch its head and tail
        const int U = nch + 1;
        int jr = tid / U, k = tid - jr * U;
        for (int w = tid; w < (jb - ja) * U; w += nthr, k += nthr, jr += wrap_count(k, U)) {
            uint8_t *row = orow0 + (int64_t)(ja + jr) * out_pitch;
            const int h = min((int)((16u - (uint32_t)(reinterpret_cast<uintptr_t>(row) & 15u)) & 15u), row_bytes);
            const int nfull = (row_bytes - h) >> 4;
            if (k < nfull) {
                const uint4 lo = *reinterpret_cast<const uint4 *>(P + 16 * k);
                const uint4 hi = *reinterpret_cast<const uint4 *>(P + 16 * k + 16);
                if (ok(row + h + 16 * k, 16)) *reinterpret_cast<uint4 *>(row + h + 16 * k) = window16(lo, hi, h);
            } else if (k == nch) {
                for (int i = 0; i < h; ++i)
                    if (ok(row + i, 1)) row[i] = P[i];
                for (int i = h + 16 * nfull; i < row_bytes; ++i)
                    if (ok(row + i, 1)) row[i] = P[i];
            }
        }
        buf ^= 1;  // the next group builds into the other buffer; the barrier above already ordered this one
        ja = jb;
    }
}

}  // namespace dppix
