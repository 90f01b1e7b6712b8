// k_batch_stream.cu -- streaming kernels of the ragged batch: the tile classification of every image from
// its mask or matte (Alg. 3 steps 5-6), and the release of every image with, optionally, its pixelized
// image (Alg. 3 steps 7-17 and the restoring steps of Sec. VI-F), each one launch over all images' items.
//
// The rows of a batch image start at any byte alignment (N * C bytes per row, N arbitrary).  A thread owns
// one 16-byte column chunk of an item and walks the item's rows: it loads the aligned 16-byte granule under
// its chunk, takes the next granule from its neighbour lane (the last lane of a warp loads it itself), and
// shifts the pair by the row's misalignment, so that its registers hold the same columns in every row.
// Nothing is staged on the way in: each source byte is read once, by one 16-byte load of one lane.
#include <algorithm>

#include "seg_write.cuh"

namespace dppix {
namespace {

constexpr int kBsThreads = 256;
constexpr int kBsMaxSeg = 32;         // tiles of one release item
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint4 ld_nc16(const uint8_t *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }

__device__ __forceinline__ uint4 shfl_down4(const uint4 &v) {
    return make_uint4(__shfl_down_sync(kFull, v.x, 1), __shfl_down_sync(kFull, v.y, 1), __shfl_down_sync(kFull, v.z, 1),
                      __shfl_down_sync(kFull, v.w, 1));
}
__device__ __forceinline__ uint4 shfl_up4(const uint4 &v) {
    return make_uint4(__shfl_up_sync(kFull, v.x, 1), __shfl_up_sync(kFull, v.y, 1), __shfl_up_sync(kFull, v.z, 1),
                      __shfl_up_sync(kFull, v.w, 1));
}
__device__ __forceinline__ uint32_t word4(const uint4 &v, int q) { return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w)); }

// ------------------------------------------------------------------------------------------------------
// k_bcls_stream: one item per (image, tile row).  Work unit = (granule k of the row, block of kRows rows):
// the unit's kRows loads are issued together, then counted.  Granule k of an image row holds pixels of at
// most two tiles (T * ES >= 32), tile tA or tA + 1, so a unit counts into two registers and adds them to the
// item's per-tile counters once.  A sample is simple when the mask byte is nonzero (ES = 1) or when not
// alpha >= thr (ES = 4, f32 matte).  Mirrored columns past the right edge all fall in the last tile and are
// counted from their source columns.  A tile is simple (region 0) iff 2 * #simple > its samples, a tie going
// to complex (region 1).
// ------------------------------------------------------------------------------------------------------
constexpr int kRows = 8;

template <int ES>
__global__ void __launch_bounds__(kBsThreads) k_bcls_stream(const BatchEntry *__restrict__ tab, uint32_t n_img,
                                                             uint32_t items) {
    extern __shared__ uint32_t cnt_s[];  // one counter per tile of the item's tile row
    for (uint32_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int i = batch_find(tab, n_img, item, 0);
        const Geom &g = tab[i].g;
        const int T = g.T, M = g.M, N = g.N, GC = g.GC, pad = g.pad_mode;
        const uint8_t *src = tab[i].a.src;
        const int64_t pitch = tab[i].a.src_pitch;
        const float thr = g.matte_thr;
        const int ty = (int)(item - tab[i].base[0]);
        const bool strict = pad == DP_PIX_PAD_NONE;
        const int hv = strict ? min(T, M - ty * T) : T;
        for (int t = threadIdx.x; t < GC; t += blockDim.x) cnt_s[t] = 0u;
        __syncthreads();
        const int rb = N * ES;               // bytes of a source row
        const int nch = (rb + 15) / 16 + 1;  // aligned granules a row can touch
        const int nblk = (hv + kRows - 1) / kRows;
        for (int u = threadIdx.x; u < nch * nblk; u += blockDim.x) {
            const int blk = u / nch, k = u - blk * nch;
            const int tA = min(max(0, 16 * k - 15) / ES / T, GC - 1);
            const int bnd = (tA + 1) * T;  // pixels from here on belong to tile tA + 1
            uint4 v[kRows];
            int xb[kRows];
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                const int j = blk * kRows + r;
                v[r] = make_uint4(0u, 0u, 0u, 0u);
                xb[r] = 1 << 30;  // no pixel
                if (j < hv) {
                    const int sy = reflect_idx(ty * T + j, M, pad);
                    const uintptr_t rowp = reinterpret_cast<uintptr_t>(src + (int64_t)sy * pitch);
                    const int o = (int)(rowp & 15u);
                    if (16 * k < o + rb) {  // the granule holds bytes of the row
                        v[r] = ld_nc16(reinterpret_cast<const uint8_t *>(rowp - (uintptr_t)o) + 16 * k);
                        xb[r] = 16 * k - o;  // byte of the row at the granule's first byte (may be negative)
                    }
                }
            }
            uint32_t cA = 0, cB = 0;
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                if (ES == 4) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int x = (xb[r] >> 2) + q;
                        const bool simple = !(__uint_as_float(word4(v[r], q)) >= thr);
                        if (x >= 0 && x < N && simple) {
                            if (x >= bnd) ++cB; else ++cA;
                        }
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int x = xb[r] + q;
                        const bool simple = ((word4(v[r], q >> 2) >> (8 * (q & 3))) & 0xFFu) != 0u;
                        if (x >= 0 && x < N && simple) {
                            if (x >= bnd) ++cB; else ++cA;
                        }
                    }
                }
            }
            if (cA) atomicAdd(&cnt_s[tA], cA);
            if (cB) atomicAdd(&cnt_s[tA + 1], cB);
        }
        if (!strict) {  // mirrored columns past the right edge: all in the last tile
            const int pc = GC * T - N;
            uint32_t cP = 0;
            for (int u = threadIdx.x; u < T * pc; u += blockDim.x) {
                const int j = u / pc, p = u - j * pc;
                const int sy = reflect_idx(ty * T + j, M, pad), sx = reflect_idx(N + p, N, pad);
                const uint8_t *q = src + (int64_t)sy * pitch + (int64_t)sx * ES;
                const bool simple = ES == 4 ? !(*reinterpret_cast<const float *>(q) >= thr) : *q != 0;
                cP += simple ? 1u : 0u;
            }
            if (cP) atomicAdd(&cnt_s[GC - 1], cP);
        }
        __syncthreads();
        uint8_t *map = tab[i].a.records + g.map_offset + (uint64_t)ty * GC;
        for (int t = threadIdx.x; t < GC; t += blockDim.x) {
            const int wv = strict ? min(T, N - t * T) : T;
            map[t] = (2u * cnt_s[t] > (uint32_t)hv * (uint32_t)wv) ? 0 : 1;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------------------
// k_brel_stream: one item per (image, tile row, segment of S tiles).
//  1. Columns: lane L < 31 of warp w owns the item's columns [16k, 16k + 16), k = 31 w + L (bytes of the
//     segment, realigned as above; lane 31 only loads the granule lane 30 needs), issues the loads of four
//     rows at a time, and adds every row into sixteen 16-bit column sums.  When a row ends a cell band of the tile that owns
//     some of its columns (the chunk meets at most two tiles, A and B: T * C >= 16), those sums go to V[band]
//     (shared memory, one u16 per segment column) and restart.  Mirrored columns past the right edge come from
//     their source columns, gathered into shared memory by the whole block first (a right-edge item has at most
//     (T - 1) C of them per row); without padding (Alg. 1 partial cells) they, and rows past the bottom edge,
//     add 0.
//  2. Cells: one thread per cell adds its b columns of its band per channel -- the exact cell sums -- and
//     draws the noise, clips and writes the record values (as the single-image release), keeping the value
//     a reconstruction reads back (Sec. VI-F) in shared memory.
//  3. Image (kRecon): the same chunks, now per output row: each lane builds its 16 bytes from the cell values
//     once per cell band and stores them at the output row's own alignment (the shift needs the previous
//     chunk: lane L of warp w owns chunk 31 w + L - 1 and lane 0 only feeds lane 1); the edge granules of the
//     segment are written byte by byte.
// ------------------------------------------------------------------------------------------------------
struct BrelShape {
    int S;          // tiles per item
    int NB;         // cell bands per tile of the finest grid (T / b_min)
    int vpitch;     // u16 values per band row of V: S * T * C rounded up to 8, + 16
    int csq;        // cells per tile of the finest grid
    int cellv_off;  // byte offset of the staged cell values
    int edge_off;   // byte offset of the mirrored columns of a right-edge item
    int edge_pitch; // bytes per row of them: (T - 1) * C + 16 rounded up to 16, + 16
    int smem;
};

template <int C>
__device__ __forceinline__ void add_bytes(uint32_t (&acc)[8], const uint4 &w) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t x = word4(w, q);
        acc[2 * q] += __byte_perm(x, 0u, 0x4240);      // bytes 0 and 2 of the word: columns 4q, 4q + 2
        acc[2 * q + 1] += __byte_perm(x, 0u, 0x4341);  // bytes 1 and 3: columns 4q + 1, 4q + 3
    }
}

// Column sums of the chunk in column order: word m holds columns 2m (low half) and 2m + 1.
__device__ __forceinline__ void natural_pairs(const uint32_t (&acc)[8], uint32_t (&nw)[8]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        nw[2 * q] = __byte_perm(acc[2 * q], acc[2 * q + 1], 0x5410);
        nw[2 * q + 1] = __byte_perm(acc[2 * q], acc[2 * q + 1], 0x7632);
    }
}

constexpr int kRelRows = 4;  // rows whose loads a release thread has in flight together

template <int C, bool kRecon>
__global__ void __launch_bounds__(kBsThreads, 3) k_brel_stream(const BatchEntry *__restrict__ tab, uint32_t n_img,
                                                             uint32_t items, const BrelShape sh) {
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ int32_t tb_s[kBsMaxSeg], tcs_s[kBsMaxSeg], treg_s[kBsMaxSeg], tbase_s[kBsMaxSeg + 1];
    __shared__ uint32_t toff_s[kBsMaxSeg];
    uint16_t *V = reinterpret_cast<uint16_t *>(dyn);
    uint32_t *cellv = reinterpret_cast<uint32_t *>(dyn + sh.cellv_off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int i = batch_find(tab, n_img, item, 2);
        const Geom &g = tab[i].g;
        const CallArgs &a = tab[i].a;
        const int T = g.T, TC = T * C, M = g.M, N = g.N, GC = g.GC, pad = g.pad_mode;
        const int nseg = (GC + sh.S - 1) / sh.S;
        const uint32_t local = item - tab[i].base[2];
        const int ty = (int)(local / (uint32_t)nseg), tx0 = (int)(local - (uint32_t)ty * (uint32_t)nseg) * sh.S;
        const int ns = min(sh.S, GC - tx0);
        const int x0 = tx0 * T;
        const int SB = ns * TC;                      // bytes of a segment row
        const int VB = min(ns * T, N - x0) * C;      // of them inside the image
        const bool strict = pad == DP_PIX_PAD_NONE;
        const int hv = strict ? min(T, M - ty * T) : T;
        uint8_t *rec = a.records;
        if ((int)threadIdx.x < ns) {
            const int t = threadIdx.x;
            const uint32_t tile = (uint32_t)ty * GC + tx0 + t;
            int r = rec[g.map_offset + tile];
            if (r >= g.K) r = 0;
            treg_s[t] = r;
            tb_s[t] = g.grid[r];
            tcs_s[t] = g.cells_side[r];
            toff_s[t] = reinterpret_cast<const uint32_t *>(a.ws + g.ws_tileoff)[tile];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc_c = 0;
            for (int t = 0; t < ns; ++t) {
                tbase_s[t] = acc_c;
                acc_c += tcs_s[t] * tcs_s[t];
            }
            tbase_s[ns] = acc_c;
        }

        // ---- 0: the mirrored columns of a right-edge item, gathered by the whole block: row j's columns
        //      [VB, SB) at edge[j * edge_pitch + (c - VBa)], VBa = VB rounded down to 16 (without padding: 0)
        const int VBa = VB & ~15;
        uint8_t *edge = dyn + sh.edge_off;
        if (VB < SB) {
            const int nb = SB - VBa;
            for (int u = threadIdx.x; u < T * nb; u += blockDim.x) {
                const int j = u / nb, c = VBa + (u - j * nb);
                uint8_t v = 0;
                if (c >= VB && !strict) {
                    const int px = c / C, chn = c - px * C;
                    const int sy = reflect_idx(ty * T + j, M, pad), sx = reflect_idx(x0 + px, N, pad);
                    v = a.frames[(int64_t)sy * g.pitch + (int64_t)sx * C + chn];
                }
                edge[j * sh.edge_pitch + (c - VBa)] = v;
            }
            __syncthreads();
        }

        // ---- 1: column sums per cell band ----
        {
            // lanes 0..30 of warp w own chunks 31 w + lane; lane 31 loads chunk 31 w + 31 for lane 30 only
            const int c0 = 16 * (31 * warp + lane);
            const bool act = lane < 31 && c0 < SB;
            int tA = 0, tB = 0, split = 16;
            if (act) {
                tA = c0 / TC;
                tB = min(ns - 1, (c0 + 15) / TC);
                split = tB == tA ? 16 : (tA + 1) * TC - c0;
            }
            const int bA = act ? tb_s[tA] : T, bB = act ? tb_s[tB] : T;
            int remA = bA, remB = bB, bandA = 0, bandB = 0;
            uint32_t acc[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
            const uint8_t *fbase = a.frames + (int64_t)x0 * C;
            const int64_t pitch = g.pitch;
            // rows in batches of kRelRows; the next batch's loads are issued before this one is consumed, so
            // that up to 2 kRelRows loads per lane are in flight
            uint4 lo[kRelRows], nlo[kRelRows];
            int o[kRelRows], no[kRelRows];
            auto issue = [&](int jb, uint4 (&L)[kRelRows], int (&Oo)[kRelRows]) {
#pragma unroll
                for (int r = 0; r < kRelRows; ++r) {
                    const int j = jb + r;
                    L[r] = make_uint4(0u, 0u, 0u, 0u);
                    Oo[r] = 0;
                    if (j < hv) {
                        const int sy = reflect_idx(ty * T + j, M, pad);
                        const uintptr_t rowp = reinterpret_cast<uintptr_t>(fbase + (int64_t)sy * pitch);
                        Oo[r] = (int)(rowp & 15u);
                        if (c0 < Oo[r] + VB) L[r] = ld_nc16(reinterpret_cast<const uint8_t *>(rowp - (uintptr_t)Oo[r]) + c0);
                    }
                }
            };
            issue(0, lo, o);
            for (int j0 = 0; j0 < T; j0 += kRelRows) {
                if (j0 + kRelRows < T) issue(j0 + kRelRows, nlo, no);
#pragma unroll
                for (int r = 0; r < kRelRows; ++r) {
                    const int j = j0 + r;
                    if (j >= T) break;
                    if (j < hv) {
                        const uint4 hi = shfl_down4(lo[r]);
                        uint4 w = o[r] ? window16(lo[r], hi, o[r]) : lo[r];
                        // columns past the image take their mirrored samples (gathered above; none without
                        // padding); columns past the segment are summed too but never read
                        if (act && VB < SB && c0 + 16 > VB) {
                            const uint4 e = *reinterpret_cast<const uint4 *>(edge + j * sh.edge_pitch + (c0 - VBa));
                            const int nv = VB - c0;  // bytes of the chunk inside the image (may be <= 0)
                            uint32_t ww[4] = {w.x, w.y, w.z, w.w};
                            const uint32_t ee[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const int keep = nv - 4 * q;  // leading bytes of word q from the image row
                                const uint32_t m = keep >= 4 ? 0xFFFFFFFFu : (keep <= 0 ? 0u : (1u << (8 * keep)) - 1u);
                                ww[q] = (ww[q] & m) | (ee[q] & ~m);
                            }
                            w = make_uint4(ww[0], ww[1], ww[2], ww[3]);
                        }
                        add_bytes<C>(acc, w);
                    }
                    const bool endA = --remA == 0, endB = tB != tA && --remB == 0;
                    // most rows end no band in any lane of the warp: one vote skips the flush for all of them
                    if (__any_sync(kFull, act && (endA || endB)) && act && (endA || endB)) {
                        uint32_t nw[8];
                        natural_pairs(acc, nw);
                        if (split == 16) {  // one tile: the whole chunk ends its band
                            uint4 *dst = reinterpret_cast<uint4 *>(V + (size_t)bandA * sh.vpitch + c0);
                            dst[0] = make_uint4(nw[0], nw[1], nw[2], nw[3]);
                            dst[1] = make_uint4(nw[4], nw[5], nw[6], nw[7]);
#pragma unroll
                            for (int q = 0; q < 8; ++q) acc[q] = 0u;
                        } else {
                            uint16_t *va = V + (size_t)bandA * sh.vpitch + c0, *vb = V + (size_t)bandB * sh.vpitch + c0;
#pragma unroll
                            for (int m = 0; m < 8; ++m) {
                                const int cl = 2 * m, ch = 2 * m + 1;  // the word's two columns
                                if (endA) {
                                    if (ch < split) *reinterpret_cast<uint32_t *>(va + cl) = nw[m];
                                    else if (cl < split) va[cl] = (uint16_t)(nw[m] & 0xFFFFu);
                                }
                                if (endB) {
                                    if (cl >= split) *reinterpret_cast<uint32_t *>(vb + cl) = nw[m];
                                    else if (ch >= split) vb[ch] = (uint16_t)(nw[m] >> 16);
                                }
                            }
#pragma unroll
                            for (int q = 0; q < 4; ++q) {  // restart the columns whose band ended
                                const int cLo = 4 * q, cHi = 4 * q + 2;  // acc[2q]; acc[2q + 1]: cLo + 1, cHi + 1
                                const bool z0 = (endA && cLo < split) || (endB && cLo >= split);
                                const bool z1 = (endA && cHi < split) || (endB && cHi >= split);
                                const bool z2 = (endA && cLo + 1 < split) || (endB && cLo + 1 >= split);
                                const bool z3 = (endA && cHi + 1 < split) || (endB && cHi + 1 >= split);
                                acc[2 * q] &= (z0 ? 0u : 0xFFFFu) | (z1 ? 0u : 0xFFFF0000u);
                                acc[2 * q + 1] &= (z2 ? 0u : 0xFFFFu) | (z3 ? 0u : 0xFFFF0000u);
                            }
                        }
                    }
                    if (endA) {
                        remA = bA;
                        ++bandA;
                    }
                    if (endB) {
                        remB = bB;
                        ++bandB;
                    }
                }
#pragma unroll
                for (int r = 0; r < kRelRows; ++r) {
                    lo[r] = nlo[r];
                    o[r] = no[r];
                }
            }
        }
        __syncthreads();

        // ---- 2: cells ----
        {
            const int ncells = tbase_s[ns];
            const uint64_t frame = a.frame_idx0;
            const uint32_t sid = a.stream_id;
            const bool noisy = !g.noise_free && g.dtype != DP_PIX_REC_SUM_U32;
            int t = 0;
            for (int e = threadIdx.x; e < ncells; e += blockDim.x) {
                while (e >= tbase_s[t + 1]) ++t;
                const int r = treg_s[t], b = tb_s[t], cs = tcs_s[t];
                const int c = e - tbase_s[t];
                const int cy = c / cs, cx = c - cy * cs;
                uint32_t S[4] = {0u, 0u, 0u, 0u};
                const uint16_t *vp = V + (size_t)cy * sh.vpitch + t * TC + cx * b * C;
                for (int q = 0; q < b; ++q) {
#pragma unroll
                    for (int chn = 0; chn < C; ++chn) S[chn] += vp[q * C + chn];
                }
                float sigma = g.sigma_f[r], b2 = g.b2_f[r], ib2 = g.inv_b2_f[r];
                int n = b * b;
                if (strict) {  // Alg. 1's partial cell: its h x w samples in the frame, scale R m / (h w eps_r)
                    const int h = max(0, min(b, hv - cy * b));
                    const int w = max(0, min(b, N - (tx0 + t) * T - cx * b));
                    n = h * w;
                    if (n > 0 && n < b * b) {
                        b2 = (float)n;
                        ib2 = 0.0f;
                        sigma = __fdiv_rn(g.sigma_f[r] * g.b2_f[r], (float)n);
                    }
                }
                uint8_t *dst = rec + toff_s[t] + (uint64_t)c * C * g.es;
                float ov[4] = {0.f, 0.f, 0.f, 0.f};
                if (!chk(dst, (uint64_t)C * g.es, a.records, a.records_bytes, a.status, kChkRecord)) {
                    // bounds-checked build: a write outside the record is skipped
                } else if (n == 0) {  // wholly outside the frame: no sample, stored as 0
#pragma unroll
                    for (int chn = 0; chn < C; ++chn) {
                        if (g.es == 4) reinterpret_cast<uint32_t *>(dst)[chn] = 0u;
                        else dst[chn] = 0;
                    }
                } else {
                    const uint32_t cell_idx =
                        (uint32_t)(ty * cs + cy) * (uint32_t)(GC * cs) + (uint32_t)((tx0 + t) * cs + cx);
                    const uint4 words = noisy ? cell_noise_words(g.seed, cell_idx, (uint32_t)r, sid, frame)
                                              : make_uint4(0u, 0u, 0u, 0u);
                    emit_values(g, C, dst, S, words, sigma, b2, ib2, ov);
                }
                if (kRecon) {
                    uint32_t pk = 0;
#pragma unroll
                    for (int chn = 0; chn < C; ++chn) pk |= to_u8(ov[chn]) << (8 * chn);
                    cellv[t * sh.csq + c] = pk;
                }
            }
        }

        // ---- 3: the pixelized rows ----
        if (kRecon && tab[i].out != nullptr) {
            __syncthreads();
            constexpr int NPX = FastK<C>::NPX8;
            uint8_t *obase = tab[i].out + (int64_t)x0 * C;
            const int64_t opitch = tab[i].out_pitch;
            const int ck = 16 * (31 * warp + lane - 1);  // this lane's chunk (lane 0: the previous warp's last)
            const int lastpx = ns * T - 1;
            const int cc = max(ck, 0);
            const int p = cc % C, l0 = cc / C;
            const int tAo = min(l0, lastpx) / T, tBo = min(tAo + 1, ns - 1);
            uint32_t meta[(NPX + 3) / 4];
#pragma unroll
            for (int q = 0; q < (NPX + 3) / 4; ++q) meta[q] = 0u;
#pragma unroll
            for (int l = 0; l < NPX; ++l) {
                const int px = min(l0 + l, lastpx);
                const int tt = px / T;
                const uint32_t m = (uint32_t)((px - tt * T) / tb_s[tt]) | (tt != tAo ? 0x80u : 0u);
                meta[l >> 2] |= m << (8 * (l & 3));
            }
            const int bA = tb_s[tAo], bB = tb_s[tBo], csA = tcs_s[tAo], csB = tcs_s[tBo];
            int nextA = 0, nextB = 0, bandA = -1, bandB = -1;
            uint4 vec = make_uint4(0u, 0u, 0u, 0u);
            const int jmax = min(T, M - ty * T);
            for (int j = 0; j < jmax; ++j) {
                bool need = false;
                if (j == nextA) {
                    ++bandA;
                    nextA += bA;
                    need = true;
                }
                if (j == nextB) {
                    ++bandB;
                    nextB += bB;
                    need = true;
                }
                if (need) {
                    const int baseA = tAo * sh.csq + bandA * csA, baseB = tBo * sh.csq + bandB * csB;
                    uint32_t pv[NPX];
#pragma unroll
                    for (int l = 0; l < NPX; ++l) {
                        const uint32_t m = (meta[l >> 2] >> (8 * (l & 3))) & 0xFFu;
                        pv[l] = cellv[((m & 0x80u) ? baseB : baseA) + (int)(m & 0x7Fu)];
                    }
                    vec = build_u8_phase<C>(p, pv);
                }
                const uintptr_t orow = reinterpret_cast<uintptr_t>(obase + (int64_t)(ty * T + j) * opitch);
                const int o2 = (int)(orow & 15u);
                const uint4 prev = shfl_up4(vec);
                if (lane > 0) {
                    const int f0 = ck - o2;  // segment column of the granule's first byte
                    if (f0 + 16 > 0 && f0 < VB) {
                        const uint4 d = o2 ? window16(prev, vec, 16 - o2) : vec;
                        uint8_t *gp = reinterpret_cast<uint8_t *>(orow - (uintptr_t)o2) + ck;
                        const uint64_t img_bytes = (uint64_t)(M - 1) * (uint64_t)opitch + (uint64_t)N * C;
                        if (!chk(gp + max(f0, 0) - f0, (uint64_t)(min(f0 + 16, VB) - max(f0, 0)), tab[i].out,
                                 img_bytes, a.status, kChkOutput)) {
                            // bounds-checked build: a store outside the image is skipped
                        } else if (f0 >= 0 && f0 + 16 <= VB) {
                            __stcs(reinterpret_cast<uint4 *>(gp), d);
                        } else {
#pragma unroll
                            for (int q = 0; q < 16; ++q)
                                if (f0 + q >= 0 && f0 + q < VB) gp[q] = (uint8_t)(word4(d, q >> 2) >> (8 * (q & 3)));
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace

// Streaming classification applies when a granule's pixels meet at most two tiles.
bool batch_classify_stream_ok(int T, int matte) { return T * (matte ? 4 : 1) >= 32; }

cudaError_t launch_batch_classify_stream(const BatchEntry *tab, uint32_t n_img, uint32_t items, int matte,
                                         uint32_t max_gc, cudaStream_t s) {
    const size_t smem = (size_t)max_gc * 4;
    const void *kern = matte ? reinterpret_cast<const void *>(k_bcls_stream<4>)
                             : reinterpret_cast<const void *>(k_bcls_stream<1>);
    const int per_sm = launch_prep(kern, kBsThreads, smem);
    const int grid = (int)std::min<uint64_t>(items, (uint64_t)per_sm * sm_count());
    prof_begin("k_bcls_stream", s);
    if (grid > 0) {
        if (matte) k_bcls_stream<4><<<grid, kBsThreads, smem, s>>>(tab, n_img, items);
        else k_bcls_stream<1><<<grid, kBsThreads, smem, s>>>(tab, n_img, items);
    }
    prof_end("k_bcls_stream", s);
    return cudaGetLastError();
}

// Item shape of the streaming release for tiles of side T, C channels, finest grid b_min and at most
// max_seg tiles per item; S = 0 when the kernel does not apply (a chunk meeting three tiles, or the band
// sums of one tile past the shared memory it may use).  recon_ok: the cell values of an item fit too.
BatchStreamShape batch_release_stream_shape(int T, int C, int b_min, int max_seg) {
    BatchStreamShape r{};
    const int TC = T * C, NB = T / b_min;
    if (TC < 16 || C < 1 || C > 4) return r;
    int S = std::min({kBsMaxSeg, max_seg, (16 * (kBsThreads / 32 * 31 - 2)) / TC, (28672 / NB - 24) / TC});
    if (S < 1) return r;
    r.S = S;
    r.NB = NB;
    r.vpitch = (S * TC + 7) / 8 * 8 + 16;  // 16-byte aligned band rows, 16 values of slack for the last chunk
    r.csq = NB * NB;
    r.edge_pitch = ((T - 1) * C + 16 + 15) / 16 * 16 + 16;
    r.edge_off = (int)(((size_t)NB * r.vpitch * 2 + 15) / 16 * 16);
    const size_t edge = (size_t)T * r.edge_pitch;
    if (edge > 32 * 1024) return BatchStreamShape{};  // mirrored columns past what an item may stage
    r.cellv_off = r.edge_off + (int)edge;
    const size_t cellv = (size_t)S * r.csq * 4;
    r.recon_ok = cellv <= 48 * 1024 ? 1 : 0;
    r.smem = r.cellv_off + (r.recon_ok ? (int)cellv : 0);
    return r;
}

cudaError_t launch_batch_release_stream(const BatchEntry *tab, uint32_t n_img, uint32_t items, int C,
                                        const BatchStreamShape &bs, int recon, cudaStream_t s) {
    BrelShape sh{bs.S, bs.NB, bs.vpitch, bs.csq, bs.cellv_off, bs.edge_off, bs.edge_pitch, bs.smem};
    if (!recon) sh.smem = bs.cellv_off;
    const void *kern = nullptr;
#define DPPIX_BRS_KERN(CC, RR) kern = reinterpret_cast<const void *>(k_brel_stream<CC, RR>)
    switch (C * 2 + (recon ? 1 : 0)) {
        case 2: DPPIX_BRS_KERN(1, false); break;
        case 3: DPPIX_BRS_KERN(1, true); break;
        case 4: DPPIX_BRS_KERN(2, false); break;
        case 5: DPPIX_BRS_KERN(2, true); break;
        case 6: DPPIX_BRS_KERN(3, false); break;
        case 7: DPPIX_BRS_KERN(3, true); break;
        case 8: DPPIX_BRS_KERN(4, false); break;
        case 9: DPPIX_BRS_KERN(4, true); break;
        default: return cudaErrorInvalidValue;
    }
#undef DPPIX_BRS_KERN
    const int per_sm = launch_prep(kern, kBsThreads, sh.smem);
    const int grid = (int)std::min<uint64_t>(items, (uint64_t)per_sm * sm_count());
    const char *name = recon ? "k_brel_stream_recon" : "k_brel_stream";
    prof_begin(name, s);
    if (grid > 0) {
        void *args[] = {(void *)&tab, (void *)&n_img, (void *)&items, (void *)&sh};
        const cudaError_t e = cudaLaunchKernel(kern, dim3(grid), dim3(kBsThreads), args, sh.smem, s);
        if (e != cudaSuccess) {
            prof_end(name, s);
            return e;
        }
    }
    prof_end(name, s);
    return cudaGetLastError();
}

}  // namespace dppix
