// k_frame.cu -- per-frame kernels: region-map finalisation and variance-quantile ranking.
//
// One CTA per frame.  Given the frame's u8 tile -> region map, the CTA counts tiles per region, lays out
// the region-major payload (Table IV: mu'_G then mu'_Gs, generalised to K regions), writes each tile's
// payload byte offset to the workspace, writes the tile-row index and the 512-byte header into the
// record.  The rank kernel first builds the map from the per-tile variance keys (exact integers) by
// sorting the packed (key, tile index) values: warp runs in registers, then merges in shared memory.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace dppix {

namespace {

constexpr int kFrameThreads = 1024;

// Per-region tile counters packed into 64-bit words: FB-bit fields, 64 / FB per word, NWORDS words (enough
// for the frame's K regions).  Fields never carry into each other while every count stays below 2^FB.
template <int FB, int NWORDS>
struct PackedCounts {
    static constexpr int FPW = 64 / FB;
    static constexpr int NW = NWORDS;
    static constexpr uint64_t kMask = FB == 64 ? ~0ull : (1ull << FB) - 1ull;
    uint64_t w[NW];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int q = 0; q < NW; ++q) w[q] = 0ull;
    }
    __device__ __forceinline__ uint32_t get(int r) const {
        uint64_t x = 0ull;
#pragma unroll
        for (int q = 0; q < NW; ++q)
            if (r / FPW == q) x = w[q];
        return (uint32_t)((x >> (FB * (r % FPW))) & kMask);
    }
    __device__ __forceinline__ void inc(int r) {
#pragma unroll
        for (int q = 0; q < NW; ++q)
            if (r / FPW == q) w[q] += 1ull << (FB * (r % FPW));
    }
};

// Exclusive scan of packed counters across the block (fields add independently).  warp_tot: smem [32][4].
template <int NW>
__device__ __forceinline__ void block_excl_scan_packed(const uint64_t (&v)[NW], uint64_t (&excl)[NW], uint64_t (&total)[NW],
                                       uint64_t (*warp_tot)[4]) {
    static_assert(NW <= 4, "warp_tot holds four words per warp");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
    uint64_t incl[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) incl[q] = v[q];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            const uint64_t t = __shfl_up_sync(0xffffffffu, incl[q], off);
            if (lane >= off) incl[q] += t;
        }
    }
    if (lane == 31) {
#pragma unroll
        for (int q = 0; q < NW; ++q) warp_tot[warp][q] = incl[q];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            uint64_t x = lane < nwarps ? warp_tot[lane][q] : 0ull;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint64_t t = __shfl_up_sync(0xffffffffu, x, off);
                if (lane >= off) x += t;
            }
            if (lane < nwarps) warp_tot[lane][q] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        const uint64_t base = warp > 0 ? warp_tot[warp - 1][q] : 0ull;
        excl[q] = base + incl[q] - v[q];
        total[q] = warp_tot[nwarps - 1][q];
    }
    __syncthreads();
}

struct FinalizeSmem {
    uint64_t warp_tot[32][4];
    uint64_t roff[kMaxK];
    uint64_t tile_bytes[kMaxK];
    uint32_t count[kMaxK];
    uint32_t tstart[kMaxK];  // first position of region r's tiles in the region-ordered tile list
    dp_pix_record_header hdr;
};
static_assert(offsetof(FinalizeSmem, hdr) % 16 == 0, "the header is zeroed in 16-byte words");

// Lays out the record of frame f from its map (see file comment); also writes the workspace's per-tile
// payload offsets and the tile ids in record order (region-major, row-major).  map_s: the map in shared
// memory, or in global memory for frames of more than kFinalizeSmemTiles tiles; a label >= K counts as 0
// (k_finalize has flagged it).  FB: bits per packed region counter (the frame has fewer than 2^FB tiles).
template <int FB, int NWORDS>
__device__ __forceinline__ void finalize_frame_t(const Geom &g, const CallArgs &a, uint32_t f, const uint8_t *map_s, bool write_map,
                                 FinalizeSmem &sm) {
    using PC = PackedCounts<FB, NWORDS>;
    const uint32_t n = g.ntiles;
    const uint32_t chunk = (n + blockDim.x - 1) / blockDim.x;
    const uint32_t c0 = min(n, threadIdx.x * chunk), c1 = min(n, c0 + chunk);
    if (threadIdx.x < kHeaderBytes / 16) reinterpret_cast<uint4 *>(&sm.hdr)[threadIdx.x] = make_uint4(0, 0, 0, 0);
    PC cnt, excl, total;
    cnt.clear();
    for (uint32_t i = c0; i < c1; ++i) {
        const uint32_t r = map_s[i];
        cnt.inc(r < (uint32_t)g.K ? r : 0u);
    }
    block_excl_scan_packed<PC::NW>(cnt.w, excl.w, total.w, sm.warp_tot);

    uint8_t *rec = a.records + (uint64_t)f * (uint64_t)a.record_stride;
    const int tr = threadIdx.x;
    if (tr < g.K) {  // region tr: its payload offset follows the regions before it (16-byte aligned each)
        uint64_t off = g.payload_offset;
        uint32_t tacc = 0;
        for (int q = 0; q < tr; ++q) {
            const uint64_t cq = (uint64_t)g.cells_side[q];
            const uint32_t nq = total.get(q);
            off = align16_u64(off + (uint64_t)nq * cq * cq * (uint64_t)g.C * (uint64_t)g.es);
            tacc += nq;
        }
        const uint64_t cs = (uint64_t)g.cells_side[tr];
        const uint64_t tb = cs * cs * (uint64_t)g.C * (uint64_t)g.es;
        const uint32_t tot = total.get(tr);
        sm.tile_bytes[tr] = tb;
        sm.roff[tr] = off;
        sm.count[tr] = tot;
        sm.tstart[tr] = tacc;
        dp_pix_record_header &h = sm.hdr;  // zeroed above, ordered by the scan's barriers
        h.grid[tr] = g.grid[tr];
        h.eps[tr] = g.eps[tr];
        h.sigma[tr] = g.sigma[tr];
        h.count[tr] = tot;
        h.region_offset[tr] = off;
        if (tr == g.K - 1) h.total_bytes = align16_u64(off + (uint64_t)tot * tb);
    }
    if (tr == 32) {  // the scalar fields, from another warp
        dp_pix_record_header &h = sm.hdr;
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
        h.map_offset = g.map_offset;
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
    PC run = excl;
    uint32_t ty = c0 / (uint32_t)g.GC, tx = c0 - ty * (uint32_t)g.GC;
    for (uint32_t i = c0; i < c1; ++i) {
        if (tx == 0) {
            for (int r = 0; r < g.K; ++r) rowidx[ty * g.K + r] = run.get(r);
        }
        uint32_t r = map_s[i];
        if (r >= (uint32_t)g.K) r = 0;
        const uint32_t ri = run.get(r);
        run.inc(r);
        if (++tx == (uint32_t)g.GC) {
            tx = 0;
            ++ty;
        }
        tileoff[i] = (uint32_t)(sm.roff[r] + (uint64_t)ri * sm.tile_bytes[r]);
        tilelist[sm.tstart[r] + ri] = i;  // tiles in record (payload) order
    }
    if (write_map) {
        uint8_t *map = rec + g.map_offset;
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
            const uint8_t r = map_s[i];
            map[i] = r < (uint32_t)g.K ? r : 0;
        }
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

__device__ __forceinline__ void finalize_frame(const Geom &g, const CallArgs &a, uint32_t f, const uint8_t *map_s, bool write_map,
                               FinalizeSmem &sm) {
    if (g.ntiles < 65536u) {
        if (g.K <= 4) finalize_frame_t<16, 1>(g, a, f, map_s, write_map, sm);
        else finalize_frame_t<16, 2>(g, a, f, map_s, write_map, sm);
    } else {
        finalize_frame_t<32, 4>(g, a, f, map_s, write_map, sm);
    }
}

// Map given by the caller (tile labels) or already written into the record by k_classify.
__global__ void __launch_bounds__(kFrameThreads, 1) k_finalize(const Geom g, const CallArgs a, int from_labels) {
    extern __shared__ __align__(16) uint8_t dyn[];
    FinalizeSmem &sm = *reinterpret_cast<FinalizeSmem *>(dyn);
    uint8_t *map_s = dyn + sizeof(FinalizeSmem);
    const uint32_t f = blockIdx.x;
    const uint8_t *src = from_labels ? a.src + (uint64_t)f * (uint64_t)a.src_frame_stride
                                     : a.records + (uint64_t)f * (uint64_t)a.record_stride + g.map_offset;
    const bool smem_map = g.ntiles <= (uint32_t)kFinalizeSmemTiles;
    for (uint32_t i = threadIdx.x; i < g.ntiles; i += blockDim.x) {
        uint8_t r = src[i];
        if (r >= (uint32_t)g.K) {
            raise_status(a.status, DP_PIX_E_DEVICE, 0x100u | r);
            r = 0;
        }
        if (smem_map) map_s[i] = r;
    }
    __syncthreads();
    finalize_frame(g, a, f, smem_map ? map_s : src, from_labels != 0, sm);
}

// Batch: one CTA per image (map written by k_batch_classify, or caller labels).
__global__ void __launch_bounds__(kFrameThreads, 1) k_batch_finalize(const BatchEntry *tab, uint32_t n_img) {
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
        const bool smem_map = g.ntiles <= (uint32_t)kFinalizeSmemTiles;
        for (uint32_t t = threadIdx.x; t < g.ntiles; t += blockDim.x) {
            uint8_t r = src[t];
            if (r >= (uint32_t)g.K) {
                raise_status(a.status, DP_PIX_E_DEVICE, 0x100u | r);
                r = 0;
            }
            if (smem_map) map_s[t] = r;
        }
        __syncthreads();
        finalize_frame(g, a, 0u, smem_map ? map_s : src, from_labels, sm);
        __syncthreads();
    }
}

// VARIANCE classes: tiles ranked by (key, index) ascending get class q = floor(K * rank / n).  The packed
// values key << idx_bits | index are unique, so the ranking is a total order.

__device__ __forceinline__ uint64_t min_u64(uint64_t x, uint64_t y) { return x < y ? x : y; }
__device__ __forceinline__ uint64_t max_u64(uint64_t x, uint64_t y) { return x < y ? y : x; }

// Sorts, ascending, the 1024 E values v held by the CTA's 1024 threads (thread t holds positions
// t E .. t E + E - 1) and hands them back the same way.
//  1. Each warp sorts its run of 32 E values with a bitonic network in registers: compare distances below
//     E inside a thread, the others by lane shuffles; every run ends ascending.
//  2. The 32 runs are merged pairwise in five rounds through shared memory s (1024 E values): a value's
//     place in the merged run is its place in its own run plus the number of partner-run values before it,
//     found by a binary search.  A value of the left run counts partner values below it, one of the right
//     run those not above it, so equal values (the padding) keep distinct places.
template <int E>
__device__ __forceinline__ void block_merge_sort(uint64_t (&v)[E], uint64_t *s) {
    constexpr int L0 = 32 * E, NP = kFrameThreads * E;
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 2; k <= L0; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j >= E; j >>= 1) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = t * E + e;
                const uint64_t o = __shfl_xor_sync(0xffffffffu, v[e], j / E);
                const bool asc = k == L0 || (i & k) == 0;
                v[e] = (((i & j) == 0) == asc) ? min_u64(o, v[e]) : max_u64(o, v[e]);
            }
        }
#pragma unroll
        for (int j = E / 2; j >= 1; j >>= 1) {
            if (j > (k >> 1)) continue;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if (e & j) continue;
                const bool asc = k == L0 || ((t * E + e) & k) == 0;
                const uint64_t lo = v[e], hi = v[e + j];
                v[e] = asc ? min_u64(lo, hi) : max_u64(lo, hi);
                v[e + j] = asc ? max_u64(lo, hi) : min_u64(lo, hi);
            }
        }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) s[t * E + e] = v[e];
    __syncthreads();
#pragma unroll 1
    for (int L = L0; L < NP; L <<= 1) {
        const int i0 = t * E;                     // the thread's positions share one run
        const int run = i0 / L, pos0 = i0 & (L - 1);
        const bool left = (run & 1) == 0;
        const uint64_t *p = s + (size_t)(run ^ 1) * L;
        int c[E];
#pragma unroll
        for (int e = 0; e < E; ++e) c[e] = 0;
#pragma unroll 1
        for (int step = L >> 1; step >= 1; step >>= 1) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const uint64_t x = p[c[e] + step - 1];
                if (x < v[e] || (!left && x == v[e])) c[e] += step;
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const uint64_t x = p[c[e]];
            if (x < v[e] || (!left && x == v[e])) ++c[e];
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) s[(run & ~1) * L + pos0 + e + c[e]] = v[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = s[i0 + e];
    }
}

// Boundary selection without a full sort.  The class boundaries are the values of ranks
// t_q = ceil((q + 1) n / K), q < K - 1.  One histogram over a log-scale digit of the packed value (the
// position of its top bit, then the 8 bits below it: monotone in the value, and fine-grained where
// variance keys crowd) locates each t_q's bin and its rank inside the bin; the bin's values are then
// collected and the one of that rank found by counting.  Frames whose boundary bins hold more than
// kSelCap values (nearly equal keys) take the sort instead.
constexpr int kSelBins = 16384;
constexpr int kSelCap = 128;

__device__ __forceinline__ uint32_t log_digit(uint64_t v) {
    if (v == 0ull) return 0u;
    const int e = 63 - __clzll((long long)v);  // <= 62: packed values stay below 2^63
    const uint32_t m = e >= 8 ? (uint32_t)(v >> (e - 8)) & 255u : (uint32_t)(v << (8 - e)) & 255u;
    return (uint32_t)e * 256u + m;
}

struct SelSmem {
    uint32_t hist[kSelBins];
    uint64_t lst[kMaxK - 1][kSelCap];
    uint64_t bnd[kMaxK - 1];
    uint32_t target[kMaxK - 1], bin[kMaxK - 1], rank[kMaxK - 1], count[kMaxK - 1], fill[kMaxK - 1];
    uint32_t warp_sum[32];
};

__host__ __device__ constexpr size_t rank_scratch_bytes(int E) {
    return (size_t)kFrameThreads * E * 8 > sizeof(SelSmem) ? (size_t)kFrameThreads * E * 8 : sizeof(SelSmem);
}

// Fills ss.bnd[0 .. K-2] and returns true, or returns false (every thread) when a bin is too full.
template <int E>
__device__ __forceinline__ bool select_boundaries(const uint64_t (&v)[E], uint32_t n, int K, SelSmem &ss) {
    constexpr int kPer = kSelBins / kFrameThreads;  // bins per thread in the scan
    static_assert(kPer == 16, "the scan reads four 16-byte words of bins per thread");
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, Q = K - 1;
    uint4 *h4 = reinterpret_cast<uint4 *>(ss.hist);
#pragma unroll
    for (int k = 0; k < 4; ++k) h4[t * 4 + k] = make_uint4(0u, 0u, 0u, 0u);
    if (t < Q) {  // a target rank t_q >= n (fewer tiles than classes) has no value: boundary above all
        ss.fill[t] = 0u;
        ss.count[t] = 0u;
        ss.bnd[t] = ~0ull;
        ss.target[t] = ((uint32_t)(t + 1) * n + (uint32_t)K - 1u) / (uint32_t)K;  // < 2^32: n <= 16384, K <= 8
    }
    __syncthreads();
    uint32_t d[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        d[e] = log_digit(v[e]);
        if ((uint32_t)(t * E + e) < n) atomicAdd(&ss.hist[d[e]], 1u);
    }
    __syncthreads();
    uint32_t c[kPer], sum = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint4 x = h4[t * 4 + k];
        c[4 * k] = x.x; c[4 * k + 1] = x.y; c[4 * k + 2] = x.z; c[4 * k + 3] = x.w;
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) sum += c[j];
    uint32_t incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) ss.warp_sum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t x = ss.warp_sum[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        ss.warp_sum[lane] = x;
    }
    __syncthreads();
    const uint32_t excl = (warp > 0 ? ss.warp_sum[warp - 1] : 0u) + incl - sum;
    for (int q = 0; q < Q; ++q) {
        const uint32_t tq = ss.target[q];
        if (excl <= tq && tq < excl + sum) {
            uint32_t acc = excl, below = 0u, cnt = 0u;
            int bj = -1;
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                if (bj < 0 && tq < acc + c[j]) {
                    bj = j;
                    below = acc;
                    cnt = c[j];
                }
                acc += c[j];
            }
            ss.bin[q] = (uint32_t)(t * kPer + bj);
            ss.rank[q] = tq - below;
            ss.count[q] = cnt;
        }
    }
    __syncthreads();
    for (int q = 0; q < Q; ++q)
        if (ss.count[q] > (uint32_t)kSelCap) return false;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const bool valid = (uint32_t)(t * E + e) < n;
        for (int q = 0; q < Q; ++q) {
            const bool match = valid && d[e] == ss.bin[q];
            const unsigned m = __ballot_sync(0xffffffffu, match);
            if (m != 0u) {
                const int leader = __ffs(m) - 1;
                uint32_t base = 0u;
                if (lane == leader) base = atomicAdd(&ss.fill[q], (uint32_t)__popc(m));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (match) ss.lst[q][base + __popc(m & ((1u << lane) - 1u))] = v[e];
            }
        }
    }
    __syncthreads();
    for (int slot = t; slot < Q * kSelCap; slot += kFrameThreads) {
        const int q = slot / kSelCap, j = slot - q * kSelCap;  // a warp's slots share q
        const uint32_t m = ss.count[q];
        if ((uint32_t)j < m) {
            const uint64_t x = ss.lst[q][j];
            uint32_t below = 0u;
            for (uint32_t i = 0; i < m; ++i) below += ss.lst[q][i] < x ? 1u : 0u;
            if (below == ss.rank[q]) ss.bnd[q] = x;
        }
    }
    __syncthreads();
    return true;
}

// One CTA per frame; frames of up to 1024 E tiles.  Padding values (all ones) sort behind every real value
// (the plan keeps packed values below 2^63).
template <int E>
__global__ void __launch_bounds__(kFrameThreads, 1) k_rank_sort(const Geom g, const CallArgs a) {
    extern __shared__ __align__(16) uint8_t dyn[];
    FinalizeSmem &sm = *reinterpret_cast<FinalizeSmem *>(dyn);
    uint8_t *scratch = dyn + sizeof(FinalizeSmem);  // the sort's values or the selection's tables
    uint64_t *s = reinterpret_cast<uint64_t *>(scratch);
    uint8_t *map_s = scratch + rank_scratch_bytes(E);
    const uint32_t f = blockIdx.x, n = g.ntiles;
    const uint64_t *keys = reinterpret_cast<const uint64_t *>(a.ws + (uint64_t)f * g.ws_per_frame + g.ws_keys);
    const int t = threadIdx.x;
    uint64_t v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const uint32_t i = (uint32_t)(t * E + e);
        v[e] = i < n ? (keys[i] << g.idx_bits) | (uint64_t)i : ~0ull;
    }
    if (g.K == 1) {
#pragma unroll
        for (int e = 0; e < E; ++e)
            if ((uint32_t)(t * E + e) < n) map_s[t * E + e] = 0;
    } else if (select_boundaries<E>(v, n, g.K, *reinterpret_cast<SelSmem *>(scratch))) {
        const SelSmem &ss = *reinterpret_cast<const SelSmem *>(scratch);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if ((uint32_t)(t * E + e) >= n) continue;
            int cls = 0;
            for (int q = 0; q + 1 < g.K; ++q) cls += v[e] >= ss.bnd[q] ? 1 : 0;
            map_s[t * E + e] = (uint8_t)cls;
        }
    } else {
        __syncthreads();  // the sort overwrites the selection's tables
        block_merge_sort<E>(v, s);
        const uint64_t mask = (1ull << g.idx_bits) - 1ull;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const uint32_t i = (uint32_t)(t * E + e);  // rank of v[e]
            if (i < n) map_s[(uint32_t)(v[e] & mask)] = (uint8_t)((uint64_t)g.K * i / n);
        }
    }
    __syncthreads();
    finalize_frame(g, a, f, map_s, true, sm);
}

template <int E>
cudaError_t launch_rank_sort(const Geom &g, const CallArgs &a, cudaStream_t s) {
    const size_t smem = sizeof(FinalizeSmem) + rank_scratch_bytes(E) + g.ntiles;
    launch_prep(reinterpret_cast<const void *>(k_rank_sort<E>), kFrameThreads, smem);
    prof_begin("k_rank", s);
    k_rank_sort<E><<<a.n_frames, kFrameThreads, smem, s>>>(g, a);
    prof_end("k_rank", s);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_finalize_labels(const Geom &g, const CallArgs &a, cudaStream_t s) {
    const size_t smem = sizeof(FinalizeSmem) + (g.ntiles <= (uint32_t)kFinalizeSmemTiles ? g.ntiles : 0u);
    launch_prep(reinterpret_cast<const void *>(k_finalize), kFrameThreads, smem);
    prof_begin("k_finalize", s);
    k_finalize<<<a.n_frames, kFrameThreads, smem, s>>>(g, a, 1);
    prof_end("k_finalize", s);
    return cudaGetLastError();
}

cudaError_t launch_finalize_map(const Geom &g, const CallArgs &a, cudaStream_t s) {
    const size_t smem = sizeof(FinalizeSmem) + (g.ntiles <= (uint32_t)kFinalizeSmemTiles ? g.ntiles : 0u);
    launch_prep(reinterpret_cast<const void *>(k_finalize), kFrameThreads, smem);
    prof_begin("k_finalize", s);
    k_finalize<<<a.n_frames, kFrameThreads, smem, s>>>(g, a, 0);
    prof_end("k_finalize", s);
    return cudaGetLastError();
}

cudaError_t launch_batch_finalize(const BatchEntry *tab, uint32_t n_img, uint32_t max_tiles, cudaStream_t s) {
    const size_t smem = sizeof(FinalizeSmem) + std::min<uint32_t>(max_tiles, (uint32_t)kFinalizeSmemTiles);
    launch_prep(reinterpret_cast<const void *>(k_batch_finalize), kFrameThreads, smem);
    const int grid = (int)std::min<uint32_t>(n_img, (uint32_t)sm_count());
    prof_begin("k_batch_finalize", s);
    k_batch_finalize<<<grid, kFrameThreads, smem, s>>>(tab, n_img);
    prof_end("k_batch_finalize", s);
    return cudaGetLastError();
}

cudaError_t launch_rank(const Geom &g, const CallArgs &a, cudaStream_t s) {
    // the plan admits at most kMaxRankTiles tiles and packed values below 2^64 - 1 (padding sorts last)
    static_assert(kMaxRankTiles <= 16 * kFrameThreads, "one CTA sorts at most 16 values per thread");
    if (g.val_bits >= 64 || g.ntiles > (uint32_t)kMaxRankTiles) return cudaErrorInvalidValue;
    if (g.ntiles <= kFrameThreads) return launch_rank_sort<1>(g, a, s);
    if (g.ntiles <= 2 * kFrameThreads) return launch_rank_sort<2>(g, a, s);
    if (g.ntiles <= 4 * kFrameThreads) return launch_rank_sort<4>(g, a, s);
    if (g.ntiles <= 8 * kFrameThreads) return launch_rank_sort<8>(g, a, s);
    return launch_rank_sort<16>(g, a, s);
}

}  // namespace dppix
