// k_stats_fast.cu -- variance-class statistics pass for aligned frames, read straight from HBM.
//
// One thread owns a CHUNK-byte column of one tile row (CHUNK = lcm(16, C*g) bytes, a whole number of g x g
// cells), streams the T rows of the tile row with 16-byte loads, and accumulates
//  - the exact per-channel sums of its g x g cells, one g-band of rows at a time, with dp4a against
//    compile-time byte masks that pick one channel out of the interleaved samples (Eq. 2 on g-cells);
//  - the tile's sum of squares (dp4a of a word with itself) and sum, reduced over the tile's threads by
//    shuffles into the exact rank key n*Q - S^2.
// The g-cell sums go to a "g-image" (rows of g-cells, C u16 each) so that neighbouring threads store
// neighbouring bytes (rows gpitch values apart).  With few frames the T/g bands of a tile row are split over
// 2^bs_log2 threads (the tile's column threads and band threads are adjacent lanes, so the key is still
// reduced by shuffles), so that a single frame fills the GPU.  Used when the frame needs no column padding and rows are 16-byte aligned; the
// staged kernel in k_release.cu covers everything else.
#include "common.cuh"

namespace dppix {
namespace {

constexpr int kThreads = 256;

__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }
__host__ __device__ constexpr int lcm_c(int a, int b) { return a / gcd_c(a, b) * b; }

// dp4a mask selecting the bytes of channel ch in word `word` of a row of C-interleaved samples whose
// first byte is channel 0.
__host__ __device__ constexpr uint32_t chan_mask(int word, int ch, int C) {
    uint32_t m = 0;
    for (int i = 0; i < 4; ++i)
        if ((4 * word + i) % C == ch) m |= 1u << (8 * i);
    return m;
}

template <int C, int G>
struct Chunk {
    static constexpr int CG = C * G;             // bytes in one row of a g-cell
    static constexpr int BYTES = lcm_c(16, CG);  // bytes per thread per row
    static constexpr int NV = BYTES / 16;        // 16-byte loads per row
    static constexpr int NW = BYTES / 4;         // words per row
    static constexpr int NG = BYTES / CG;        // g-cells per chunk
    static_assert(CG % 4 == 0, "g-cell rows must be whole words");
};

__device__ __forceinline__ uint4 ld_stream(const void *p) {
    uint4 v;
    asm volatile("ld.global.cs.v4.u32 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

template <int C, int G, bool kSplit>
__global__ void __launch_bounds__(kThreads) k_tile_stats_fast(const Geom g, const CallArgs a, int bs_log2) {
    using K = Chunk<C, G>;
    const int T = g.T;
    const int NQ = g.N * C / K::BYTES;   // chunks per image row (no column padding)
    const int CPT = T * C / K::BYTES;    // chunks per tile, a power of two; CPT << bs_log2 <= 32
    if (!kSplit) bs_log2 = 0;
    bool valid;
    int q, ty, split = 0;
    uint32_t f;
    if (kSplit) {
        // lane order: chunk of the tile (CPT), then band split (2^bs_log2), then tile column, tile row, frame;
        // the launcher keeps these launches below 2^31 threads
        const int lcpt = __ffs(CPT) - 1;
        const uint32_t total = ((uint32_t)a.n_frames * (uint32_t)g.GR * (uint32_t)NQ) << bs_log2;
        const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
        valid = gid < total;
        const uint32_t id = valid ? gid : total - 1u;  // idle lanes shadow a valid one (whole idle lane groups)
        const uint32_t id2 = id >> lcpt;
        split = (int)(id2 & ((1u << bs_log2) - 1u));
        const uint32_t id3 = id2 >> bs_log2;
        const uint32_t NT = (uint32_t)(NQ >> lcpt);  // tiles per tile row
        const uint32_t fr = id3 / NT;
        q = (int)(id3 - fr * NT) * CPT + (int)(id & (uint32_t)(CPT - 1));
        f = fr / (uint32_t)g.GR;
        ty = (int)(fr - f * (uint32_t)g.GR);
    } else {
        const uint64_t total = (uint64_t)a.n_frames * (uint64_t)g.GR * (uint64_t)NQ;
        const uint64_t gid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
        valid = gid < total;
        const uint64_t id = valid ? gid : total - 1;  // idle lanes shadow a valid one for the shuffles
        q = (int)(id % NQ);
        const uint64_t fr = id / NQ;
        ty = (int)(fr % g.GR);
        f = (uint32_t)(fr / g.GR);
    }
    const int cq = q & (CPT - 1);
    const uint8_t *fbase = a.frames + (uint64_t)f * (uint64_t)a.frame_stride + (uint64_t)q * K::BYTES;
    uint16_t *gimg = reinterpret_cast<uint16_t *>(a.ws + (uint64_t)f * g.ws_per_frame + g.ws_gsum);
    const int GP = g.gpitch;
    const int bands = T / G;
    const int bpt = bands >> bs_log2;    // bands of this thread
    uint32_t Ssum = 0, Qsum = 0;
    for (int band = split * bpt; band < (split + 1) * bpt; ++band) {
        uint32_t acc[K::NG][C];
#pragma unroll
        for (int c = 0; c < K::NG; ++c)
#pragma unroll
            for (int ch = 0; ch < C; ++ch) acc[c][ch] = 0;
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const int sy = reflect_idx(ty * T + band * G + i, g.M, g.pad_mode);
            const uint8_t *src = fbase + (int64_t)sy * g.pitch;
            uint32_t w[K::NW];
            const bool in = chk(src, K::BYTES, a.frames, a.frames_bytes, a.status, kChkFrame);
#pragma unroll
            for (int v = 0; v < K::NV; ++v) {
                const uint4 x = in ? ld_stream(src + 16 * v) : make_uint4(0u, 0u, 0u, 0u);
                w[4 * v] = x.x; w[4 * v + 1] = x.y; w[4 * v + 2] = x.z; w[4 * v + 3] = x.w;
            }
#pragma unroll
            for (int k = 0; k < K::NW; ++k) {
                Qsum = __dp4a(w[k], w[k], Qsum);
                const int cell = (4 * k) / K::CG;
#pragma unroll
                for (int ch = 0; ch < C; ++ch) {
                    const uint32_t m = chan_mask(k, ch, C);
                    if (m != 0u) acc[cell][ch] = __dp4a(w[k], m, acc[cell][ch]);
                }
            }
        }
        // g-cell sums of this band -> g-image row ty*T/G + band, cells q*NG .. q*NG+NG-1
        uint16_t *gdst = gimg + (size_t)(ty * bands + band) * GP + (size_t)q * K::NG * C;
        if (valid && chk(gdst, K::NG * C * 2, a.ws, a.ws_bytes, a.status, kChkWorkspace)) {
            uint16_t *dst = gdst;
            constexpr int NVAL = K::NG * C;
            if (NVAL % 2 == 0 && (reinterpret_cast<uintptr_t>(dst) & 3) == 0) {
#pragma unroll
                for (int v = 0; v < NVAL; v += 2) {
                    const uint32_t lo = acc[v / C][v % C], hi = acc[(v + 1) / C][(v + 1) % C];
                    reinterpret_cast<uint32_t *>(dst)[v / 2] = (lo & 0xFFFFu) | (hi << 16);
                }
            } else {
#pragma unroll
                for (int v = 0; v < NVAL; ++v) dst[v] = (uint16_t)acc[v / C][v % C];
            }
        }
#pragma unroll
        for (int c = 0; c < K::NG; ++c)
#pragma unroll
            for (int ch = 0; ch < C; ++ch) Ssum += acc[c][ch];
    }
    // tile totals over the tile's CPT << bs_log2 consecutive lanes
    unsigned long long Q64 = Qsum;
    for (int off = (CPT << bs_log2) >> 1; off > 0; off >>= 1) {
        Ssum += __shfl_xor_sync(0xffffffffu, Ssum, off);
        Q64 += __shfl_xor_sync(0xffffffffu, Q64, off);
    }
    if (valid && cq == 0 && split == 0) {
        const uint32_t tile = (uint32_t)ty * g.GC + (uint32_t)(q / CPT);
        const unsigned long long n = (unsigned long long)T * T * C;
        uint64_t *keys = reinterpret_cast<uint64_t *>(a.ws + (uint64_t)f * g.ws_per_frame + g.ws_keys);
        if (chk(&keys[tile], 8, a.ws, a.ws_bytes, a.status, kChkWorkspace))
            keys[tile] = n * Q64 - (unsigned long long)Ssum * Ssum;
    }
}

template <int C, int G>
cudaError_t launch_fast(const Geom &g, const CallArgs &a, cudaStream_t s) {
    using K = Chunk<C, G>;
    const uint64_t base = (uint64_t)a.n_frames * g.GR * (uint64_t)(g.N * C / K::BYTES);
    // split the bands of a tile row over more threads until the launch covers every SM with a few blocks
    // (single frames, small batches); a power of two that divides the band count, lanes of one tile <= 32
    const int bands = g.T / G, cpt = g.T * C / K::BYTES;
    int bs_log2 = 0;
    while ((base << bs_log2) < (uint64_t)sm_count() * 4 * kThreads && (bands >> bs_log2) % 2 == 0 &&
           (cpt << (bs_log2 + 1)) <= 32)
        ++bs_log2;
    const uint64_t total = base << bs_log2;
    const uint64_t blocks = (total + kThreads - 1) / kThreads;
    prof_begin("k_tile_stats_gsum", s);
    if (bs_log2 > 0)  // only for small launches (below a few SM waves of threads)
        k_tile_stats_fast<C, G, true><<<(unsigned)blocks, kThreads, 0, s>>>(g, a, bs_log2);
    else
        k_tile_stats_fast<C, G, false><<<(unsigned)blocks, kThreads, 0, s>>>(g, a, 0);
    prof_end("k_tile_stats_gsum", s);
    return cudaGetLastError();
}

template <int C, int G>
bool fits(const Geom &g) {
    using K = Chunk<C, G>;
    if (g.C != C || g.g != G) return false;
    if ((g.T * C) % K::BYTES != 0) return false;
    const int cpt = g.T * C / K::BYTES;
    return cpt >= 1 && cpt <= 32 && (cpt & (cpt - 1)) == 0;
}

}  // namespace

// Returns cudaErrorNotSupported (nothing launched) when this frame layout has no fast instance.
cudaError_t launch_tile_stats_fast(const Geom &g, const CallArgs &a, cudaStream_t s) {
    if (!g.var_onepass || g.PC != 0 || a.vec != 16) return cudaErrorNotSupported;
#define DPPIX_TRY_FAST(CC, GG) \
    if (fits<CC, GG>(g)) return launch_fast<CC, GG>(g, a, s);
    DPPIX_TRY_FAST(3, 4)
    DPPIX_TRY_FAST(3, 8)
    DPPIX_TRY_FAST(3, 16)
    DPPIX_TRY_FAST(1, 4)
    DPPIX_TRY_FAST(1, 8)
    DPPIX_TRY_FAST(1, 16)
    DPPIX_TRY_FAST(4, 4)
    DPPIX_TRY_FAST(4, 8)
    DPPIX_TRY_FAST(4, 16)
#undef DPPIX_TRY_FAST
    return cudaErrorNotSupported;
}

}  // namespace dppix
