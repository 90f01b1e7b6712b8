// k_classify.cu -- tile classification from a per-pixel region source (Alg. 3 steps 3-6).
//
// One CTA per (tile row, frame).  Each thread owns padded pixel columns, counts the simple samples of the
// column over the tile row's T mirror-padded rows, and adds the count to its tile's counter.  A tile is
// simple (region 0) iff 2 * #simple > T^2 -- the paper's mask mean > 1/2 on exact integers, a tie going
// to complex (region 1); without padding (DP_PIX_PAD_NONE) over the tile's pixels inside the frame.  MASK_U8: nonzero = simple.  MATTE_F32: a pixel is complex iff alpha >= thr.
#include <algorithm>

#include "common.cuh"

namespace dppix {
namespace {

constexpr int kThreads = 256;

// Tile row ty of frame f: the map bytes of its GC tiles.  cnt_s: GC counters in shared memory.
template <bool kMatte>
__device__ __forceinline__ void classify_row(const Geom &g, const CallArgs &a, int ty, uint32_t f, uint32_t *cnt_s) {
    const int T = g.T;
    for (int i = threadIdx.x; i < g.GC; i += blockDim.x) cnt_s[i] = 0u;
    __syncthreads();
    const uint8_t *src = a.src + (uint64_t)f * (uint64_t)a.src_frame_stride;
    const bool strict = g.pad_mode == DP_PIX_PAD_NONE;       // only samples inside the frame count
    const int Wp = strict ? g.N : g.GC * T;
    const int rows = strict ? min(T, g.M - ty * T) : T;
    int x_first = 0;  // first column left to the per-column loop below
    if (kMatte) {
        // in-image columns in groups of 4, read as 16-byte granules (rows are 4-byte aligned, so a group spans
        // at most two granules, the second loaded only when it holds wanted bytes); the 4 per-column counts
        // are kept in registers over the tile row's T rows
        const int ngrp = (g.N + 3) >> 2;
        for (int q = threadIdx.x; q < ngrp; q += blockDim.x) {
            const int c0 = 4 * q, cnt = min(4, g.N - c0);
            uint32_t c[4] = {0u, 0u, 0u, 0u};
#pragma unroll 8
            for (int j = 0; j < rows; ++j) {
                const int sy = reflect_idx(ty * T + j, g.M, g.pad_mode);
                const uintptr_t addr = reinterpret_cast<uintptr_t>(src + (int64_t)sy * a.src_pitch) + 16u * (uint32_t)q;
                const int o = (int)(addr & 15u);
                const uint4 *ga = reinterpret_cast<const uint4 *>(addr - (uintptr_t)o);
                const uint4 x0 = __ldg(ga);
                const uint4 x1 = o + 4 * cnt > 16 ? __ldg(ga + 1) : make_uint4(0u, 0u, 0u, 0u);
                const uint32_t w[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                const int qw = o >> 2;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    uint32_t v = w[k];
                    if (qw == 1) v = w[k + 1];
                    if (qw == 2) v = w[k + 2];
                    if (qw == 3) v = w[k + 3];
                    c[k] += (k < cnt && !(__uint_as_float(v) >= g.matte_thr)) ? 1u : 0u;
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k < cnt) atomicAdd(&cnt_s[(c0 + k) / T], c[k]);
        }
        x_first = g.N;
    }
    for (int x = x_first + threadIdx.x; x < Wp; x += blockDim.x) {
        const int sx = reflect_idx(x, g.N, g.pad_mode);
        uint32_t c = 0;
#pragma unroll 8
        for (int j = 0; j < rows; ++j) {
            const int sy = reflect_idx(ty * T + j, g.M, g.pad_mode);
            const uint8_t *row = src + (int64_t)sy * a.src_pitch;
            if (kMatte) {
                const float alpha = reinterpret_cast<const float *>(row)[sx];
                c += (alpha >= g.matte_thr) ? 0u : 1u;
            } else {
                c += row[sx] != 0 ? 1u : 0u;
            }
        }
        atomicAdd(&cnt_s[x / T], c);
    }
    __syncthreads();
    uint8_t *map = a.records + (uint64_t)f * (uint64_t)a.record_stride + g.map_offset + (uint64_t)ty * g.GC;
    for (int tx = threadIdx.x; tx < g.GC; tx += blockDim.x) {
        const uint32_t n = (uint32_t)rows * (uint32_t)(strict ? min(T, g.N - tx * T) : T);  // samples counted
        map[tx] = (2u * cnt_s[tx] > n) ? 0 : 1;
    }
}

template <bool kMatte>
__global__ void __launch_bounds__(kThreads) k_classify(const Geom g, const CallArgs a) {
    extern __shared__ uint32_t cnt_s[];  // [GC]
    classify_row<kMatte>(g, a, blockIdx.x, blockIdx.y, cnt_s);
}

}  // namespace

cudaError_t launch_classify(const Geom &g, const CallArgs &a, cudaStream_t s) {
    const dim3 grid(g.GR, a.n_frames);
    const size_t smem = (size_t)g.GC * 4;
    if (g.source == DP_PIX_SRC_MATTE_F32) {
        prof_begin("k_classify_matte", s);
        k_classify<true><<<grid, kThreads, smem, s>>>(g, a);
        prof_end("k_classify_matte", s);
    } else {
        prof_begin("k_classify_mask", s);
        k_classify<false><<<grid, kThreads, smem, s>>>(g, a);
        prof_end("k_classify_mask", s);
    }
    return cudaGetLastError();
}

}  // namespace dppix
