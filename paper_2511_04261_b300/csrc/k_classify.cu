// k_classify.cu -- tile classification from a per-pixel region source (Alg. 3 steps 3-6).
//
// One CTA per (tile row, frame).  Each thread owns padded pixel columns, counts the simple samples of the
// column over the tile row's T mirror-padded rows, and adds the count to its tile's counter.  A tile is
// simple (region 0) iff 2 * #simple > T^2 -- the paper's mask mean > 1/2 on exact integers, a tie going
// to complex (region 1).  MASK_U8: nonzero = simple.  MATTE_F32: a pixel is complex iff alpha >= thr.
#include "common.cuh"

namespace dppix {
namespace {

constexpr int kThreads = 256;

template <bool kMatte>
__global__ void __launch_bounds__(kThreads) k_classify(const Geom g, const CallArgs a) {
    extern __shared__ uint32_t cnt_s[];  // [GC]
    const int ty = blockIdx.x;
    const uint32_t f = blockIdx.y;
    const int T = g.T;
    for (int i = threadIdx.x; i < g.GC; i += blockDim.x) cnt_s[i] = 0u;
    __syncthreads();
    const uint8_t *src = a.src + (uint64_t)f * (uint64_t)a.src_frame_stride;
    const int Wp = g.GC * T;
    for (int x = threadIdx.x; x < Wp; x += blockDim.x) {
        const int sx = reflect_idx(x, g.N, g.pad_mode);
        uint32_t c = 0;
        for (int j = 0; j < T; ++j) {
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
    const uint32_t half2 = (uint32_t)T * (uint32_t)T;
    for (int tx = threadIdx.x; tx < g.GC; tx += blockDim.x) map[tx] = (2u * cnt_s[tx] > half2) ? 0 : 1;
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
