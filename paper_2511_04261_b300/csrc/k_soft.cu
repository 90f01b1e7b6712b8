// k_soft.cu -- the differentiable soft layer: y = w * P~_{b0}(x) + (1 - w) * P~_{b1}(x) and its adjoint.
//
// Each P~_b is the uniform release of Alg. 2 (pad, cell mean, Laplace noise of scale R m / (b^2 eps),
// clip to [0, R], repeat, crop) applied to every channel plane of planar f32 images; the noise of grid j,
// cell (cy, cx) of image n uses the counter (cy * G_C,j + cx, j | stream << 8, frame0 + n) so that forward
// and backward see the same draws.  The backward holds the noise constant:
//   dL/dw(p) = sum_ch g(p) (P~_{b0}(p) - P~_{b1}(p)),
//   dL/dx(q) = sum_j sum_{cells c whose padded samples include q} [0 < pre_c < R] mult(q, c) / b_j^2
//              * sum_{p in c inside the image} g(p) w_j(p),      w_0 = w, w_1 = 1 - w.
// The forward saves the unclipped noisy means ("pre") per cell: [B][2][C][G_R,j][G_C,j] (grid 0's block,
// then grid 1's, per image); the backward reads them back for the clip flags and for dL/dw.
//
// Fast path (both grids powers of two, 4 <= b <= 128, one dividing the other, no padding, W a multiple of 128,
// 16-byte aligned planes): one warp per (image, strip of b_large rows, 128 columns), lane = 4 columns; cell
// sums by shuffles across the lanes of a cell, so x (or g) is read once and y (or dx, dw) written once.
// Otherwise: generic per-cell and per-pixel kernels with mirror-padding index arithmetic.
#include <algorithm>

#include "common.cuh"

namespace dppix {
namespace {

constexpr int kSoftThreads = 128;

struct SoftGeom {
    int32_t B, C, H, W;
    int32_t b[2];
    int32_t gr[2], gc[2];
    float sigma[2];
    float inv_b2[2];  // 1 / b^2 (exact for powers of two)
    float b2[2];
    float R;
    int32_t pad_mode, noise_free;
    uint32_t stream_id;
    uint64_t seed, frame0;
    int64_t pre_img;      // floats of pre per image: C * (gr0 gc0 + gr1 gc1)
    int64_t pre_off1;     // offset of grid 1's block inside an image's pre
};

__device__ __forceinline__ float soft_mean(float sum, const SoftGeom &sg, int j) {
    return sg.inv_b2[j] != 0.0f ? sum * sg.inv_b2[j] : __fdiv_rn(sum, sg.b2[j]);
}

__device__ __forceinline__ float clip_r(float v, float R) { return fminf(fmaxf(v, 0.0f), R); }

__device__ __forceinline__ uint4 soft_words(const SoftGeom &sg, int j, uint32_t cell, uint32_t n) {
    const uint64_t frame = sg.frame0 + n;
    return philox4x32_10(make_uint4(cell, (uint32_t)j | (sg.stream_id << 8), (uint32_t)frame, (uint32_t)(frame >> 32)),
                         make_uint2((uint32_t)sg.seed, (uint32_t)(sg.seed >> 32)));
}

__device__ __forceinline__ float soft_eta(const SoftGeom &sg, const uint4 &wd, int ch, int j) {
    return sg.noise_free ? 0.0f : laplace_from_word(word_of(wd, ch), sg.sigma[j]);
}

__device__ __forceinline__ int64_t pre_index(const SoftGeom &sg, uint32_t n, int j, int ch, int cy, int cx) {
    return (int64_t)n * sg.pre_img + (j ? sg.pre_off1 : 0) + ((int64_t)ch * sg.gr[j] + cy) * sg.gc[j] + cx;
}

__device__ __forceinline__ float4 ld4(const float *p) { return __ldcs(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ void st4(float *p, float4 v) { __stcs(reinterpret_cast<float4 *>(p), v); }

template <int LANES>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int off = 1; off < LANES; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// ---------------------------------------------------------------------------------------------------------
// Fast forward.  LS / LL: lanes per small / large cell (b / 4); js: the grid index of the small grid.
// ---------------------------------------------------------------------------------------------------------
template <int C, int LS, int LL>
__global__ void __launch_bounds__(kSoftThreads) k_soft_fwd_fast(const SoftGeom sg, int js, const float *__restrict__ x,
                                                                  const float *__restrict__ w, float *__restrict__ y,
                                                                  float *__restrict__ pre) {
    constexpr int BS = 4 * LS, BL = 4 * LL, NB = LL / LS;
    const int jl = 1 - js;
    const int lane = threadIdx.x & 31;
    const int H = sg.H, W = sg.W;
    const uint32_t strips = (uint32_t)(H / BL), cblocks = (uint32_t)(W / 128);
    const uint32_t items = (uint32_t)sg.B * strips * cblocks;
    const uint32_t nw = gridDim.x * (kSoftThreads / 32);
    for (uint32_t item = blockIdx.x * (kSoftThreads / 32) + (threadIdx.x >> 5); item < items; item += nw) {
        const uint32_t cb = item % cblocks, t = item / cblocks;
        const uint32_t sy = t % strips, n = t / strips;
        const int c0 = (int)cb * 128 + 4 * lane;
        const int y0 = (int)sy * BL;
        float acc[C][NB];
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            const float *xp = x + (((size_t)n * C + ch) * H + y0) * W + c0;
#pragma unroll
            for (int bnd = 0; bnd < NB; ++bnd) {
                float s = 0.0f;
#pragma unroll
                for (int r = 0; r < BS; ++r) {
                    const float4 v = ld4(xp + (size_t)(bnd * BS + r) * W);
                    s += (v.x + v.y) + (v.z + v.w);
                }
                acc[ch][bnd] = s;
            }
        }
        // cell sums, noise, noisy means
        const int cxs = c0 / BS, cxl = c0 / BL;
        float ps[C][NB], pl[C];
#pragma unroll
        for (int bnd = 0; bnd < NB; ++bnd) {
            const int cy = (int)sy * NB + bnd;
            const uint4 wd = soft_words(sg, js, (uint32_t)(cy * sg.gc[js] + cxs), n);
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                const float v = soft_mean(group_sum<LS>(acc[ch][bnd]), sg, js) + soft_eta(sg, wd, ch, js);
                ps[ch][bnd] = v;
                if ((lane & (LS - 1)) == 0) pre[pre_index(sg, n, js, ch, cy, cxs)] = v;
            }
        }
        {
            const uint4 wd = soft_words(sg, jl, (uint32_t)((int)sy * sg.gc[jl] + cxl), n);
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                float tot = 0.0f;
#pragma unroll
                for (int bnd = 0; bnd < NB; ++bnd) tot += acc[ch][bnd];
                const float v = soft_mean(group_sum<LL>(tot), sg, jl) + soft_eta(sg, wd, ch, jl);
                pl[ch] = v;
                if ((lane & (LL - 1)) == 0) pre[pre_index(sg, n, jl, ch, (int)sy, cxl)] = v;
            }
        }
        // broadcast: y = w p0 + (1 - w) p1 = p1 + w (p0 - p1)
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            pl[ch] = clip_r(pl[ch], sg.R);
#pragma unroll
            for (int bnd = 0; bnd < NB; ++bnd) ps[ch][bnd] = clip_r(ps[ch][bnd], sg.R);
        }
        const float *wp = w + ((size_t)n * H + y0) * W + c0;
#pragma unroll
        for (int bnd = 0; bnd < NB; ++bnd) {
#pragma unroll 4
            for (int r = 0; r < BS; ++r) {
                const float4 wv = ld4(wp + (size_t)(bnd * BS + r) * W);
#pragma unroll
                for (int ch = 0; ch < C; ++ch) {
                    const float p0 = js == 0 ? ps[ch][bnd] : pl[ch], p1 = js == 0 ? pl[ch] : ps[ch][bnd];
                    const float d = p0 - p1;
                    float4 o;
                    o.x = fmaf(wv.x, d, p1);
                    o.y = fmaf(wv.y, d, p1);
                    o.z = fmaf(wv.z, d, p1);
                    o.w = fmaf(wv.w, d, p1);
                    st4(y + (((size_t)n * C + ch) * H + y0 + bnd * BS + r) * W + c0, o);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------------------
// Fast backward.
// ---------------------------------------------------------------------------------------------------------
template <int C, int LS, int LL>
__global__ void __launch_bounds__(kSoftThreads) k_soft_bwd_fast(const SoftGeom sg, int js, const float *__restrict__ w,
                                                                  const float *__restrict__ gy,
                                                                  const float *__restrict__ pre, float *__restrict__ dx,
                                                                  float *__restrict__ dw) {
    constexpr int BS = 4 * LS, BL = 4 * LL, NB = LL / LS;
    const int jl = 1 - js;
    const int lane = threadIdx.x & 31;
    const int H = sg.H, W = sg.W;
    const uint32_t strips = (uint32_t)(H / BL), cblocks = (uint32_t)(W / 128);
    const uint32_t items = (uint32_t)sg.B * strips * cblocks;
    const uint32_t nw = gridDim.x * (kSoftThreads / 32);
    for (uint32_t item = blockIdx.x * (kSoftThreads / 32) + (threadIdx.x >> 5); item < items; item += nw) {
        const uint32_t cb = item % cblocks, t = item / cblocks;
        const uint32_t sy = t % strips, n = t / strips;
        const int c0 = (int)cb * 128 + 4 * lane;
        const int y0 = (int)sy * BL;
        const int cxs = c0 / BS, cxl = c0 / BL;
        // saved noisy means of this lane's cells
        float qs[C][NB], ql[C];
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            ql[ch] = __ldg(pre + pre_index(sg, n, jl, ch, (int)sy, cxl));
#pragma unroll
            for (int bnd = 0; bnd < NB; ++bnd) qs[ch][bnd] = __ldg(pre + pre_index(sg, n, js, ch, (int)sy * NB + bnd, cxs));
        }
        float gw[C][NB], gs[C][NB];
#pragma unroll
        for (int ch = 0; ch < C; ++ch)
#pragma unroll
            for (int bnd = 0; bnd < NB; ++bnd) gw[ch][bnd] = gs[ch][bnd] = 0.0f;
        const float *wp = w + ((size_t)n * H + y0) * W + c0;
#pragma unroll
        for (int bnd = 0; bnd < NB; ++bnd) {
            float dl[C];  // P~_{b0} - P~_{b1} of this lane's pixels
#pragma unroll
            for (int ch = 0; ch < C; ++ch) {
                const float a = clip_r(qs[ch][bnd], sg.R), b = clip_r(ql[ch], sg.R);
                dl[ch] = js == 0 ? a - b : b - a;
            }
#pragma unroll 4
            for (int r = 0; r < BS; ++r) {
                const size_t row = (size_t)(bnd * BS + r);
                const float4 wv = ld4(wp + row * W);
                float4 dwv = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int ch = 0; ch < C; ++ch) {
                    const float4 g = ld4(gy + (((size_t)n * C + ch) * H + y0) * W + row * W + c0);
                    gw[ch][bnd] += (g.x * wv.x + g.y * wv.y) + (g.z * wv.z + g.w * wv.w);
                    gs[ch][bnd] += (g.x + g.y) + (g.z + g.w);
                    dwv.x = fmaf(g.x, dl[ch], dwv.x);
                    dwv.y = fmaf(g.y, dl[ch], dwv.y);
                    dwv.z = fmaf(g.z, dl[ch], dwv.z);
                    dwv.w = fmaf(g.w, dl[ch], dwv.w);
                }
                st4(dw + ((size_t)n * H + y0) * W + row * W + c0, dwv);
            }
        }
        // per-cell coefficients: [unclipped] / b^2 * sum g w_j
        float as[C][NB], al[C];
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            float tgw = 0.0f, tgs = 0.0f;
#pragma unroll
            for (int bnd = 0; bnd < NB; ++bnd) {
                const float cgw = group_sum<LS>(gw[ch][bnd]), cgs = group_sum<LS>(gs[ch][bnd]);
                const float coef = js == 0 ? cgw : cgs - cgw;
                const float q = qs[ch][bnd];
                as[ch][bnd] = (q > 0.0f && q < sg.R) ? soft_mean(coef, sg, js) : 0.0f;
                tgw += gw[ch][bnd];
                tgs += gs[ch][bnd];
            }
            const float cgw = group_sum<LL>(tgw), cgs = group_sum<LL>(tgs);
            const float coef = jl == 0 ? cgw : cgs - cgw;
            al[ch] = (ql[ch] > 0.0f && ql[ch] < sg.R) ? soft_mean(coef, sg, jl) : 0.0f;
        }
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
            float *dp = dx + (((size_t)n * C + ch) * H + y0) * W + c0;
#pragma unroll
            for (int bnd = 0; bnd < NB; ++bnd) {
                const float v = as[ch][bnd] + al[ch];
                const float4 o = make_float4(v, v, v, v);
#pragma unroll 4
                for (int r = 0; r < BS; ++r) st4(dp + (size_t)(bnd * BS + r) * W, o);
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------------------
// Generic kernels (any grids, mirror padding).
// ---------------------------------------------------------------------------------------------------------
__device__ __forceinline__ int soft_reflect(int p, int n, int pad_mode) { return reflect_idx(p, n, pad_mode); }

// One thread per (image, grid, cell): sums over the padded cell, noise, unclipped mean into pre.
__global__ void k_soft_cells(const SoftGeom sg, const float *__restrict__ x, float *__restrict__ pre) {
    const uint64_t cells0 = (uint64_t)sg.gr[0] * sg.gc[0], cells1 = (uint64_t)sg.gr[1] * sg.gc[1];
    const uint64_t total = (uint64_t)sg.B * (cells0 + cells1);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t n = (uint32_t)(i / (cells0 + cells1));
        uint64_t rem = i - (uint64_t)n * (cells0 + cells1);
        const int j = rem < cells0 ? 0 : 1;
        if (j) rem -= cells0;
        const int cy = (int)(rem / sg.gc[j]), cx = (int)(rem - (uint64_t)cy * sg.gc[j]);
        const int b = sg.b[j];
        const uint4 wd = soft_words(sg, j, (uint32_t)rem, n);
        for (int ch = 0; ch < sg.C; ++ch) {
            const float *plane = x + ((size_t)n * sg.C + ch) * sg.H * sg.W;
            float s = 0.0f;
            for (int yy = cy * b; yy < (cy + 1) * b; ++yy) {
                const float *row = plane + (size_t)soft_reflect(yy, sg.H, sg.pad_mode) * sg.W;
                for (int xx = cx * b; xx < (cx + 1) * b; ++xx) s += row[soft_reflect(xx, sg.W, sg.pad_mode)];
            }
            pre[pre_index(sg, n, j, ch, cy, cx)] = soft_mean(s, sg, j) + soft_eta(sg, wd, ch, j);
        }
    }
}

// One thread per (image, pixel): y for every channel from the two cells covering the pixel.
__global__ void k_soft_broadcast(const SoftGeom sg, const float *__restrict__ w, const float *__restrict__ pre,
                                 float *__restrict__ y) {
    const uint64_t hw = (uint64_t)sg.H * sg.W, total = (uint64_t)sg.B * hw;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t n = (uint32_t)(i / hw);
        const int p = (int)(i - (uint64_t)n * hw);
        const int py = p / sg.W, px = p - py * sg.W;
        const float wv = w[i];
        for (int ch = 0; ch < sg.C; ++ch) {
            const float p0 = clip_r(pre[pre_index(sg, n, 0, ch, py / sg.b[0], px / sg.b[0])], sg.R);
            const float p1 = clip_r(pre[pre_index(sg, n, 1, ch, py / sg.b[1], px / sg.b[1])], sg.R);
            y[((size_t)n * sg.C + ch) * hw + p] = fmaf(wv, p0 - p1, p1);
        }
    }
}

// One thread per (image, grid, cell): A = [0 < pre < R] / b^2 * sum over the cell's in-image pixels of g w_j.
__global__ void k_soft_coef(const SoftGeom sg, const float *__restrict__ w, const float *__restrict__ gy,
                            const float *__restrict__ pre, float *__restrict__ coef) {
    const uint64_t cells0 = (uint64_t)sg.gr[0] * sg.gc[0], cells1 = (uint64_t)sg.gr[1] * sg.gc[1];
    const uint64_t total = (uint64_t)sg.B * (cells0 + cells1);
    const uint64_t hw = (uint64_t)sg.H * sg.W;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t n = (uint32_t)(i / (cells0 + cells1));
        uint64_t rem = i - (uint64_t)n * (cells0 + cells1);
        const int j = rem < cells0 ? 0 : 1;
        if (j) rem -= cells0;
        const int cy = (int)(rem / sg.gc[j]), cx = (int)(rem - (uint64_t)cy * sg.gc[j]);
        const int b = sg.b[j];
        const int y1 = min((cy + 1) * b, sg.H), x1 = min((cx + 1) * b, sg.W);
        for (int ch = 0; ch < sg.C; ++ch) {
            const int64_t pi = pre_index(sg, n, j, ch, cy, cx);
            const float q = pre[pi];
            float a = 0.0f;
            if (q > 0.0f && q < sg.R) {
                const float *gp = gy + ((size_t)n * sg.C + ch) * hw;
                const float *wp = w + (size_t)n * hw;
                float s = 0.0f;
                for (int yy = cy * b; yy < y1; ++yy)
                    for (int xx = cx * b; xx < x1; ++xx) {
                        const size_t o = (size_t)yy * sg.W + xx;
                        s += gp[o] * (j == 0 ? wp[o] : 1.0f - wp[o]);
                    }
                a = soft_mean(s, sg, j);
            }
            coef[pi] = a;
        }
    }
}

// Padded positions along one axis that read source index q: q itself and, inside the padded extent, its
// mirror image.  Returns the count (1 or 2).
__device__ __forceinline__ int mirror_sources(int q, int n, int padded, int pad_mode, int out[2]) {
    out[0] = q;
    const int m = pad_mode == DP_PIX_PAD_REFLECT ? 2 * (n - 1) - q : 2 * n - 1 - q;
    if (m >= n && m < padded && m != q) {
        out[1] = m;
        return 2;
    }
    return 1;
}

// One thread per (image, pixel): dx from every padded sample that reads the pixel, dw from the two means.
__global__ void k_soft_grad(const SoftGeom sg, const float *__restrict__ gy, const float *__restrict__ pre,
                            const float *__restrict__ coef, float *__restrict__ dx, float *__restrict__ dw) {
    const uint64_t hw = (uint64_t)sg.H * sg.W, total = (uint64_t)sg.B * hw;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t n = (uint32_t)(i / hw);
        const int p = (int)(i - (uint64_t)n * hw);
        const int py = p / sg.W, px = p - py * sg.W;
        float dwv = 0.0f;
        for (int ch = 0; ch < sg.C; ++ch) {
            float acc = 0.0f;
            for (int j = 0; j < 2; ++j) {
                int ys[2], xs[2];
                const int ny = mirror_sources(py, sg.H, sg.gr[j] * sg.b[j], sg.pad_mode, ys);
                const int nx = mirror_sources(px, sg.W, sg.gc[j] * sg.b[j], sg.pad_mode, xs);
                for (int a = 0; a < ny; ++a)
                    for (int c = 0; c < nx; ++c) acc += coef[pre_index(sg, n, j, ch, ys[a] / sg.b[j], xs[c] / sg.b[j])];
            }
            dx[((size_t)n * sg.C + ch) * hw + p] = acc;
            const float p0 = clip_r(pre[pre_index(sg, n, 0, ch, py / sg.b[0], px / sg.b[0])], sg.R);
            const float p1 = clip_r(pre[pre_index(sg, n, 1, ch, py / sg.b[1], px / sg.b[1])], sg.R);
            dwv = fmaf(gy[((size_t)n * sg.C + ch) * hw + p], p0 - p1, dwv);
        }
        dw[i] = dwv;
    }
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Fast-path eligibility; js = index of the smaller grid.
bool soft_fast(const SoftGeom &sg, const void *const *ptrs, int nptr, int *js) {
    const int bs = std::min(sg.b[0], sg.b[1]), bl = std::max(sg.b[0], sg.b[1]);
    if (!is_pow2(bs) || !is_pow2(bl) || bs < 4 || bl > 128) return false;
    if (sg.H % bl != 0 || sg.W % 128 != 0) return false;
    for (int i = 0; i < nptr; ++i)
        if (reinterpret_cast<uintptr_t>(ptrs[i]) & 15) return false;
    *js = sg.b[0] <= sg.b[1] ? 0 : 1;
    return true;
}

int soft_grid(const void *kern, int threads, uint64_t work) {
    const int per_sm = launch_prep(kern, threads, 0);
    const uint64_t cap = (uint64_t)per_sm * (uint64_t)sm_count();
    const uint64_t want = (work + threads - 1) / threads;
    return (int)std::max<uint64_t>(1, std::min(cap, want));
}

// Dispatch of the fast kernels over C in 1..4 and the (LS, LL) pairs.
template <template <int, int, int> class Launch, typename... Args>
cudaError_t soft_dispatch(const SoftGeom &sg, Args... args) {
    const int LS = std::min(sg.b[0], sg.b[1]) / 4, LL = std::max(sg.b[0], sg.b[1]) / 4;
#define DPPIX_SOFT_CASE(CC, S, L) \
    if (sg.C == CC && LS == S && LL == L) return Launch<CC, S, L>::run(sg, args...);
#define DPPIX_SOFT_C(CC)                                                                                   \
    DPPIX_SOFT_CASE(CC, 1, 1) DPPIX_SOFT_CASE(CC, 1, 2) DPPIX_SOFT_CASE(CC, 1, 4) DPPIX_SOFT_CASE(CC, 1, 8)  \
    DPPIX_SOFT_CASE(CC, 1, 16) DPPIX_SOFT_CASE(CC, 1, 32) DPPIX_SOFT_CASE(CC, 2, 2) DPPIX_SOFT_CASE(CC, 2, 4) \
    DPPIX_SOFT_CASE(CC, 2, 8) DPPIX_SOFT_CASE(CC, 2, 16) DPPIX_SOFT_CASE(CC, 2, 32) DPPIX_SOFT_CASE(CC, 4, 4) \
    DPPIX_SOFT_CASE(CC, 4, 8) DPPIX_SOFT_CASE(CC, 4, 16) DPPIX_SOFT_CASE(CC, 4, 32) DPPIX_SOFT_CASE(CC, 8, 8) \
    DPPIX_SOFT_CASE(CC, 8, 16) DPPIX_SOFT_CASE(CC, 8, 32) DPPIX_SOFT_CASE(CC, 16, 16) DPPIX_SOFT_CASE(CC, 16, 32) \
    DPPIX_SOFT_CASE(CC, 32, 32)
    DPPIX_SOFT_C(1) DPPIX_SOFT_C(2) DPPIX_SOFT_C(3) DPPIX_SOFT_C(4)
#undef DPPIX_SOFT_C
#undef DPPIX_SOFT_CASE
    return cudaErrorNotSupported;
}

template <int C, int LS, int LL>
struct FwdLaunch {
    static cudaError_t run(const SoftGeom &sg, int js, const float *x, const float *w, float *y, float *pre,
                           cudaStream_t s) {
        const uint64_t items = (uint64_t)sg.B * (sg.H / (4 * LL)) * (sg.W / 128);
        const int grid = soft_grid((const void *)k_soft_fwd_fast<C, LS, LL>, kSoftThreads, items * 32);
        prof_begin("k_soft_fwd", s);
        k_soft_fwd_fast<C, LS, LL><<<grid, kSoftThreads, 0, s>>>(sg, js, x, w, y, pre);
        prof_end("k_soft_fwd", s);
        return cudaGetLastError();
    }
};

template <int C, int LS, int LL>
struct BwdLaunch {
    static cudaError_t run(const SoftGeom &sg, int js, const float *w, const float *gy, const float *pre, float *dx,
                           float *dw, cudaStream_t s) {
        const uint64_t items = (uint64_t)sg.B * (sg.H / (4 * LL)) * (sg.W / 128);
        const int grid = soft_grid((const void *)k_soft_bwd_fast<C, LS, LL>, kSoftThreads, items * 32);
        prof_begin("k_soft_bwd", s);
        k_soft_bwd_fast<C, LS, LL><<<grid, kSoftThreads, 0, s>>>(sg, js, w, gy, pre, dx, dw);
        prof_end("k_soft_bwd", s);
        return cudaGetLastError();
    }
};

}  // namespace

// Host-side geometry of a soft-layer call (validation as dp_pix_plan: positive sizes, mirror padding
// inside the image).  Returns 0 or a DP_PIX_E_* code with the message set.
int soft_geometry(const dp_pix_soft_desc *d, SoftGeom *sg) {
    if (!d) return set_last_error(DP_PIX_E_INVALID_ARG, "soft desc is NULL");
    if (d->B < 1 || d->C < 1 || d->C > 4 || d->H < 1 || d->W < 1)
        return set_last_error(DP_PIX_E_INVALID_ARG, "soft layer needs B, H, W >= 1 and C in 1..4");
    if (d->pad_mode != DP_PIX_PAD_REFLECT && d->pad_mode != DP_PIX_PAD_SYMMETRIC)
        return set_last_error(DP_PIX_E_INVALID_ARG, "bad pad_mode");
    if (!(d->value_range > 0.0) || !(d->m > 0.0)) return set_last_error(DP_PIX_E_INVALID_ARG, "R and m must be > 0");
    SoftGeom g{};
    g.B = d->B;
    g.C = d->C;
    g.H = d->H;
    g.W = d->W;
    for (int j = 0; j < 2; ++j) {
        const int b = d->grid[j];
        if (b < 1 || b > 128) return set_last_error(DP_PIX_E_UNSUPPORTED, "soft grids must be 1..128");
        if (!d->noise_free && !(d->eps[j] > 0.0)) return set_last_error(DP_PIX_E_INVALID_ARG, "eps must be > 0");
        g.b[j] = b;
        g.gr[j] = (d->H + b - 1) / b;
        g.gc[j] = (d->W + b - 1) / b;
        const int pr = g.gr[j] * b - d->H, pc = g.gc[j] * b - d->W;
        const int lr = d->pad_mode == DP_PIX_PAD_REFLECT ? d->H - 1 : d->H;
        const int lc = d->pad_mode == DP_PIX_PAD_REFLECT ? d->W - 1 : d->W;
        if (pr > lr || pc > lc) return set_last_error(DP_PIX_E_PAD_TOO_LARGE, "mirror padding reaches past the image");
        const double sigma = d->noise_free ? 0.0 : d->value_range * d->m / ((double)b * b * d->eps[j]);
        g.sigma[j] = (float)sigma;
        g.b2[j] = (float)(b * b);
        g.inv_b2[j] = is_pow2(b) ? 1.0f / (float)(b * b) : 0.0f;
    }
    g.R = (float)d->value_range;
    g.pad_mode = d->pad_mode;
    g.noise_free = d->noise_free ? 1 : 0;
    g.stream_id = d->stream_id;
    g.seed = d->seed;
    g.frame0 = d->frame0;
    g.pre_off1 = (int64_t)d->C * g.gr[0] * g.gc[0];
    g.pre_img = g.pre_off1 + (int64_t)d->C * g.gr[1] * g.gc[1];
    if ((uint64_t)d->B * (uint64_t)d->H * (uint64_t)d->W >= (1ull << 40))
        return set_last_error(DP_PIX_E_UNSUPPORTED, "soft batch too large");
    *sg = g;
    return DP_PIX_OK;
}

}  // namespace dppix

using namespace dppix;

extern "C" {

int dp_pix_soft_sizes(const dp_pix_soft_desc *d, uint64_t *pre_bytes) {
    SoftGeom sg;
    const int rc = soft_geometry(d, &sg);
    if (rc) return rc;
    if (!pre_bytes) return set_last_error(DP_PIX_E_INVALID_ARG, "pre_bytes is NULL");
    *pre_bytes = (uint64_t)sg.B * (uint64_t)sg.pre_img * 4ull;
    return DP_PIX_OK;
}

int dp_pix_soft_forward(const dp_pix_soft_desc *d, const float *x, const float *w, float *y, float *pre,
                        void *cuda_stream) {
    DPPIX_RANGE();
    SoftGeom sg;
    int rc = soft_geometry(d, &sg);
    if (rc) return rc;
    if (!x || !w || !y || !pre) return set_last_error(DP_PIX_E_INVALID_ARG, "null buffer");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const void *ptrs[3] = {x, w, y};
    int js = 0;
    cudaError_t e;
    if (soft_fast(sg, ptrs, 3, &js)) {
        e = soft_dispatch<FwdLaunch>(sg, js, x, w, y, pre, s);
    } else {
        const uint64_t cells = (uint64_t)sg.B * ((uint64_t)sg.gr[0] * sg.gc[0] + (uint64_t)sg.gr[1] * sg.gc[1]);
        prof_begin("k_soft_cells", s);
        k_soft_cells<<<soft_grid((const void *)k_soft_cells, 256, cells), 256, 0, s>>>(sg, x, pre);
        prof_end("k_soft_cells", s);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            const uint64_t px = (uint64_t)sg.B * sg.H * sg.W;
            prof_begin("k_soft_broadcast", s);
            k_soft_broadcast<<<soft_grid((const void *)k_soft_broadcast, 256, px), 256, 0, s>>>(sg, w, pre, y);
            prof_end("k_soft_broadcast", s);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) return set_last_error(DP_PIX_E_CUDA, cudaGetErrorString(e));
    return DP_PIX_OK;
}

int dp_pix_soft_backward(const dp_pix_soft_desc *d, const float *w, const float *gy, const float *pre, float *dx,
                         float *dw, float *d_ws, void *cuda_stream) {
    DPPIX_RANGE();
    SoftGeom sg;
    int rc = soft_geometry(d, &sg);
    if (rc) return rc;
    if (!w || !gy || !pre || !dx || !dw) return set_last_error(DP_PIX_E_INVALID_ARG, "null buffer");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const void *ptrs[4] = {w, gy, dx, dw};
    int js = 0;
    cudaError_t e;
    if (soft_fast(sg, ptrs, 4, &js)) {
        e = soft_dispatch<BwdLaunch>(sg, js, w, gy, pre, dx, dw, s);
    } else {
        if (!d_ws) return set_last_error(DP_PIX_E_INVALID_ARG, "this shape needs the workspace (dp_pix_soft_sizes bytes)");
        const uint64_t cells = (uint64_t)sg.B * ((uint64_t)sg.gr[0] * sg.gc[0] + (uint64_t)sg.gr[1] * sg.gc[1]);
        prof_begin("k_soft_coef", s);
        k_soft_coef<<<soft_grid((const void *)k_soft_coef, 256, cells), 256, 0, s>>>(sg, w, gy, pre, d_ws);
        prof_end("k_soft_coef", s);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            const uint64_t px = (uint64_t)sg.B * sg.H * sg.W;
            prof_begin("k_soft_grad", s);
            k_soft_grad<<<soft_grid((const void *)k_soft_grad, 256, px), 256, 0, s>>>(sg, gy, pre, d_ws, dx, dw);
            prof_end("k_soft_grad", s);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) return set_last_error(DP_PIX_E_CUDA, cudaGetErrorString(e));
    return DP_PIX_OK;
}

}  // extern "C"
