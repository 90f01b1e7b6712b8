// k_utility.cu -- utility metrics of a release against its original (MSE, SSIM; Sec. VII-A, VII-B) and an
// edge-based simple/complex pixel mask (the Sobel operator named for region masks in Sec. VI-A).
//
// - k_sobel_mask: one CTA per (frame, 32 rows, 256 columns): the channel-sum intensity of the block and a
//   one-pixel mirrored border is staged in shared memory as u16, then each thread walks one column down the
//   32 rows with the 3 x 3 window in registers: Gx, Gy from the
//   Sobel taps in exact integers, mask = (Gx^2 + Gy^2 < tau) ? 1 : 0.
// - k_ssim: one CTA per (frame, 8 window rows, 512 window columns; 384 for C = 4); the 14 x 518-pixel input
//   block of both images is staged in shared memory as one plane per channel; each thread keeps, per channel,
//   the five exact integer window sums (Sx, Sy, Sxx, Syy, Sxy) of four adjacent columns' 7 x 7 windows (a
//   row's ten taps are three aligned words: the first window from dp4a, the others slid by a tap) and slides
//   them down the rows
//   (adding the entering row's 7 taps, subtracting the leaving one's).  The window value is evaluated from
//   the exact sums: with D = 49 Sxx - Sx^2 (and likewise), the 1/49^2 and 1/(49*48) factors of the means,
//   variances and covariance cancel, so SSIM = (2 Sx Sy + c1)(2 Dxy + c2) / ((Sx^2 + Sy^2 + c1)(Dx + Dy + c2))
//   with c1 = 49^2 C1 and c2 = 49*48 C2; only that last expression is rounded (fp32).  A thread's window
//   values of one channel (at most 32) are summed in fp32, those partial sums in fp64 per thread, block and
//   (atomically) frame.  The exact u64 sum of squared
//   sample differences is taken while staging, each block taking the pixels of its own window corners (the
//   last block row and column also the image's last six rows and columns).
// - k_utility_finalize: MSE = SSE / (M N C), SSIM = sum / ((M-6)(N-6) C).
#include "common.cuh"

namespace dppix {
namespace {

constexpr int kSobRows = 32, kSobCols = 256;
constexpr int kSsimRows = 8, kWin = 7;  // window rows per block; four window columns per thread
template <int C> struct SsimShape {
    static constexpr int COLS = C == 4 ? 384 : 512;  // window columns per block (staged block within 48 KB)
    static constexpr int THREADS = COLS / 4;
};

// Mirror index on both sides for one-pixel borders and clamped overhangs (n >= 2).
__device__ __forceinline__ int mirror2(int p, int n, int mode) {
    if (p < 0) p = mode == DP_PIX_PAD_REFLECT ? -p : -p - 1;
    if (p > n) p = n;
    if (p == n) p = mode == DP_PIX_PAD_REFLECT ? n - 2 : n - 1;
    return p;
}

template <int C>
__global__ void __launch_bounds__(kSobCols) k_sobel_mask(const uint8_t *frames, int M, int N, int64_t pitch,
                                                         int64_t fstride, int pad_mode, uint32_t tau, uint8_t *mask,
                                                         int64_t mpitch, int64_t mfstride) {
    __shared__ uint16_t I[kSobRows + 2][kSobCols + 2];
    const int x0 = blockIdx.x * kSobCols, y0 = blockIdx.y * kSobRows;
    const uint8_t *fb = frames + (int64_t)blockIdx.z * fstride;
    constexpr int W = kSobCols + 2;
    // blocks whose staged rows and columns all lie inside the frame index directly (no mirroring)
    const bool interior = x0 >= 1 && x0 - 1 + W <= N && y0 >= 1 && y0 - 1 + kSobRows + 2 <= M;
    if (interior) {
        const uint8_t *fb1 = fb + (int64_t)(y0 - 1) * pitch + (int64_t)(x0 - 1) * C;
        for (int idx = threadIdx.x; idx < (kSobRows + 2) * W; idx += blockDim.x) {
            const int r = idx / W, c = idx - r * W;
            const uint8_t *p = fb1 + (int64_t)r * pitch + c * C;
            uint32_t s = 0;
#pragma unroll
            for (int ch = 0; ch < C; ++ch) s += __ldg(p + ch);
            I[r][c] = (uint16_t)s;
        }
    } else {
        for (int idx = threadIdx.x; idx < (kSobRows + 2) * W; idx += blockDim.x) {
            const int r = idx / W, c = idx - r * W;
            const int y = mirror2(y0 - 1 + r, M, pad_mode), x = mirror2(x0 - 1 + c, N, pad_mode);
            const uint8_t *p = fb + (int64_t)y * pitch + (int64_t)x * C;
            uint32_t s = 0;
#pragma unroll
            for (int ch = 0; ch < C; ++ch) s += __ldg(p + ch);
            I[r][c] = (uint16_t)s;
        }
    }
    __syncthreads();
    const int c = threadIdx.x, x = x0 + c;
    if (x >= N) return;
    uint8_t *mb = mask + (int64_t)blockIdx.z * mfstride + x;
    const int rows = min(kSobRows, M - y0);
    // the 3 x 3 window slides down the column: rows r, r + 1, r + 2 held in registers
    int a0 = I[0][c], a1 = I[0][c + 1], a2 = I[0][c + 2];
    int b0 = I[1][c], b1 = I[1][c + 1], b2 = I[1][c + 2];
    for (int r = 0; r < rows; ++r) {
        const int c0 = I[r + 2][c], c1 = I[r + 2][c + 1], c2 = I[r + 2][c + 2];
        const int gx = (a2 - a0) + 2 * (b2 - b0) + (c2 - c0);
        const int gy = (c0 + 2 * c1 + c2) - (a0 + 2 * a1 + a2);
        mb[(int64_t)(y0 + r) * mpitch] = ((uint32_t)(gx * gx + gy * gy) < tau) ? 1 : 0;
        a0 = b0, a1 = b1, a2 = b2;
        b0 = c0, b1 = c1, b2 = c2;
    }
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Five exact sums (x, y, x^2, y^2, xy) of one staged channel row over window columns t4 .. t4 + 3 (taps t4 + i
// .. t4 + i + 6 for column i); S[i][q].  The row is a plane of one channel, so the ten taps are the first ten
// bytes of three aligned words: the first window's sums are dp4a of whole words (the seventh tap's word masked
// to three bytes), the others slide by one tap.
__device__ __forceinline__ void row_taps4(const uint8_t *xrow, const uint8_t *yrow, int t4, int (&S)[4][5]) {
    const uint32_t *wx = reinterpret_cast<const uint32_t *>(xrow + t4), *wy = reinterpret_cast<const uint32_t *>(yrow + t4);
    const uint32_t x0 = wx[0], x1 = wx[1], x2 = wx[2], y0 = wy[0], y1 = wy[1], y2 = wy[2];
    const uint32_t x1m = x1 & 0x00FFFFFFu, y1m = y1 & 0x00FFFFFFu;
    int sx = (int)(__dp4a(x0, 0x01010101u, 0u) + __dp4a(x1m, 0x01010101u, 0u));
    int sy = (int)(__dp4a(y0, 0x01010101u, 0u) + __dp4a(y1m, 0x01010101u, 0u));
    int sxx = (int)(__dp4a(x0, x0, 0u) + __dp4a(x1m, x1m, 0u));
    int syy = (int)(__dp4a(y0, y0, 0u) + __dp4a(y1m, y1m, 0u));
    int sxy = (int)(__dp4a(x0, y0, 0u) + __dp4a(x1m, y1m, 0u));
    S[0][0] = sx, S[0][1] = sy, S[0][2] = sxx, S[0][3] = syy, S[0][4] = sxy;
    // leaving taps 0, 1, 2 (bytes 0-2 of word 0) and entering taps 7, 8, 9 (byte 3 of word 1, bytes 0-1 of word 2)
    const int xo[3] = {(int)(x0 & 255u), (int)((x0 >> 8) & 255u), (int)((x0 >> 16) & 255u)};
    const int yo[3] = {(int)(y0 & 255u), (int)((y0 >> 8) & 255u), (int)((y0 >> 16) & 255u)};
    const int xn[3] = {(int)(x1 >> 24), (int)(x2 & 255u), (int)((x2 >> 8) & 255u)};
    const int yn[3] = {(int)(y1 >> 24), (int)(y2 & 255u), (int)((y2 >> 8) & 255u)};
#pragma unroll
    for (int i = 1; i < 4; ++i) {
        const int o = xo[i - 1], n = xn[i - 1], p = yo[i - 1], m = yn[i - 1];
        sx += n - o;
        sy += m - p;
        sxx += n * n - o * o;
        syy += m * m - p * p;
        sxy += n * m - o * p;
        S[i][0] = sx, S[i][1] = sy, S[i][2] = sxx, S[i][3] = syy, S[i][4] = sxy;
    }
}

// SSIM of one 7 x 7 window from its exact sums (the 1/49^2 and 1/(49*48) factors cancel; see the header).
// Every integer here fits in 32 bits (sums of 49 u8 samples: Sx <= 12495, 49 Sxx <= 1.6e8, Dx + Dy <=
// 3.2e8), so nothing touches the FP64 pipe.
__device__ __forceinline__ float ssim_of(const int *S, float c1, float c2) {
    const int sx = S[0], sy = S[1];
    const int dx = 49 * S[2] - sx * sx;
    const int dy = 49 * S[3] - sy * sy;
    const int dxy = 49 * S[4] - sx * sy;
    const float num = (2.0f * (float)(sx * sy) + c1) * (2.0f * (float)dxy + c2);
    const float den = ((float)(sx * sx + sy * sy) + c1) * ((float)(dx + dy) + c2);
    return __fdiv_rn(num, den);
}

template <int C>
__global__ void __launch_bounds__(SsimShape<C>::THREADS) k_ssim(const uint8_t *x, const uint8_t *y, int M, int N,
                                                              int64_t px, int64_t py, int64_t fsx, int64_t fsy, float c1,
                                                              float c2, dp_pix_utility_t *out) {
    constexpr int COLS = SsimShape<C>::COLS, NT = SsimShape<C>::THREADS;
    constexpr int SR = kSsimRows + kWin - 1, SC = COLS + kWin - 1;
    constexpr int SCP = (SC + 2 + 3) / 4 * 4;  // bytes per staged plane row: the last thread reads up to SC + 1
    __shared__ __align__(16) uint8_t xs[C * SR * SCP], ys[C * SR * SCP];  // plane ch, row r at (ch SR + r) SCP
    __shared__ double part[(NT + 31) / 32];
    const int f = blockIdx.z;
    const int cy0 = blockIdx.y * kSsimRows, cx0 = blockIdx.x * COLS;  // first window (top-left corner)
    const int nwy = M - kWin + 1, nwx = N - kWin + 1;                 // windows per column / row
    const int rows_in = min(SR, M - cy0), cols_in = min(SC, N - cx0);
    const uint8_t *xb = x + (int64_t)f * fsx + (int64_t)cy0 * px + (int64_t)cx0 * C;
    const uint8_t *yb = y + (int64_t)f * fsy + (int64_t)cy0 * py + (int64_t)cx0 * C;
    const int nb = cols_in * C;
    // staging into channel planes; the squared differences of the pixels this block owns (its window corners,
    // extended to the image's last rows / columns in the last block row / column) are summed on the way
    const int ro = blockIdx.y + 1 == gridDim.y ? rows_in : kSsimRows;
    const int co = (blockIdx.x + 1 == gridDim.x ? cols_in : COLS) * C;
    unsigned long long e = 0;
    for (int r = 0; r < rows_in; ++r)
        for (int k = threadIdx.x; k < nb; k += blockDim.x) {
            const int xv = __ldg(xb + (int64_t)r * px + k), yv = __ldg(yb + (int64_t)r * py + k);
            const int pxl = k / C, ch = k - pxl * C;
            xs[(ch * SR + r) * SCP + pxl] = (uint8_t)xv;
            ys[(ch * SR + r) * SCP + pxl] = (uint8_t)yv;
            if (r < ro && k < co) e += (unsigned long long)((xv - yv) * (xv - yv));
        }
    e = warp_sum_u64(e);
    if ((threadIdx.x & 31) == 0 && e) atomicAdd(reinterpret_cast<unsigned long long *>(&out[f].sse), e);
    __syncthreads();
    const int t4 = 4 * threadIdx.x;
    const int nvalid = min(4, nwx - (cx0 + t4));  // window columns of this thread inside the image
    const int nrows = min(kSsimRows, nwy - cy0);
    double acc = 0.0;
    if (nvalid > 0) {
#pragma unroll 1
        for (int ch = 0; ch < C; ++ch) {
            int V[4][5] = {};
            for (int r = 0; r < kWin; ++r) {
                int a[4][5];
                row_taps4(xs + (ch * SR + r) * SCP, ys + (ch * SR + r) * SCP, t4, a);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int q = 0; q < 5; ++q) V[i][q] += a[i][q];
            }
            float part_sum = 0.0f;  // at most 4 x 8 window values in [-1, 1] per channel
            for (int i = 0; i < nrows; ++i) {
#pragma unroll
                for (int w = 0; w < 4; ++w)
                    if (w < nvalid) part_sum += ssim_of(V[w], c1, c2);
                if (i + 1 < nrows) {
                    int a[4][5], d[4][5];
                    row_taps4(xs + (ch * SR + i + kWin) * SCP, ys + (ch * SR + i + kWin) * SCP, t4, a);
                    row_taps4(xs + (ch * SR + i) * SCP, ys + (ch * SR + i) * SCP, t4, d);
#pragma unroll
                    for (int w = 0; w < 4; ++w)
#pragma unroll
                        for (int q = 0; q < 5; ++q) V[w][q] += a[w][q] - d[w][q];
                }
            }
            acc += (double)part_sum;
        }
    }
    acc = warp_sum_f64(acc);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < (NT + 31) / 32; ++w) sum += part[w];
        atomicAdd(&out[f].ssim_sum, sum);
    }
}

__global__ void k_utility_finalize(dp_pix_utility_t *out, uint32_t n, int M, int N, int C) {
    const uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    const uint64_t w = (uint64_t)(M - kWin + 1) * (uint64_t)(N - kWin + 1);
    out[f].windows = w;
    out[f].mse = (double)out[f].sse / ((double)M * (double)N * (double)C);
    out[f].ssim = out[f].ssim_sum / ((double)w * (double)C);
}

}  // namespace
}  // namespace dppix

using namespace dppix;

extern "C" {

int dp_pix_sobel_mask(const void *d_frames, int32_t M, int32_t N, int32_t C, int64_t row_pitch, int64_t frame_stride,
                      uint32_t n_frames, int32_t pad_mode, uint32_t tau, void *d_mask, int64_t mask_pitch,
                      int64_t mask_frame_stride, void *cuda_stream) {
    DPPIX_RANGE();
    if (n_frames == 0) return DP_PIX_OK;  // nothing to do
    if (!d_frames || !d_mask) return set_last_error(DP_PIX_E_INVALID_ARG, "null frame or mask pointer");
    if (M < 2 || N < 2 || C < 1 || C > 4 || n_frames > 65535)
        return set_last_error(DP_PIX_E_INVALID_ARG, "need M, N >= 2, C in 1..4, n_frames <= 65535");
    if (M > (1 << 24) || N > (1 << 24)) return set_last_error(DP_PIX_E_UNSUPPORTED, "M or N too large");
    if (pad_mode != DP_PIX_PAD_REFLECT && pad_mode != DP_PIX_PAD_SYMMETRIC)
        return set_last_error(DP_PIX_E_INVALID_ARG, "pad_mode must be REFLECT or SYMMETRIC");
    if (row_pitch < (int64_t)N * C || mask_pitch < N)
        return set_last_error(DP_PIX_E_INVALID_ARG, "row_pitch < N*C or mask_pitch < N");
    if (n_frames > 1 && (frame_stride < row_pitch * M || mask_frame_stride < mask_pitch * M))
        return set_last_error(DP_PIX_E_INVALID_ARG, "frame strides smaller than a frame");
    const int rc = cuda_device_ok();
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const dim3 grid((N + kSobCols - 1) / kSobCols, (M + kSobRows - 1) / kSobRows, n_frames);
    const uint8_t *fr = static_cast<const uint8_t *>(d_frames);
    uint8_t *mk = static_cast<uint8_t *>(d_mask);
    prof_begin("k_sobel_mask", s);
    switch (C) {
        case 1: k_sobel_mask<1><<<grid, kSobCols, 0, s>>>(fr, M, N, row_pitch, frame_stride, pad_mode, tau, mk, mask_pitch, mask_frame_stride); break;
        case 2: k_sobel_mask<2><<<grid, kSobCols, 0, s>>>(fr, M, N, row_pitch, frame_stride, pad_mode, tau, mk, mask_pitch, mask_frame_stride); break;
        case 3: k_sobel_mask<3><<<grid, kSobCols, 0, s>>>(fr, M, N, row_pitch, frame_stride, pad_mode, tau, mk, mask_pitch, mask_frame_stride); break;
        default: k_sobel_mask<4><<<grid, kSobCols, 0, s>>>(fr, M, N, row_pitch, frame_stride, pad_mode, tau, mk, mask_pitch, mask_frame_stride); break;
    }
    prof_end("k_sobel_mask", s);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DP_PIX_OK : set_last_error(DP_PIX_E_CUDA, cudaGetErrorString(e));
}

int dp_pix_utility(const void *d_x, const void *d_y, int32_t M, int32_t N, int32_t C, int64_t pitch_x, int64_t pitch_y,
                   int64_t frame_stride_x, int64_t frame_stride_y, uint32_t n_frames, dp_pix_utility_t *d_out,
                   void *cuda_stream) {
    DPPIX_RANGE();
    if (n_frames == 0) return DP_PIX_OK;  // nothing to do
    if (!d_x || !d_y || !d_out) return set_last_error(DP_PIX_E_INVALID_ARG, "null pointer");
    if (M < kWin || N < kWin || C < 1 || C > 4 || n_frames > 65535)
        return set_last_error(DP_PIX_E_INVALID_ARG, "need M, N >= 7, C in 1..4, n_frames <= 65535");
    if (M > (1 << 24) || N > (1 << 24)) return set_last_error(DP_PIX_E_UNSUPPORTED, "M or N too large");
    if (pitch_x < (int64_t)N * C || pitch_y < (int64_t)N * C)
        return set_last_error(DP_PIX_E_INVALID_ARG, "row pitch < N*C");
    if (n_frames > 1 && (frame_stride_x < pitch_x * M || frame_stride_y < pitch_y * M))
        return set_last_error(DP_PIX_E_INVALID_ARG, "frame strides smaller than a frame");
    if (reinterpret_cast<uintptr_t>(d_out) % 8) return set_last_error(DP_PIX_E_INVALID_ARG, "d_out not 8-byte aligned");
    const int rc = cuda_device_ok();
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMemsetAsync(d_out, 0, sizeof(dp_pix_utility_t) * n_frames, s);
    if (e != cudaSuccess) return set_last_error(DP_PIX_E_CUDA, cudaGetErrorString(e));
    const uint8_t *xp = static_cast<const uint8_t *>(d_x), *yp = static_cast<const uint8_t *>(d_y);
    const float L = 255.0f;
    const float c1 = (float)(49.0 * 49.0 * (0.01 * L) * (0.01 * L));
    const float c2 = (float)(49.0 * 48.0 * (0.03 * L) * (0.03 * L));
    const int nwy = M - kWin + 1, nwx = N - kWin + 1;
#define DPPIX_SSIM(CC)                                                                                            \
    k_ssim<CC><<<dim3((nwx + SsimShape<CC>::COLS - 1) / SsimShape<CC>::COLS, (nwy + kSsimRows - 1) / kSsimRows,     \
                      n_frames),                                                                                 \
                 SsimShape<CC>::THREADS, 0, s>>>(xp, yp, M, N, pitch_x, pitch_y, frame_stride_x, frame_stride_y, c1, \
                                                 c2, d_out)
    prof_begin("k_ssim", s);
    switch (C) {
        case 1: DPPIX_SSIM(1); break;
        case 2: DPPIX_SSIM(2); break;
        case 3: DPPIX_SSIM(3); break;
        default: DPPIX_SSIM(4); break;
    }
#undef DPPIX_SSIM
    prof_end("k_ssim", s);
    k_utility_finalize<<<(n_frames + 127) / 128, 128, 0, s>>>(d_out, n_frames, M, N, C);
    e = cudaGetLastError();
    return e == cudaSuccess ? DP_PIX_OK : set_last_error(DP_PIX_E_CUDA, cudaGetErrorString(e));
}

}  // extern "C"
