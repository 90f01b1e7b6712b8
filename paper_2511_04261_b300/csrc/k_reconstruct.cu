// k_reconstruct.cu -- rebuild pixelized frames from their records alone (Sec. VI-F; Alg. 2 steps 10-11).
//
// Geometry comes from each record's header on the device, so one launch serves any mix of records.
// Work item = (record, tile row, segment of tiles).  All output rows of a segment that lie in the same
// cell band of every tile are identical, so the CTA builds that row once in shared memory (each pixel
// takes its cell's stored value; u8 output rounds half to even) and streams it to every row of the band
// with the widest aligned stores.  Rows and columns past M, N (the padding) are cropped.
#include "common.cuh"

namespace dppix {
namespace {

constexpr int kThreads = 256;
constexpr int kRowBytes = 2048;  // shared-memory row pattern

struct RecGeom {
    int32_t ok;
    int32_t M, N, C, T, K, GR, GC, dtype, es, SR, nseg;
    int32_t grid[kMaxK];
    uint32_t count[kMaxK];
    uint64_t map_offset, rowidx_offset;
    uint64_t region_offset[kMaxK];
};

// Reads and checks a record header: geometry within the caller's bounds, and every section (tile-row
// index, map, region payloads) inside total_bytes <= cap, so that no later read leaves the record.
__device__ bool read_header(const uint8_t *rec, uint64_t cap, int max_M, int max_N, int max_C, RecGeom &rg, int oes) {
    const dp_pix_record_header *h = reinterpret_cast<const dp_pix_record_header *>(rec);
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
    for (int r = 0; r < rg.K; ++r) {
        rg.grid[r] = (int)h->grid[r];
        rg.count[r] = h->count[r];
        rg.region_offset[r] = h->region_offset[r];
        if (rg.grid[r] < 1 || rg.T % rg.grid[r] != 0) return false;
        const uint64_t cs = (uint64_t)(rg.T / rg.grid[r]);
        if (rg.region_offset[r] > total || (uint64_t)rg.count[r] * cs * cs * rg.C * rg.es > total - rg.region_offset[r])
            return false;
    }
    rg.map_offset = h->map_offset;
    rg.rowidx_offset = h->rowidx_offset;
    const uint64_t ntiles = (uint64_t)rg.GR * rg.GC;
    if (rg.map_offset > total || ntiles > total - rg.map_offset) return false;
    if (rg.rowidx_offset > total || (uint64_t)rg.GR * rg.K * 4 > total - rg.rowidx_offset || rg.rowidx_offset % 4)
        return false;
    const int tile_row_bytes = rg.T * rg.C * oes;
    int sr = kRowBytes / tile_row_bytes;
    rg.SR = sr < 1 ? 1 : (sr > 16 ? 16 : sr);
    rg.nseg = (rg.GC + rg.SR - 1) / rg.SR;
    return true;
}

template <int kOutF32>
__global__ void __launch_bounds__(kThreads)
    k_reconstruct(const uint8_t *records, int64_t record_stride, uint32_t n, uint8_t *out, int64_t out_frame_stride,
                  int64_t out_pitch, int max_M, int max_N, int max_C, int out_align, int32_t *status) {
    __shared__ __align__(16) uint8_t rowpat[kRowBytes];
    __shared__ RecGeom rg;
    __shared__ int32_t t_b[16], t_cs[16];
    __shared__ uint64_t t_off[16];
    constexpr int oes = kOutF32 ? 4 : 1;
    uint64_t base = 0;  // global item index of the current record's first item
    for (uint32_t i = 0; i < n; ++i) {
        const uint8_t *rec = records + (uint64_t)i * (uint64_t)record_stride;
        if (threadIdx.x == 0) {
            rg.ok = read_header(rec, (uint64_t)record_stride, max_M, max_N, max_C, rg, oes) ? 1 : 0;
            if (!rg.ok && blockIdx.x == 0) raise_status(status, DP_PIX_E_DEVICE, 0x200u | (i & 0xFFu));
        }
        __syncthreads();
        if (!rg.ok) {
            __syncthreads();
            continue;
        }
        const uint64_t items = (uint64_t)rg.GR * rg.nseg;
        // items of this record handled by this CTA: global index = base + k, k in [0, items)
        uint64_t first = (blockIdx.x >= base % gridDim.x) ? blockIdx.x - base % gridDim.x
                                                          : blockIdx.x + gridDim.x - base % gridDim.x;
        const int T = rg.T, C = rg.C;
        const int es = rg.es;
        uint8_t *obase = out + (uint64_t)i * (uint64_t)out_frame_stride;
        for (uint64_t k = first; k < items; k += gridDim.x) {
            const int ty = (int)(k / rg.nseg), sg = (int)(k - (uint64_t)ty * rg.nseg);
            const int tx0 = sg * rg.SR;
            const int ns = min(rg.SR, rg.GC - tx0);
            if (threadIdx.x < ns) {
                const int t = threadIdx.x;
                const uint8_t *maprow = rec + rg.map_offset + (uint64_t)ty * rg.GC;
                int r = maprow[tx0 + t];
                if (r >= rg.K) r = 0;
                uint32_t before = reinterpret_cast<const uint32_t *>(rec + rg.rowidx_offset)[ty * rg.K + r];
                for (int x = 0; x < tx0 + t; ++x) before += (maprow[x] == r);
                int b = rg.grid[r], cs = T / b;
                uint64_t off = rg.region_offset[r] + (uint64_t)before * (uint64_t)(cs * cs * C * es);
                if (before >= rg.count[r]) {  // inconsistent index: read the header instead of leaving the record
                    raise_status(status, DP_PIX_E_DEVICE, 0x300u | (i & 0xFFu));
                    b = T;
                    cs = 1;
                    off = 0;
                }
                t_b[t] = b;
                t_cs[t] = cs;
                t_off[t] = off;
            }
            __syncthreads();
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
                    const int nb = (j / t_b[t] + 1) * t_b[t];
                    jn = min(jn, nb);
                }
                // build the row pattern of rows [j, jn)
                const int elems = ns * T * C;
                for (int e = threadIdx.x; e < elems; e += blockDim.x) {
                    const int t = e / (T * C);
                    const int rem = e - t * (T * C);
                    const int px = rem / C, ch = rem - px * C;
                    const int b = t_b[t], cs = t_cs[t];
                    const int cell = (j / b) * cs + px / b;
                    const uint8_t *src = rec + t_off[t] + ((uint64_t)cell * C + ch) * es;
                    float v;
                    if (rg.dtype == DP_PIX_REC_F32)
                        v = *reinterpret_cast<const float *>(src);
                    else if (rg.dtype == DP_PIX_REC_U8)
                        v = (float)*src;
                    else
                        v = __fdiv_rn(__uint2float_rn(*reinterpret_cast<const uint32_t *>(src)), (float)(b * b));
                    if (kOutF32)
                        reinterpret_cast<float *>(rowpat)[e] = v;
                    else
                        rowpat[e] = (uint8_t)__float2uint_rn(fminf(fmaxf(v, 0.0f), 255.0f));
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
        base += items;
        __syncthreads();
    }
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

}  // namespace

cudaError_t launch_reconstruct(const uint8_t *records, int64_t record_stride, uint32_t n, uint8_t *out,
                               int64_t out_frame_stride, int64_t out_pitch, int out_type, int max_M, int max_N,
                               int max_C, int out_align, int32_t *status, cudaStream_t s) {
    int per_sm = 0;
    if (out_type == DP_PIX_OUT_F32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_reconstruct<1>, kThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_reconstruct<0>, kThreads, 0);
    if (per_sm < 1) per_sm = 1;
    const int grid = per_sm * sm_count();
    if (out_type == DP_PIX_OUT_F32) {
        prof_begin("k_reconstruct_f32", s);
        k_reconstruct<1><<<grid, kThreads, 0, s>>>(records, record_stride, n, out, out_frame_stride, out_pitch, max_M,
                                                   max_N, max_C, out_align, status);
        prof_end("k_reconstruct_f32", s);
    } else {
        prof_begin("k_reconstruct_u8", s);
        k_reconstruct<0><<<grid, kThreads, 0, s>>>(records, record_stride, n, out, out_frame_stride, out_pitch, max_M,
                                                   max_N, max_C, out_align, status);
        prof_end("k_reconstruct_u8", s);
    }
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
