// noalloc.cu -- dp_pix_release_noalloc: the release for callers that cannot allocate device memory.
//
// dp_pix_release needs a caller-provided workspace.  Some callers have no way to get one: code that runs
// while a CUDA graph is being captured (where cudaMalloc is not allowed), plug-ins whose host framework
// owns every device allocation and hands out only the input and output buffers, and real-time loops that
// must never enter an allocator.  For them this entry point takes the same inputs and outputs and uses a
// fixed scratch array that lives in the library itself instead of a workspace argument.
#include <cstdio>
#include <mutex>

#include "common.cuh"

namespace dppix {
namespace {

// The scratch: one array per GPU that loads the library, held until the process exits.
constexpr uint64_t kNoAllocScratchBytes = 16ull << 20;  // 16 MiB
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

// Device addresses of the scratch, found once per device (host code only sees a stand-in symbol).
std::mutex g_setup_mu;
uint8_t *g_scratch_ptr[64] = {nullptr};

int scratch_for_current_device(uint8_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        char msg[160];
        snprintf(msg, sizeof(msg), "dp_pix_release_noalloc: no usable CUDA device (%s)", cudaGetErrorString(e));
        return set_last_error(DP_PIX_E_CUDA, msg);
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            char msg[200];
            snprintf(msg, sizeof(msg), "dp_pix_release_noalloc: cudaGetSymbolAddress of the scratch failed (%s)",
                     cudaGetErrorString(e));
            return set_last_error(DP_PIX_E_CUDA, msg);
        }
        g_scratch_ptr[dev] = static_cast<uint8_t *>(p);
    }
    *out = g_scratch_ptr[dev];
    return DP_PIX_OK;
}

}  // namespace
}  // namespace dppix

extern "C" DPPIX_API int dp_pix_release_noalloc(dp_pix_plan_t plan, const void *d_frames, int64_t frame_stride,
                                                const void *d_region_src, int64_t src_pitch, int64_t src_frame_stride,
                                                uint32_t n_frames, uint32_t stream_id, uint64_t frame_idx0,
                                                void *d_records, int64_t record_stride, void *cuda_stream) {
    using namespace dppix;
    clear_last_error();
    if (!plan) return set_last_error(DP_PIX_E_INVALID_ARG, "dp_pix_release_noalloc: plan is NULL");
    if (n_frames == 0) return DP_PIX_OK;
    const uint64_t need = (uint64_t)n_frames * plan_ws_per_frame(plan);
    if (need > kNoAllocScratchBytes) {
        char msg[240];
        snprintf(msg, sizeof(msg),
                 "dp_pix_release_noalloc: %u frames need %llu bytes of scratch but the built-in scratch holds %llu "
                 "bytes; release fewer frames per call or use dp_pix_release with a workspace",
                 n_frames, (unsigned long long)need, (unsigned long long)kNoAllocScratchBytes);
        return set_last_error(DP_PIX_E_BUFFER_TOO_SMALL, msg);
    }
    uint8_t *scratch = nullptr;
    const int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    // Every scratch byte the kernels read is written earlier in the same call (tile offsets by the
    // finalize/rank kernel, rank keys and g-cell sums by the statistics kernel), so the previous call's
    // contents never leak into a result and nothing has to be cleared.
    return dp_pix_release(plan, d_frames, frame_stride, d_region_src, src_pitch, src_frame_stride, n_frames,
                          stream_id, frame_idx0, d_records, record_stride, scratch, kNoAllocScratchBytes, cuda_stream);
}
