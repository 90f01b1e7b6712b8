// api.cu -- the C ABI of libdppix (see include/dppix.h): plans, release orchestration, store,
// reconstruction, status, and launch accounting.
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"

static_assert(sizeof(dp_pix_record_header) == DP_PIX_RECORD_HEADER_BYTES, "record header must be 512 bytes");
static_assert(offsetof(dp_pix_record_header, total_bytes) == 96, "record header layout");
static_assert(offsetof(dp_pix_record_header, grid) == 112, "record header layout");
static_assert(offsetof(dp_pix_record_header, eps) == 144, "record header layout");
static_assert(offsetof(dp_pix_record_header, sigma) == 208, "record header layout");
static_assert(offsetof(dp_pix_record_header, count) == 272, "record header layout");
static_assert(offsetof(dp_pix_record_header, region_offset) == 304, "record header layout");
static_assert(offsetof(dp_pix_record_header, payload_offset) == 376, "record header layout");

struct dp_pix_plan_s {
    dppix::Geom g;
};

// Device status word of the library: [0] first error code, [1] detail.
__device__ int32_t g_dppix_status[2];

namespace dppix {
namespace {

thread_local char t_err[512] = "";

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(DP_PIX_E_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

uint64_t a16(uint64_t x) { return (x + 15ull) & ~15ull; }
uint64_t a256(uint64_t x) { return (x + 255ull) & ~255ull; }
int64_t gcd64(int64_t a, int64_t b) {
    while (b) {
        const int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}
int bits_for(unsigned __int128 v) {
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

// ---- launch accounting -------------------------------------------------------------------------------
struct ProfEntry {
    uint64_t launches = 0;
    double total_ms = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};
std::mutex g_prof_mu;
std::map<std::string, ProfEntry> g_prof;
bool g_prof_timing = false;

}  // namespace

void prof_begin(const char *name, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfEntry &e = g_prof[name];
    e.launches++;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (g_prof_timing && cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone) {
        cudaEvent_t a = nullptr, b = nullptr;
        if (cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess) {
            cudaEventRecord(a, s);
            e.pending.emplace_back(a, b);
        }
    }
}

void prof_end(const char *name, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_timing) return;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
    ProfEntry &e = g_prof[name];
    if (!e.pending.empty()) cudaEventRecord(e.pending.back().second, s);
}

int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cached[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 1;
    }
    return cached[dev];
}

uint64_t plan_ws_per_frame(const dp_pix_plan_s *plan) { return plan ? plan->g.ws_per_frame : 0; }

int set_last_error(int code, const char *msg) { return fail(code, "%s", msg); }

void clear_last_error() { t_err[0] = 0; }

// Blocks of `kernel` resident per SM at `threads` threads and `smem` dynamic bytes, on the current device.
// The first call for a kernel on a device also raises its dynamic shared-memory limit to the device's opt-in
// maximum, so launches never need to set it again; results are cached (these queries cost microseconds of
// host time per launch otherwise).
int launch_prep(const void *kernel, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, int, size_t>, int> occ;
    static std::map<std::pair<const void *, int>, bool> raised;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(kernel, dev, threads, smem);
    auto it = occ.find(key);
    if (it != occ.end()) return it->second;
    if (!raised[std::make_pair(kernel, dev)]) {
        // the dynamic limit is the opt-in maximum less the kernel's static shared memory
        int optin = 0;
        cudaFuncAttributes fa{};
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (optin > 0 && cudaFuncGetAttributes(&fa, kernel) == cudaSuccess && optin > (int)fa.sharedSizeBytes)
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
        cudaGetLastError();  // a refused attribute surfaces at the launch, not here
        raised[std::make_pair(kernel, dev)] = true;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    occ[key] = per_sm;
    return per_sm;
}

// Non-blocking side streams of the current device (created once, kept for the process).
cudaStream_t *side_streams(int n) {
    static std::mutex mu;
    static cudaStream_t streams[64][8] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || n < 1 || n > 8) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < n; ++i)
        if (!streams[dev][i] && cudaStreamCreateWithFlags(&streams[dev][i], cudaStreamNonBlocking) != cudaSuccess) {
            streams[dev][i] = nullptr;
            return nullptr;
        }
    return streams[dev];
}

int32_t *status_word() {
    static std::mutex mu;
    static int32_t *cached[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);  // host threads making their first call on a device at once
    if (!cached[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_dppix_status) != cudaSuccess) return nullptr;
        cached[dev] = static_cast<int32_t *>(p);
    }
    return cached[dev];
}

namespace {

int make_geom(const dp_pix_desc *d, Geom &g) {
    memset(&g, 0, sizeof(g));
    if (!d) return fail(DP_PIX_E_INVALID_ARG, "desc is NULL");
    if (d->M < 1 || d->N < 1) return fail(DP_PIX_E_INVALID_ARG, "M and N must be >= 1");
    if (d->C < 1 || d->C > 4) return fail(DP_PIX_E_INVALID_ARG, "C must be in 1..4");
    if (d->K < 1 || d->K > kMaxK) return fail(DP_PIX_E_INVALID_ARG, "K must be in 1..8");
    if (d->row_pitch < (int64_t)d->N * d->C) return fail(DP_PIX_E_INVALID_ARG, "row_pitch < N*C");
    if (!(d->value_range > 0) || !(d->m > 0)) return fail(DP_PIX_E_INVALID_ARG, "value_range and m must be > 0");
    if (d->pad_mode != DP_PIX_PAD_REFLECT && d->pad_mode != DP_PIX_PAD_SYMMETRIC && d->pad_mode != DP_PIX_PAD_NONE)
        return fail(DP_PIX_E_INVALID_ARG, "bad pad_mode");
    if (d->pad_mode == DP_PIX_PAD_NONE && d->region_source == DP_PIX_SRC_VARIANCE)
        return fail(DP_PIX_E_UNSUPPORTED, "pad_mode NONE with variance classes (tiles of unequal sample counts)");
    if (d->region_source < 0 || d->region_source > 3) return fail(DP_PIX_E_INVALID_ARG, "bad region_source");
    if (d->record_dtype < 0 || d->record_dtype > 2) return fail(DP_PIX_E_INVALID_ARG, "bad record_dtype");
    if ((d->region_source == DP_PIX_SRC_MASK_U8 || d->region_source == DP_PIX_SRC_MATTE_F32) && d->K != 2)
        return fail(DP_PIX_E_INVALID_ARG, "mask and matte sources need K == 2");
    if (d->value_range > 255.0) return fail(DP_PIX_E_UNSUPPORTED, "u8 frames need value_range <= 255");
    int64_t T = 1;
    int64_t gg = 0;
    int bmin = 1 << 30;
    for (int r = 0; r < d->K; ++r) {
        const int b = d->grid[r];
        if (b < 1) return fail(DP_PIX_E_INVALID_ARG, "grid[%d] must be >= 1", r);
        if (b > kMaxT) return fail(DP_PIX_E_UNSUPPORTED, "grid[%d] = %d > %d", r, b, kMaxT);
        if (!d->noise_free && !(d->eps[r] > 0)) return fail(DP_PIX_E_INVALID_ARG, "eps[%d] must be > 0", r);
        T = T / gcd64(T, b) * b;
        if (T > kMaxT) return fail(DP_PIX_E_UNSUPPORTED, "T = lcm(grids) > %d", kMaxT);
        gg = gcd64(gg, b);
        bmin = b < bmin ? b : bmin;
    }
    if (T * T * d->C > kMaxTileBytes) return fail(DP_PIX_E_UNSUPPORTED, "T*T*C > %d", kMaxTileBytes);
    g.M = d->M; g.N = d->N; g.C = d->C; g.K = d->K; g.T = (int)T;
    g.GR = (int)((d->M + T - 1) / T);
    g.GC = (int)((d->N + T - 1) / T);
    g.PR = (int)(g.GR * T - d->M);
    g.PC = (int)(g.GC * T - d->N);
    const int64_t lim_r = d->pad_mode == DP_PIX_PAD_REFLECT ? d->M - 1 : d->M;
    const int64_t lim_c = d->pad_mode == DP_PIX_PAD_REFLECT ? d->N - 1 : d->N;
    if (d->pad_mode != DP_PIX_PAD_NONE && (g.PR > lim_r || g.PC > lim_c))
        return fail(DP_PIX_E_PAD_TOO_LARGE, "padding (%d, %d) reaches past the image (%d x %d)", g.PR, g.PC, d->M, d->N);
    const uint64_t ntiles = (uint64_t)g.GR * (uint64_t)g.GC;
    if (ntiles > (uint64_t)kMaxFrameTiles) return fail(DP_PIX_E_UNSUPPORTED, "more than %d tiles per frame", kMaxFrameTiles);
    g.ntiles = (uint32_t)ntiles;
    g.pad_mode = d->pad_mode;
    g.source = d->region_source;
    g.dtype = d->record_dtype;
    g.noise_free = d->noise_free ? 1 : 0;
    g.es = d->record_dtype == DP_PIX_REC_U8 ? 1 : 4;
    g.pitch = d->row_pitch;
    g.R = d->value_range;
    g.R_f = (float)d->value_range;
    g.m = d->m;
    g.matte_thr = d->matte_threshold;
    g.seed = d->seed;
    uint64_t maxcells = 0;
    for (int r = 0; r < d->K; ++r) {
        const int b = d->grid[r];
        g.grid[r] = b;
        g.cells_side[r] = (int)(T / b);
        g.eps[r] = d->eps[r];
        // Eq. 11 with Eq. 8: sigma = R m / (b^2 eps)
        g.sigma[r] = d->value_range * d->m / ((double)b * (double)b * d->eps[r]);
        g.sigma_f[r] = (float)g.sigma[r];
        g.b2_f[r] = (float)(b * b);
        g.inv_b2_f[r] = (b & (b - 1)) == 0 ? 1.0f / (float)(b * b) : 0.0f;
        const uint64_t c = (uint64_t)g.cells_side[r] * g.cells_side[r];
        maxcells = c > maxcells ? c : maxcells;
    }
    g.b_min = bmin;
    g.g = (int)gg;
    g.rowidx_offset = kHeaderBytes;
    g.map_offset = g.rowidx_offset + a16((uint64_t)g.GR * g.K * 4);
    g.payload_offset = g.map_offset + a16(ntiles);
    g.record_cap = g.payload_offset + a16(ntiles * maxcells * g.C * g.es) + 16ull * g.K;
    if (g.record_cap >= (1ull << 32)) return fail(DP_PIX_E_UNSUPPORTED, "record larger than 4 GiB");
    const int TC = (int)T * g.C;
    if (g.source == DP_PIX_SRC_VARIANCE) {
        if (TC % 4 != 0) return fail(DP_PIX_E_UNSUPPORTED, "VARIANCE needs T*C to be a multiple of 4");
        if (ntiles > (uint64_t)kMaxRankTiles) return fail(DP_PIX_E_UNSUPPORTED, "VARIANCE ranks at most %d tiles", kMaxRankTiles);
        g.idx_bits = bits_for((unsigned __int128)(ntiles - 1));
        if (g.idx_bits < 1) g.idx_bits = 1;
        const unsigned __int128 n = (unsigned __int128)TC * (unsigned __int128)T;
        const unsigned __int128 kmax = (n * 255u) * (n * 255u) / 4u + 1u;
        if (bits_for(kmax) + g.idx_bits > 63) return fail(DP_PIX_E_UNSUPPORTED, "rank key does not fit 63 bits");
        g.val_bits = bits_for(kmax) + g.idx_bits;
        g.var_onepass = (g.g >= 4 && g.g <= 16) ? 1 : 0;
    }
    // workspace layout (per frame)
    uint64_t off = 0;
    g.ws_tileoff = off;
    off = a256(off + 4ull * ntiles);
    g.ws_tilelist = off;
    off = a256(off + 4ull * ntiles);
    g.ws_keys = off;
    if (g.source == DP_PIX_SRC_VARIANCE) off = a256(off + 8ull * ntiles);
    g.ws_gsum = off;
    if (g.var_onepass) {
        g.gx_cells = (int)(g.GC * T / g.g);
        g.gy_cells = (int)(g.GR * T / g.g);
        g.gpitch = (g.gx_cells * g.C + 7) / 8 * 8;
        off = a256(off + 2ull * (uint64_t)g.gpitch * g.gy_cells);
    }
    g.ws_per_frame = off;
    g.fused_px = 1024;
    g.fused_threads = 128;
    g.split = 1;
    g.fused_cap = 0;
    for (int r = 0; r < 10; ++r) {  // the Philox key schedule: each round adds the Weyl constants
        g.rkey[2 * r] = (uint32_t)d->seed + (uint32_t)r * 0x9E3779B9u;
        g.rkey[2 * r + 1] = (uint32_t)(d->seed >> 32) + (uint32_t)r * 0xBB67AE85u;
    }
    g.wait_tries = kWaitTries;
    g.test_short_tx = 0;
    g.test_shrink = 0;
    // staged segment: S tiles of one tile row, S*T*C a multiple of 16 when possible
    int s0 = 16 / (int)gcd64(TC, 16);
    int S = s0 * (int)((384 + (int64_t)s0 * TC - 1) / ((int64_t)s0 * TC));
    if (S > 16) S = 16 / s0 * s0;
    if (S < 1) S = 1;
    const int vb_rel = (int)T / bmin;
    const int vb_stat = g.var_onepass ? (int)T / g.g : 0;
    const int vbands = vb_rel > vb_stat ? vb_rel : vb_stat;
    auto smem_for = [&](int s) { return (int64_t)T * (int64_t)a16((uint64_t)s * TC) + (int64_t)s * vbands * TC * 2; };
    while (S > 1 && smem_for(S) > 96 * 1024) S = (S - s0 >= 1) ? S - s0 : S - 1;
    if (smem_for(S) > 200 * 1024) return fail(DP_PIX_E_UNSUPPORTED, "tile too large to stage");
    g.seg_tiles = S;
    g.seg_per_row = (g.GC + S - 1) / S;
    g.seg_rowstride = (int)a16((uint64_t)S * TC);
    g.vbands = vb_rel;
    set_release_units(g);
    return DP_PIX_OK;
}

}  // namespace

int plan_geometry(const dp_pix_desc *d, Geom &g) { return make_geom(d, g); }

// Release work units of each region for the plan's segment width (k_release): a cell's row parts follow the
// byte budget of rel_parts, and are doubled further while an item of S tiles of the region would hold fewer
// than kRelMinUnits units (large cells of few channels would otherwise leave most of a CTA idle).
void set_release_units(Geom &g) {
    const int S = g.seg_tiles > 0 ? g.seg_tiles : 1;
    int P[kMaxK];
    g.rel_pmax = 1;
    for (int r = 0; r < g.K; ++r) {
        const int b = g.grid[r], cs = g.cells_side[r];
        int p = rel_parts(b, g.C);
        while (S * cs * cs * p < kRelMinUnits && 2 * p <= b && p < 32) p *= 2;
        P[r] = p;
        if (p > g.rel_pmax) g.rel_pmax = p;
    }
    for (int r = 0; r < g.K; ++r) {
        int lp = 0;
        while ((1 << lp) < P[r]) ++lp;
        g.rel_lp[r] = lp;
        const int units = g.cells_side[r] * g.cells_side[r] * P[r];
        g.rel_units[r] = (units + g.rel_pmax - 1) / g.rel_pmax * g.rel_pmax;
    }
}

int check_cuda_device() {
    int n = 0;
    const cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n < 1) return fail(DP_PIX_E_CUDA, "no CUDA device available: %s", cudaGetErrorString(e));
    return DP_PIX_OK;
}

int cuda_device_ok() { return check_cuda_device(); }

namespace {

}  // namespace
}  // namespace dppix

using namespace dppix;

extern "C" {

int dp_pix_version(void) { return 10000; }

const char *dp_pix_last_error(void) { return t_err; }

int dp_pix_plan(const dp_pix_desc *d, dp_pix_plan_t *out, dp_pix_sizes *sz) {
    DPPIX_RANGE();
    t_err[0] = 0;
    if (!out) return fail(DP_PIX_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    Geom g;
    const int rc = make_geom(d, g);
    if (rc) return rc;
    dp_pix_plan_s *p = new (std::nothrow) dp_pix_plan_s;
    if (!p) return fail(DP_PIX_E_INVALID_ARG, "out of host memory");
    p->g = g;
    *out = p;
    if (sz) {
        memset(sz, 0, sizeof(*sz));
        sz->record_bytes = g.record_cap;
        sz->workspace_per_frame = g.ws_per_frame;
        sz->workspace_fixed = 0;
        sz->T = g.T; sz->GR = g.GR; sz->GC = g.GC; sz->PR = g.PR; sz->PC = g.PC;
        sz->num_tiles = g.ntiles;
        uint64_t maxcells = 0;
        for (int r = 0; r < g.K; ++r) {
            const uint64_t c = (uint64_t)g.cells_side[r] * g.cells_side[r];
            maxcells = c > maxcells ? c : maxcells;
            sz->sigma[r] = g.sigma[r];
        }
        sz->max_values = (uint64_t)g.ntiles * maxcells * g.C;
    }
    return DP_PIX_OK;
}

int dp_pix_plan_destroy(dp_pix_plan_t plan) {
    delete plan;
    return DP_PIX_OK;
}

int dp_pix_plan_tune(dp_pix_plan_t plan, int knob, int value) {
    t_err[0] = 0;
    if (!plan) return fail(DP_PIX_E_INVALID_ARG, "plan is NULL");
    switch (knob) {
        case DP_PIX_TUNE_FUSED_PX:
            if (value < 64 || value > 2048) return fail(DP_PIX_E_INVALID_ARG, "fused pixel columns must be 64..2048");
            plan->g.fused_px = value;
            return DP_PIX_OK;
        case DP_PIX_TUNE_FUSED_THREADS:
            if (value != 96 && value != 128 && value != 192 && value != 256)
                return fail(DP_PIX_E_INVALID_ARG, "fused threads must be 96, 128, 192 or 256");
            plan->g.fused_threads = value;
            return DP_PIX_OK;
        case DP_PIX_TUNE_SPLIT:
            if (value < 1 || value > kMaxSplit) return fail(DP_PIX_E_INVALID_ARG, "split must be 1..%d", kMaxSplit);
            plan->g.split = value;
            return DP_PIX_OK;
        case DP_PIX_TUNE_FUSED_CAP:
            if (value < 0 || value > 32) return fail(DP_PIX_E_INVALID_ARG, "fused blocks per SM must be 0..32");
            plan->g.fused_cap = value;
            return DP_PIX_OK;
        case DP_PIX_TUNE_WAIT_TRIES:
            if (value < 1 || value > (int)kWaitTries) return fail(DP_PIX_E_INVALID_ARG, "wait tries must be 1..%u", kWaitTries);
            plan->g.wait_tries = (uint32_t)value;
            return DP_PIX_OK;
        case DP_PIX_TUNE_TEST_SHORT_TX:
            if (value != 0 && value != 1) return fail(DP_PIX_E_INVALID_ARG, "the short-copy test knob is 0 or 1");
            plan->g.test_short_tx = value ? 16u : 0u;
            return DP_PIX_OK;
        case DP_PIX_TUNE_TEST_SHRINK:
            if (value < 0 || value > (1 << 20)) return fail(DP_PIX_E_INVALID_ARG, "the shrink test knob is 0..2^20");
            plan->g.test_shrink = (uint32_t)value;
            return DP_PIX_OK;
        default:
            return fail(DP_PIX_E_INVALID_ARG, "unknown knob %d", knob);
    }
}

int dp_pix_plan_tuning(dp_pix_plan_t plan, int knob, int *value) {
    t_err[0] = 0;
    if (!plan || !value) return fail(DP_PIX_E_INVALID_ARG, "plan or value is NULL");
    switch (knob) {
        case DP_PIX_TUNE_FUSED_PX: *value = plan->g.fused_px; return DP_PIX_OK;
        case DP_PIX_TUNE_FUSED_THREADS: *value = plan->g.fused_threads; return DP_PIX_OK;
        case DP_PIX_TUNE_SPLIT: *value = plan->g.split; return DP_PIX_OK;
        case DP_PIX_TUNE_FUSED_CAP: *value = plan->g.fused_cap; return DP_PIX_OK;
        case DP_PIX_TUNE_WAIT_TRIES: *value = (int)plan->g.wait_tries; return DP_PIX_OK;
        case DP_PIX_TUNE_TEST_SHORT_TX: *value = plan->g.test_short_tx ? 1 : 0; return DP_PIX_OK;
        case DP_PIX_TUNE_TEST_SHRINK: *value = (int)plan->g.test_shrink; return DP_PIX_OK;
        default: return fail(DP_PIX_E_INVALID_ARG, "unknown knob %d", knob);
    }
}

}  // extern "C"

namespace {

// Output of the fused release + reconstruction; `fused` tells whether the kernels wrote it.
struct FusedOut {
    uint8_t *out;
    int64_t frame_stride, pitch;
    int type, align;
    bool fused;
    int stage;       // variance classes: 0 everything, 1 statistics and rank only, 2 the emission only
    int max_per_sm;  // blocks per SM of the fused kernel (0: its occupancy limit)
};

int release_impl(dp_pix_plan_t plan, const void *d_frames, int64_t frame_stride, const void *d_region_src,
                 int64_t src_pitch, int64_t src_frame_stride, uint32_t n_frames, uint32_t stream_id, uint64_t frame_idx0,
                 void *d_records, int64_t record_stride, void *d_ws, uint64_t ws_bytes, void *cuda_stream,
                 FusedOut *fo, const dp_pix_frame_key *keys = nullptr) {
    if (!plan) return fail(DP_PIX_E_INVALID_ARG, "plan is NULL");
    const Geom &g = plan->g;
    if (n_frames == 0) return DP_PIX_OK;
    if (!d_frames || !d_records || !d_ws) return fail(DP_PIX_E_INVALID_ARG, "frames, records and workspace are required");
    if (stream_id >= (1u << 24)) return fail(DP_PIX_E_INVALID_ARG, "stream_id must be < 2^24");
    if (n_frames > 65535) return fail(DP_PIX_E_INVALID_ARG, "at most 65535 frames per call");
    if (n_frames > 1 && frame_stride < g.pitch * (int64_t)(g.M - 1) + (int64_t)g.N * g.C)
        return fail(DP_PIX_E_INVALID_ARG, "frame_stride smaller than one frame");
    if (record_stride < (int64_t)g.record_cap || record_stride % 16 != 0)
        return fail(DP_PIX_E_BUFFER_TOO_SMALL, "record_stride %lld < record capacity %llu or not a multiple of 16",
                    (long long)record_stride, (unsigned long long)g.record_cap);
    if ((uintptr_t)d_records % 16 != 0) return fail(DP_PIX_E_INVALID_ARG, "records must be 16-byte aligned");
    if ((uintptr_t)d_ws % 256 != 0) return fail(DP_PIX_E_INVALID_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < (uint64_t)n_frames * g.ws_per_frame)
        return fail(DP_PIX_E_BUFFER_TOO_SMALL, "workspace %llu < %llu", (unsigned long long)ws_bytes,
                    (unsigned long long)((uint64_t)n_frames * g.ws_per_frame));
    if (g.source != DP_PIX_SRC_VARIANCE && !d_region_src) return fail(DP_PIX_E_INVALID_ARG, "region source is required");
    if (g.source == DP_PIX_SRC_MASK_U8 && src_pitch < g.N) return fail(DP_PIX_E_INVALID_ARG, "mask pitch < N");
    if (g.source == DP_PIX_SRC_MATTE_F32 && (src_pitch < 4ll * g.N || src_pitch % 4 != 0 || (uintptr_t)d_region_src % 4))
        return fail(DP_PIX_E_INVALID_ARG, "matte pitch < 4N or not 4-byte aligned");
    if (n_frames > 1 && g.source != DP_PIX_SRC_VARIANCE && src_frame_stride <= 0)
        return fail(DP_PIX_E_INVALID_ARG, "src_frame_stride required for several frames");
    int rc = check_cuda_device();
    if (rc) return rc;

    CallArgs a;
    memset(&a, 0, sizeof(a));
    a.frames = static_cast<const uint8_t *>(d_frames);
    a.frame_stride = frame_stride;
    a.src = static_cast<const uint8_t *>(d_region_src);
    a.src_pitch = src_pitch;
    a.src_frame_stride = src_frame_stride;
    a.n_frames = n_frames;
    a.stream_id = stream_id;
    a.frame_idx0 = frame_idx0;
    a.records = static_cast<uint8_t *>(d_records);
    a.record_stride = record_stride;
    a.ws = static_cast<uint8_t *>(d_ws);
    a.status = status_word();
    a.keys = keys;
    a.frames_bytes = (uint64_t)(n_frames - 1) * (uint64_t)(n_frames > 1 ? frame_stride : 0) +
                     (uint64_t)(g.M - 1) * (uint64_t)g.pitch + (uint64_t)g.N * g.C;
    a.records_bytes = (uint64_t)n_frames * (uint64_t)record_stride;
    if (g.test_shrink) a.records_bytes = a.records_bytes > g.test_shrink ? a.records_bytes - g.test_shrink : 0;
    a.ws_bytes = ws_bytes;
    const uintptr_t base = (uintptr_t)d_frames;
    const int64_t fs = n_frames > 1 ? frame_stride : 0;
    const int64_t seg_bytes = (int64_t)g.seg_tiles * g.T * g.C;
    if (base % 16 == 0 && g.pitch % 16 == 0 && fs % 16 == 0 && seg_bytes % 16 == 0)
        a.vec = 16;
    else if (base % 4 == 0 && g.pitch % 4 == 0 && fs % 4 == 0 && seg_bytes % 4 == 0)
        a.vec = 4;
    else
        a.vec = 1;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaSuccess;
    switch (g.source) {
        case DP_PIX_SRC_TILE_LABELS:
            e = launch_finalize_labels(g, a, s);
            if (e == cudaSuccess) e = launch_release(g, a, s);
            break;
        case DP_PIX_SRC_MASK_U8:
        case DP_PIX_SRC_MATTE_F32:
            e = launch_classify(g, a, s);
            if (e == cudaSuccess) e = launch_finalize_map(g, a, s);
            if (e == cudaSuccess) e = launch_release(g, a, s);
            break;
        case DP_PIX_SRC_VARIANCE:
            if (!fo || fo->stage != 2) {
                e = launch_tile_stats(g, a, s);
                if (e == cudaSuccess) e = launch_rank(g, a, s);
            }
            if (fo && fo->stage == 1) break;
            if (e == cudaSuccess && g.var_onepass && fo) {
                e = launch_emit_recon(g, a, fo->out, fo->frame_stride, fo->pitch, fo->type, fo->align, fo->max_per_sm,
                                      s);
                fo->fused = e == cudaSuccess;
                if (e == cudaErrorNotSupported) e = launch_emit(g, a, s);
            } else if (e == cudaSuccess) {
                e = g.var_onepass ? launch_emit(g, a, s) : launch_release(g, a, s);
            }
            break;
        default:
            return fail(DP_PIX_E_INVALID_ARG, "bad region source");
    }
    if (e != cudaSuccess) return cuda_fail(e, "release launch");
    return DP_PIX_OK;
}

}  // namespace

extern "C" {

int dp_pix_release(dp_pix_plan_t plan, const void *d_frames, int64_t frame_stride, const void *d_region_src,
                   int64_t src_pitch, int64_t src_frame_stride, uint32_t n_frames, uint32_t stream_id,
                   uint64_t frame_idx0, void *d_records, int64_t record_stride, void *d_ws, uint64_t ws_bytes,
                   void *cuda_stream) {
    DPPIX_RANGE();
    t_err[0] = 0;
    return release_impl(plan, d_frames, frame_stride, d_region_src, src_pitch, src_frame_stride, n_frames, stream_id,
                        frame_idx0, d_records, record_stride, d_ws, ws_bytes, cuda_stream, nullptr);
}

int dp_pix_release_keyed(dp_pix_plan_t plan, const void *d_frames, int64_t frame_stride, const void *d_region_src,
                         int64_t src_pitch, int64_t src_frame_stride, uint32_t n_frames, const dp_pix_frame_key *d_keys,
                         void *d_records, int64_t record_stride, void *d_ws, uint64_t ws_bytes, void *cuda_stream) {
    DPPIX_RANGE();
    t_err[0] = 0;
    if (n_frames > 0 && !d_keys) return fail(DP_PIX_E_INVALID_ARG, "keys are required");
    return release_impl(plan, d_frames, frame_stride, d_region_src, src_pitch, src_frame_stride, n_frames, 0, 0,
                        d_records, record_stride, d_ws, ws_bytes, cuda_stream, nullptr, d_keys);
}

}  // extern "C"

namespace {

// dp_pix_release_reconstruct, keyed by (stream_id, frame_idx0 + i) or, when keys is set, by keys[i].
int release_reconstruct_impl(dp_pix_plan_t plan, const void *d_frames, int64_t frame_stride,
                             const void *d_region_src, int64_t src_pitch, int64_t src_frame_stride,
                             uint32_t n_frames, uint32_t stream_id, uint64_t frame_idx0, const dp_pix_frame_key *keys,
                             void *d_records, int64_t record_stride, void *d_out, int64_t out_frame_stride,
                             int64_t out_pitch, int out_type, void *d_ws, uint64_t ws_bytes, void *cuda_stream) {
    if (!plan) return fail(DP_PIX_E_INVALID_ARG, "plan is NULL");
    if (n_frames == 0) return DP_PIX_OK;
    const Geom &g = plan->g;
    if (!d_out) return fail(DP_PIX_E_INVALID_ARG, "output is required");
    if (out_type != DP_PIX_OUT_U8 && out_type != DP_PIX_OUT_F32) return fail(DP_PIX_E_INVALID_ARG, "bad out_type");
    const int oes = out_type == DP_PIX_OUT_F32 ? 4 : 1;
    if (out_pitch < (int64_t)g.N * g.C * oes) return fail(DP_PIX_E_INVALID_ARG, "out_pitch < N * C * elem");
    if (n_frames > 1 && out_frame_stride < out_pitch * g.M) return fail(DP_PIX_E_INVALID_ARG, "out_frame_stride too small");
    if (out_type == DP_PIX_OUT_F32 &&
        ((uintptr_t)d_out % 4 || out_pitch % 4 || (n_frames > 1 && out_frame_stride % 4)))
        return fail(DP_PIX_E_INVALID_ARG, "f32 output must be 4-byte aligned");
    int align = 16;
    while (align > 1 &&
           ((uintptr_t)d_out % align || out_pitch % align || (n_frames > 1 && out_frame_stride % align)))
        align >>= 1;
    int stage = 0, max_per_sm = 0;
    auto run = [&](uint32_t f0, uint32_t nf, cudaStream_t st) -> int {
        const uint8_t *fr = static_cast<const uint8_t *>(d_frames) + (uint64_t)f0 * (uint64_t)frame_stride;
        const uint8_t *src = d_region_src ? static_cast<const uint8_t *>(d_region_src) + (uint64_t)f0 * src_frame_stride
                                          : nullptr;
        uint8_t *rec = static_cast<uint8_t *>(d_records) + (uint64_t)f0 * (uint64_t)record_stride;
        uint8_t *ws = static_cast<uint8_t *>(d_ws) + (uint64_t)f0 * g.ws_per_frame;
        uint8_t *out = static_cast<uint8_t *>(d_out) + (uint64_t)f0 * (uint64_t)out_frame_stride;
        const uint64_t wsb = ws_bytes >= (uint64_t)f0 * g.ws_per_frame ? ws_bytes - (uint64_t)f0 * g.ws_per_frame : 0;
        FusedOut fo{out, nf > 1 ? out_frame_stride : 0, out_pitch, out_type, align, false, stage, max_per_sm};
        int rc = release_impl(plan, fr, frame_stride, src, src_pitch, src_frame_stride, nf, stream_id, frame_idx0 + f0,
                              rec, record_stride, ws, wsb, st, &fo, keys ? keys + f0 : nullptr);
        if (rc || fo.fused || stage == 1) return rc;
        return dp_pix_reconstruct(rec, record_stride, nf, out, out_frame_stride, out_pitch, out_type, g.M, g.N, g.C, st);
    };
    cudaStream_t caller = static_cast<cudaStream_t>(cuda_stream);
    const int split = g.split;
    if (split <= 1 || n_frames < 2u * (uint32_t)split || g.source != DP_PIX_SRC_VARIANCE) return run(0, n_frames, caller);
    // a pipeline over `split` chunks of frames: the statistics and rank of every chunk run in order on the
    // caller's stream, and each chunk's emission (records and images) on a side stream as soon as its rank is
    // done, with the fused kernel held to fused_cap blocks per SM -- so that a chunk's issue-bound emission
    // shares the SMs with the next chunk's bandwidth-bound statistics pass
    cudaStream_t *side = side_streams(1);
    if (!side) return fail(DP_PIX_E_CUDA, "side stream unavailable");
    cudaEvent_t ev[kMaxSplit + 1] = {};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i <= split && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev[split], caller);  // the side stream starts after the caller's work
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side[0], ev[split], 0);
    int rc = e == cudaSuccess ? DP_PIX_OK : cuda_fail(e, "pipeline fork");
    for (int i = 0; i < split && rc == DP_PIX_OK; ++i) {
        const uint32_t f0 = (uint32_t)((uint64_t)n_frames * i / split), f1 = (uint32_t)((uint64_t)n_frames * (i + 1) / split);
        stage = 1;
        rc = run(f0, f1 - f0, caller);
        if (rc) break;
        e = cudaEventRecord(ev[i], caller);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side[0], ev[i], 0);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "pipeline event");
            break;
        }
        stage = 2;
        max_per_sm = g.fused_cap;
        rc = run(f0, f1 - f0, side[0]);
    }
    // join: the caller's stream waits for the last emission
    e = cudaEventRecord(ev[split], side[0]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, ev[split], 0);
    if (e != cudaSuccess && rc == DP_PIX_OK) rc = cuda_fail(e, "pipeline join");
    for (int i = 0; i <= split; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    return rc;
}

}  // namespace

extern "C" {

int dp_pix_release_reconstruct(dp_pix_plan_t plan, const void *d_frames, int64_t frame_stride,
                               const void *d_region_src, int64_t src_pitch, int64_t src_frame_stride,
                               uint32_t n_frames, uint32_t stream_id, uint64_t frame_idx0, void *d_records,
                               int64_t record_stride, void *d_out, int64_t out_frame_stride, int64_t out_pitch,
                               int out_type, void *d_ws, uint64_t ws_bytes, void *cuda_stream) {
    DPPIX_RANGE();
    t_err[0] = 0;
    return release_reconstruct_impl(plan, d_frames, frame_stride, d_region_src, src_pitch, src_frame_stride, n_frames,
                                    stream_id, frame_idx0, nullptr, d_records, record_stride, d_out, out_frame_stride,
                                    out_pitch, out_type, d_ws, ws_bytes, cuda_stream);
}

int dp_pix_keys_advance(dp_pix_frame_key *d_keys, uint32_t n, uint64_t delta, void *cuda_stream) {
    t_err[0] = 0;
    if (n == 0) return DP_PIX_OK;
    if (!d_keys) return fail(DP_PIX_E_INVALID_ARG, "keys are required");
    if ((uintptr_t)d_keys % 8) return fail(DP_PIX_E_INVALID_ARG, "keys must be 8-byte aligned");
    int rc = check_cuda_device();
    if (rc) return rc;
    const cudaError_t e = launch_keys_advance(d_keys, n, delta, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? DP_PIX_OK : cuda_fail(e, "keys advance");
}

int dp_pix_release_reconstruct_keyed(dp_pix_plan_t plan, const void *d_frames, int64_t frame_stride,
                                     const void *d_region_src, int64_t src_pitch, int64_t src_frame_stride,
                                     uint32_t n_frames, const dp_pix_frame_key *d_keys, void *d_records,
                                     int64_t record_stride, void *d_out, int64_t out_frame_stride, int64_t out_pitch,
                                     int out_type, void *d_ws, uint64_t ws_bytes, void *cuda_stream) {
    DPPIX_RANGE();
    t_err[0] = 0;
    if (n_frames > 0 && !d_keys) return fail(DP_PIX_E_INVALID_ARG, "keys are required");
    return release_reconstruct_impl(plan, d_frames, frame_stride, d_region_src, src_pitch, src_frame_stride, n_frames,
                                    0, 0, d_keys, d_records, record_stride, d_out, out_frame_stride, out_pitch,
                                    out_type, d_ws, ws_bytes, cuda_stream);
}

int dp_pix_store(const void *d_record, void *dst, uint64_t cap, uint64_t *written, int dst_is_host,
                 void *cuda_stream) {
    DPPIX_RANGE();
    t_err[0] = 0;
    if (!d_record || !dst) return fail(DP_PIX_E_INVALID_ARG, "record and destination are required");
    int rc = check_cuda_device();
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    dp_pix_record_header h;
    cudaError_t e = cudaMemcpyAsync(&h, d_record, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "store: header read");
    if (memcmp(h.magic, "DPPX", 4) != 0 || h.version != 1 || h.total_bytes < sizeof(h))
        return fail(DP_PIX_E_BAD_RECORD, "store: not a record");
    if (cap < h.total_bytes)
        return fail(DP_PIX_E_BUFFER_TOO_SMALL, "store: record needs %llu bytes", (unsigned long long)h.total_bytes);
    e = cudaMemcpyAsync(dst, d_record, h.total_bytes, dst_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "store: copy");
    if (written) *written = h.total_bytes;
    return DP_PIX_OK;
}

int dp_pix_store_batch(const void *d_records, int64_t record_stride, uint32_t n, void *h_dst, int64_t dst_stride,
                       uint64_t *written, void *cuda_stream) {
    DPPIX_RANGE();
    t_err[0] = 0;
    if (n == 0) return DP_PIX_OK;
    if (!d_records || !h_dst) return fail(DP_PIX_E_INVALID_ARG, "records and destination are required");
    if (record_stride < (int64_t)sizeof(dp_pix_record_header) || dst_stride < (int64_t)sizeof(dp_pix_record_header))
        return fail(DP_PIX_E_INVALID_ARG, "strides must be >= 512");
    int rc = check_cuda_device();
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    std::vector<dp_pix_record_header> hdr(n);
    cudaError_t e = cudaMemcpy2DAsync(hdr.data(), sizeof(dp_pix_record_header), d_records, (size_t)record_stride,
                                      sizeof(dp_pix_record_header), n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "store_batch: header read");
    for (uint32_t i = 0; i < n; ++i) {
        const dp_pix_record_header &h = hdr[i];
        if (memcmp(h.magic, "DPPX", 4) != 0 || h.version != 1 || h.total_bytes < sizeof(h) ||
            h.total_bytes > (uint64_t)record_stride)
            return fail(DP_PIX_E_BAD_RECORD, "store_batch: record %u is not a record", i);
        if (h.total_bytes > (uint64_t)dst_stride)
            return fail(DP_PIX_E_BUFFER_TOO_SMALL, "store_batch: record %u needs %llu bytes", i,
                        (unsigned long long)h.total_bytes);
    }
    for (uint32_t i = 0; i < n && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(static_cast<uint8_t *>(h_dst) + (uint64_t)i * dst_stride,
                            static_cast<const uint8_t *>(d_records) + (uint64_t)i * record_stride, hdr[i].total_bytes,
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "store_batch: copy");
    if (written)
        for (uint32_t i = 0; i < n; ++i) written[i] = hdr[i].total_bytes;
    return DP_PIX_OK;
}

int dp_pix_reconstruct(const void *d_records, int64_t record_stride, uint32_t n_records, void *d_out,
                       int64_t out_frame_stride, int64_t out_pitch, int out_type, int32_t max_M, int32_t max_N,
                       int32_t max_C, void *cuda_stream) {
    DPPIX_RANGE();
    t_err[0] = 0;
    if (n_records == 0) return DP_PIX_OK;
    if (!d_records || !d_out) return fail(DP_PIX_E_INVALID_ARG, "records and output are required");
    if (out_type != DP_PIX_OUT_U8 && out_type != DP_PIX_OUT_F32) return fail(DP_PIX_E_INVALID_ARG, "bad out_type");
    if (max_M < 1 || max_N < 1 || max_C < 1 || max_C > 4) return fail(DP_PIX_E_INVALID_ARG, "bad max geometry");
    const int oes = out_type == DP_PIX_OUT_F32 ? 4 : 1;
    if (out_pitch < (int64_t)max_N * max_C * oes) return fail(DP_PIX_E_INVALID_ARG, "out_pitch < max_N * max_C * elem");
    if (n_records > 1 && out_frame_stride < out_pitch * max_M) return fail(DP_PIX_E_INVALID_ARG, "out_frame_stride too small");
    if (record_stride < DP_PIX_RECORD_HEADER_BYTES || record_stride % 16 != 0)
        return fail(DP_PIX_E_INVALID_ARG, "record_stride must be >= 512 and a multiple of 16");
    if ((uintptr_t)d_records % 16 != 0) return fail(DP_PIX_E_INVALID_ARG, "records must be 16-byte aligned");
    if (out_type == DP_PIX_OUT_F32 && ((uintptr_t)d_out % 4 || out_pitch % 4 || (n_records > 1 && out_frame_stride % 4)))
        return fail(DP_PIX_E_INVALID_ARG, "f32 output must be 4-byte aligned");
    int rc = check_cuda_device();
    if (rc) return rc;
    int align = 16;
    const uint64_t ob = (uint64_t)(uintptr_t)d_out;
    while (align > 1 && (ob % align || out_pitch % align || (n_records > 1 && out_frame_stride % align))) align >>= 1;
    const cudaError_t e = launch_reconstruct(static_cast<const uint8_t *>(d_records), record_stride, n_records,
                                             static_cast<uint8_t *>(d_out), out_frame_stride, out_pitch, out_type,
                                             max_M, max_N, max_C, align, status_word(),
                                             static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "reconstruct launch");
    return DP_PIX_OK;
}

int dp_pix_debug_noise(uint64_t seed, const uint32_t *d_ctr, uint64_t n, uint32_t *d_words, float *d_eta, float sigma,
                       void *cuda_stream) {
    DPPIX_RANGE();
    t_err[0] = 0;
    if (n == 0) return DP_PIX_OK;
    if (!d_ctr) return fail(DP_PIX_E_INVALID_ARG, "counters are required");
    int rc = check_cuda_device();
    if (rc) return rc;
    const cudaError_t e = launch_debug_noise(seed, d_ctr, n, d_words, d_eta, sigma, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "debug_noise launch");
    return DP_PIX_OK;
}

int dp_pix_status(void *cuda_stream, uint32_t *detail) {
    DPPIX_RANGE();
    t_err[0] = 0;
    int rc = check_cuda_device();
    if (rc) return rc;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return cuda_fail(e, "status: stream sync");
    int32_t st[2] = {0, 0};
    e = cudaMemcpyFromSymbol(st, g_dppix_status, sizeof(st));
    if (e != cudaSuccess) return cuda_fail(e, "status: read");
    if (detail) *detail = (uint32_t)st[1];
    if (st[0] != 0) {
        const int32_t zero[2] = {0, 0};
        cudaMemcpyToSymbol(g_dppix_status, zero, sizeof(zero));
        return fail(st[0], "device-side check failed (detail 0x%x)", (unsigned)st[1]);
    }
    return DP_PIX_OK;
}

int dp_pix_prof_enable(int timing) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_timing = timing != 0;
    return DP_PIX_OK;
}

int dp_pix_prof_read(dp_pix_prof_entry *out, int cap) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int i = 0;
    for (auto &kv : g_prof) {
        ProfEntry &e = kv.second;
        for (auto &p : e.pending) {
            float ms = 0.f;
            if (cudaEventSynchronize(p.second) == cudaSuccess && cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess)
                e.total_ms += ms;
            cudaEventDestroy(p.first);
            cudaEventDestroy(p.second);
        }
        e.pending.clear();
        if (out && i < cap) {
            memset(&out[i], 0, sizeof(out[i]));
            strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
            out[i].launches = e.launches;
            out[i].total_ms = e.total_ms;
        }
        ++i;
    }
    return i;
}

int dp_pix_prof_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &kv : g_prof)
        for (auto &p : kv.second.pending) {
            cudaEventDestroy(p.first);
            cudaEventDestroy(p.second);
        }
    g_prof.clear();
    return DP_PIX_OK;
}

}  // extern "C"
