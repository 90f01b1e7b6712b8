// batch.cu -- ragged batches: many images of different sizes released (and rebuilt) together.
//
// The paper releases frames one at a time (Alg. 3 per frame); here a batch of images with their own sizes
// shares one plan of region parameters.  Every image gets the geometry a single-image plan would give it,
// kept in a device table at the front of the caller's workspace, and each phase (tile classification,
// map finalisation, release, reconstruction) runs as ONE persistent launch over the flattened work list of
// all images -- largest images first, so the long items start early and the tail is made of small ones.
// The launches of a bound batch are captured once into a CUDA graph and replayed.  The release's segment
// width (tiles staged per work item) is chosen by timing the candidates on the bound batch.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "common.cuh"

using namespace dppix;

struct dp_pix_batch_s {
    dp_pix_desc desc;                 // common region parameters (M, N, row_pitch unused)
    uint32_t n = 0;
    std::vector<int32_t> M, N;        // caller order
    std::vector<uint32_t> order;      // work order -> caller index (largest first)
    std::vector<Geom> geo;            // caller order, pitch = N * C until bound
    std::vector<uint64_t> ws_off;     // caller order: offset of the image's workspace in d_ws
    uint64_t table_bytes = 0, ws_bytes = 0;
    int seg_tiles = 0;                // release segment width in use (0: the plan's)
    int path = -1;                    // release path: DP_PIX_BATCH_PATH_* (-1: the default for the geometry)
    // bound state
    bool bound = false;
    std::vector<BatchEntry> tab;      // work order
    uint8_t *d_ws = nullptr;
    int out_type = DP_PIX_OUT_U8, out_align = 16, any_out = 0;
    uint32_t items_cls = 0, items_rel = 0, items_rec = 0, max_gc = 0, max_tiles = 0;
    size_t rel_smem = 0;
    // streaming kernels (k_batch_stream.cu), where the geometry allows them
    bool cls_stream = false, rel_stream = false, recon_fused = false;
    // whole warps per tile (k_batch_tiles): segments of tiles_S tiles sharing a CTA's 8 warps
    bool rel_tiles = false;
    int tiles_S = 0;

    BatchStreamShape rs{};
    // graph (captured on a private stream -- capture is not possible on the legacy default stream -- and
    // launched on the caller's)
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
};

namespace {

int bfail(int code, const char *fmt, ...) {
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return set_last_error(code, buf);
}

int cfail(cudaError_t e, const char *what) {
    return bfail(DP_PIX_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

uint64_t a256(uint64_t x) { return (x + 255ull) & ~255ull; }

void drop_graph(dp_pix_batch_s *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

// Release staging bytes for S tiles per segment (two buffers of T staged rows).
size_t seg_smem_for(const Geom &g, int S) { return release_smem(g.T, g.C, S); }

void apply_seg(Geom &g, int S) {
    g.seg_tiles = S;
    g.seg_per_row = (g.GC + S - 1) / S;
    g.seg_rowstride = (S * g.T * g.C + 15) / 16 * 16;
    set_release_units(g);
}

// Fills the work-order table (host) from the caller's images and the current segment width.
int build_table(dp_pix_batch_s *b, const dp_pix_batch_image *imgs, int out_type) {
    int32_t *st = status_word();
    b->tab.assign(b->n, BatchEntry{});
    uint32_t cls = 0, rel = 0, rec = 0;
    b->max_gc = 0;
    b->max_tiles = 0;
    b->rel_smem = 0;
    b->any_out = 0;
    int align = 16;
    const int oes = out_type == DP_PIX_OUT_F32 ? 4 : 1;
    {
        const Geom &g0 = b->geo[0];
        b->cls_stream = (g0.source == DP_PIX_SRC_MASK_U8 || g0.source == DP_PIX_SRC_MATTE_F32) &&
                        batch_classify_stream_ok(g0.T, g0.source == DP_PIX_SRC_MATTE_F32);
        b->rs = batch_release_stream_shape(g0.T, g0.C, g0.b_min, b->seg_tiles > 0 ? b->seg_tiles : 1 << 20);
        // default (path -1): whole warps per tile, 2 tiles per item (256-portrait batch: 2.22 ms against 2.30
        // ms for the staged unit list); the others when chosen (dp_pix_batch_set_path, or by the autotuner)
        b->rel_stream = b->rs.S > 0 && (b->path == DP_PIX_BATCH_PATH_STREAM || b->path == DP_PIX_BATCH_PATH_STREAM_FUSED);
        // the fused image needs u8 output and stored values it can read back as the reconstruction would
        b->recon_fused = b->rel_stream && b->path == DP_PIX_BATCH_PATH_STREAM_FUSED && b->rs.recon_ok &&
                         out_type == DP_PIX_OUT_U8 && g0.dtype != DP_PIX_REC_SUM_U32;
        const bool tiles = b->path == DP_PIX_BATCH_PATH_TILES || b->path < 0;
        b->tiles_S = b->seg_tiles > 0 ? b->seg_tiles : 2;
        b->rel_tiles = tiles && batch_tiles_smem(g0.T, g0.C, b->tiles_S) > 0;
    }
    for (uint32_t k = 0; k < b->n; ++k) {
        const uint32_t i = b->order[k];
        const dp_pix_batch_image &im = imgs[i];
        Geom g = b->geo[i];
        if (!im.frame || !im.record) return bfail(DP_PIX_E_INVALID_ARG, "image %u: frame and record are required", i);
        if (im.row_pitch < (int64_t)g.N * g.C) return bfail(DP_PIX_E_INVALID_ARG, "image %u: row_pitch < N*C", i);
        if ((uintptr_t)im.record % 16) return bfail(DP_PIX_E_INVALID_ARG, "image %u: record not 16-byte aligned", i);
        if (im.stream_id >= (1u << 24)) return bfail(DP_PIX_E_INVALID_ARG, "image %u: stream_id must be < 2^24", i);
        if (g.source != DP_PIX_SRC_VARIANCE && !im.region_src)
            return bfail(DP_PIX_E_INVALID_ARG, "image %u: region source is required", i);
        if (g.source == DP_PIX_SRC_MASK_U8 && im.src_pitch < g.N)
            return bfail(DP_PIX_E_INVALID_ARG, "image %u: mask pitch < N", i);
        if (g.source == DP_PIX_SRC_MATTE_F32 &&
            (im.src_pitch < 4ll * g.N || im.src_pitch % 4 || (uintptr_t)im.region_src % 4))
            return bfail(DP_PIX_E_INVALID_ARG, "image %u: matte pitch < 4N or not 4-byte aligned", i);
        if (im.out && im.out_pitch < (int64_t)g.N * g.C * oes)
            return bfail(DP_PIX_E_INVALID_ARG, "image %u: out_pitch < N*C*element", i);
        if (im.out && oes == 4 && ((uintptr_t)im.out % 4 || im.out_pitch % 4))
            return bfail(DP_PIX_E_INVALID_ARG, "image %u: f32 output must be 4-byte aligned", i);
        g.pitch = im.row_pitch;
        if (b->rel_tiles) apply_seg(g, b->tiles_S);
        else if (b->seg_tiles > 0 && !b->rel_stream) apply_seg(g, b->seg_tiles);
        BatchEntry &e = b->tab[k];
        e.g = g;
        CallArgs &a = e.a;
        memset(&a, 0, sizeof(a));
        a.frames = static_cast<const uint8_t *>(im.frame);
        a.src = static_cast<const uint8_t *>(im.region_src);
        a.src_pitch = im.src_pitch;
        a.n_frames = 1;
        a.stream_id = im.stream_id;
        a.frame_idx0 = im.frame_idx;
        a.records = static_cast<uint8_t *>(im.record);
        a.record_stride = (int64_t)((g.record_cap + 15) / 16 * 16);
        a.ws = b->d_ws + b->ws_off[i];
        a.status = st;
        a.frames_bytes = (uint64_t)(g.M - 1) * (uint64_t)g.pitch + (uint64_t)g.N * g.C;
        a.records_bytes = (g.record_cap + 15) / 16 * 16;
        a.ws_bytes = g.ws_per_frame;
        const uintptr_t base = (uintptr_t)im.frame;
        const int64_t seg_bytes = (int64_t)g.seg_tiles * g.T * g.C;
        a.vec = (base % 16 == 0 && g.pitch % 16 == 0 && seg_bytes % 16 == 0) ? 16
                : (base % 4 == 0 && g.pitch % 4 == 0 && seg_bytes % 4 == 0) ? 4 : 1;
        e.out = static_cast<uint8_t *>(im.out);
        e.out_pitch = im.out_pitch;
        e.rec_cap = g.record_cap;
        e.base[0] = cls;
        e.base[1] = k;
        e.base[2] = rel;
        e.base[3] = rec;
        if (b->cls_stream) {
            cls += (uint32_t)g.GR;
        } else {
            const int cs = cls_seg_tiles(g.T, g.source == DP_PIX_SRC_MATTE_F32 ? 4 : 1);
            cls += (uint32_t)g.GR * (uint32_t)((g.GC + cs - 1) / cs);
        }
        if (b->rel_stream)
            rel += (uint32_t)g.GR * (uint32_t)((g.GC + b->rs.S - 1) / b->rs.S);
        else
            rel += (uint32_t)g.GR * (uint32_t)g.seg_per_row;
        rec += (uint32_t)g.GR;
        b->max_gc = std::max<uint32_t>(b->max_gc, (uint32_t)g.GC);
        b->max_tiles = std::max<uint32_t>(b->max_tiles, g.ntiles);
        b->rel_smem = std::max(b->rel_smem, seg_smem_for(g, g.seg_tiles));
        if (im.out) {
            b->any_out = 1;
            while (align > 1 && ((uintptr_t)im.out % align || im.out_pitch % align)) align >>= 1;
        }
    }
    b->items_cls = cls;
    b->items_rel = rel;
    b->items_rec = rec;
    b->out_align = align;
    b->out_type = out_type;
    return DP_PIX_OK;
}

int upload(dp_pix_batch_s *b, cudaStream_t s) {
    const cudaError_t e = cudaMemcpyAsync(b->d_ws, b->tab.data(), sizeof(BatchEntry) * b->n, cudaMemcpyHostToDevice, s);
    return e == cudaSuccess ? DP_PIX_OK : cfail(e, "batch table upload");
}

cudaError_t launch_all(dp_pix_batch_s *b, cudaStream_t s) {
    const BatchEntry *tab = reinterpret_cast<const BatchEntry *>(b->d_ws);
    const Geom &g0 = b->tab[0].g;
    const int matte = g0.source == DP_PIX_SRC_MATTE_F32;
    cudaError_t e = cudaSuccess;
    if (g0.source == DP_PIX_SRC_MASK_U8 || g0.source == DP_PIX_SRC_MATTE_F32)
        e = b->cls_stream ? launch_batch_classify_stream(tab, b->n, b->items_cls, matte, b->max_gc, s)
                          : launch_batch_classify(tab, b->n, b->items_cls, g0.T, matte, s);
    if (e == cudaSuccess) e = launch_batch_finalize(tab, b->n, b->max_tiles, s);
    const bool fused = b->recon_fused && b->any_out;
    if (e == cudaSuccess) {
        if (b->rel_stream)
            e = launch_batch_release_stream(tab, b->n, b->items_rel, g0.C, b->rs, fused ? 1 : 0, s);
        else if (b->rel_tiles)
            e = launch_batch_tiles(tab, b->n, b->items_rel, g0.T, g0.C, b->tiles_S, s);
        else
            e = launch_batch_release(tab, b->n, b->items_rel, g0.T, g0.C, g0.seg_tiles, s);
    }
    if (e == cudaSuccess && b->any_out && !fused)
        e = launch_batch_reconstruct(tab, b->n, b->items_rec, b->out_type, g0.C, b->out_align, status_word(), s);
    return e;
}

}  // namespace

extern "C" {

int dp_pix_batch_plan(const dp_pix_desc *common, const int32_t *M, const int32_t *N, uint32_t n, dp_pix_batch_t *out) {
    DPPIX_RANGE();
    if (!common || !M || !N || !out) return bfail(DP_PIX_E_INVALID_ARG, "null argument");
    *out = nullptr;
    if (n < 1 || n > (1u << 20)) return bfail(DP_PIX_E_INVALID_ARG, "batch size must be 1..2^20");
    if (common->region_source == DP_PIX_SRC_VARIANCE)
        return bfail(DP_PIX_E_UNSUPPORTED, "variance classes rank a whole frame; release such frames with dp_pix_release");
    dp_pix_batch_s *b = new dp_pix_batch_s();
    b->desc = *common;
    b->n = n;
    b->M.assign(M, M + n);
    b->N.assign(N, N + n);
    b->geo.resize(n);
    b->ws_off.resize(n);
    for (uint32_t i = 0; i < n; ++i) {
        dp_pix_desc d = *common;
        d.M = M[i];
        d.N = N[i];
        d.row_pitch = (int64_t)N[i] * common->C;
        const int rc = plan_geometry(&d, b->geo[i]);
        if (rc) {
            delete b;
            return rc;
        }
    }
    b->order.resize(n);
    std::iota(b->order.begin(), b->order.end(), 0u);
    std::stable_sort(b->order.begin(), b->order.end(), [&](uint32_t x, uint32_t y) {
        return (int64_t)b->M[x] * b->N[x] > (int64_t)b->M[y] * b->N[y];
    });
    b->table_bytes = a256(sizeof(BatchEntry) * (uint64_t)n);
    uint64_t off = b->table_bytes;
    for (uint32_t i = 0; i < n; ++i) {
        b->ws_off[i] = off;
        off += a256(b->geo[i].ws_per_frame);
    }
    b->ws_bytes = off;
    *out = b;
    return DP_PIX_OK;
}

int dp_pix_batch_destroy(dp_pix_batch_t b) {
    if (!b) return DP_PIX_OK;
    drop_graph(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
    return DP_PIX_OK;
}

int dp_pix_batch_sizes(dp_pix_batch_t b, uint64_t *record_bytes, uint64_t *ws_bytes) {
    if (!b) return bfail(DP_PIX_E_INVALID_ARG, "batch is NULL");
    if (record_bytes)
        for (uint32_t i = 0; i < b->n; ++i) record_bytes[i] = (b->geo[i].record_cap + 15) / 16 * 16;
    if (ws_bytes) *ws_bytes = b->ws_bytes;
    return DP_PIX_OK;
}

int dp_pix_batch_bind(dp_pix_batch_t b, const dp_pix_batch_image *imgs, int out_type, void *d_ws, uint64_t ws_bytes,
                      void *cuda_stream) {
    DPPIX_RANGE();
    if (!b || !imgs) return bfail(DP_PIX_E_INVALID_ARG, "batch or images NULL");
    if (out_type != DP_PIX_OUT_U8 && out_type != DP_PIX_OUT_F32) return bfail(DP_PIX_E_INVALID_ARG, "bad out_type");
    if (!d_ws || (uintptr_t)d_ws % 256) return bfail(DP_PIX_E_INVALID_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < b->ws_bytes)
        return bfail(DP_PIX_E_BUFFER_TOO_SMALL, "workspace %llu < %llu", (unsigned long long)ws_bytes,
                     (unsigned long long)b->ws_bytes);
    int rc = cuda_device_ok();
    if (rc) return rc;
    b->d_ws = static_cast<uint8_t *>(d_ws);
    b->bound = false;
    drop_graph(b);
    rc = build_table(b, imgs, out_type);
    if (rc) return rc;
    rc = upload(b, static_cast<cudaStream_t>(cuda_stream));
    if (rc) return rc;
    b->bound = true;
    return DP_PIX_OK;
}

int dp_pix_batch_run(dp_pix_batch_t b, int use_graph, void *cuda_stream) {
    DPPIX_RANGE();
    if (!b || !b->bound) return bfail(DP_PIX_E_INVALID_ARG, "batch not bound");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (!use_graph) {
        const cudaError_t e = launch_all(b, s);
        return e == cudaSuccess ? DP_PIX_OK : cfail(e, "batch launch");
    }
    if (!b->exec) {
        if (!b->cap_stream) {
            const cudaError_t ce = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
            if (ce != cudaSuccess) {
                b->cap_stream = nullptr;
                return cfail(ce, "batch capture stream");
            }
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cfail(e, "batch graph capture");
        const cudaError_t le = launch_all(b, b->cap_stream);
        e = cudaStreamEndCapture(b->cap_stream, &graph);
        if (le != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cfail(le, "batch launch (capture)");
        }
        if (e != cudaSuccess) return cfail(e, "batch graph capture end");
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return cfail(e, "batch graph instantiate");
        }
    }
    prof_begin("batch_graph", s);
    const cudaError_t e = cudaGraphLaunch(b->exec, s);
    prof_end("batch_graph", s);
    return e == cudaSuccess ? DP_PIX_OK : cfail(e, "batch graph launch");
}

int dp_pix_batch_autotune(dp_pix_batch_t b, const dp_pix_batch_image *imgs, int reps, void *cuda_stream) {
    DPPIX_RANGE();
    if (!b || !b->bound || !imgs) return bfail(DP_PIX_E_INVALID_ARG, "batch not bound or images NULL");
    if (reps < 1) reps = 1;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const Geom &g0 = b->geo[0];
    // candidates: the staged release (segments of up to 16 tiles, within its shared memory) and the streaming
    // one (segments up to what its shared memory holds), the latter with the images written by a separate
    // reconstruction or from the same kernel
    std::vector<std::pair<int, int>> cands;  // (path, segment tiles)
    for (int S : {1, 2, 3, 4, 6, 8})
        if (seg_smem_for(g0, S) <= 200 * 1024) cands.emplace_back(DP_PIX_BATCH_PATH_STAGED, S);
    const BatchStreamShape full = batch_release_stream_shape(g0.T, g0.C, g0.b_min, 1 << 20);
    if (full.S > 0) {
        const bool fusable = full.recon_ok && b->any_out && b->out_type == DP_PIX_OUT_U8 && g0.dtype != DP_PIX_REC_SUM_U32;
        int last = 0;
        for (int S : {4, 6, 9, 12, 16, 24, 32}) {
            const int Ss = std::min(S, full.S);
            if (Ss == last) continue;
            last = Ss;
            cands.emplace_back(DP_PIX_BATCH_PATH_STREAM, Ss);
            if (fusable) cands.emplace_back(DP_PIX_BATCH_PATH_STREAM_FUSED, Ss);
        }
    }
    for (int S : {1, 2, 4, 8})
        if (batch_tiles_smem(g0.T, g0.C, S) > 0) cands.emplace_back(DP_PIX_BATCH_PATH_TILES, S);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return cfail(cudaGetLastError(), "events");
    float best = 1e30f;
    int best_s = b->seg_tiles, best_p = b->path;
    int rc = DP_PIX_OK;
    for (const auto &c : cands) {
        b->path = c.first;
        b->seg_tiles = c.second;
        rc = build_table(b, imgs, b->out_type);
        if (!rc) rc = upload(b, s);
        if (rc) break;
        cudaError_t e = launch_all(b, s);  // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_all(b, s);
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = cfail(e, "autotune launch");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_s = c.second;
            best_p = c.first;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->seg_tiles = best_s;
    b->path = best_p;
    drop_graph(b);
    const int rc2 = build_table(b, imgs, b->out_type);
    if (rc2) return rc2;
    const int rc3 = upload(b, s);
    return rc ? rc : rc3;
}

int dp_pix_batch_tuning(dp_pix_batch_t b, int *seg_tiles, int *path) {
    if (!b || !seg_tiles) return bfail(DP_PIX_E_INVALID_ARG, "null argument");
    *seg_tiles = b->rel_stream ? b->rs.S
                 : b->rel_tiles ? b->tiles_S
                                : (b->seg_tiles > 0 ? b->seg_tiles : b->geo[0].seg_tiles);
    if (path)
        *path = b->rel_tiles    ? DP_PIX_BATCH_PATH_TILES
                : !b->rel_stream ? DP_PIX_BATCH_PATH_STAGED
                                 : (b->recon_fused ? DP_PIX_BATCH_PATH_STREAM_FUSED : DP_PIX_BATCH_PATH_STREAM);
    return DP_PIX_OK;
}

int dp_pix_batch_set_path(dp_pix_batch_t b, int path, int seg_tiles) {
    if (!b) return bfail(DP_PIX_E_INVALID_ARG, "batch is NULL");
    if (path < -1 || path > DP_PIX_BATCH_PATH_TILES) return bfail(DP_PIX_E_INVALID_ARG, "bad path %d", path);
    if (seg_tiles < 0 || seg_tiles > 64) return bfail(DP_PIX_E_INVALID_ARG, "segment tiles must be 0..64");
    b->path = path;
    b->seg_tiles = seg_tiles;
    b->bound = false;  // takes effect at the next dp_pix_batch_bind
    drop_graph(b);
    return DP_PIX_OK;
}

}  // extern "C"
