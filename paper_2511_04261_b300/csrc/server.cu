// server.cu -- the serving loop: frames of many cameras, continuously batched onto the GPU.
//
// Host side only (it drives the release kernels through dp_pix_release_keyed).  Requests are queued by
// any thread; one worker thread owns every CUDA call after creation.  Each resolution has a pool of device
// slots (frame, record, workspace, key) cut from the caller's arena, laid out as arrays so that a run of
// consecutive slots is one multi-frame keyed release.  Whenever one of the n_streams batch contexts is free,
// the worker admits every queued request that finds a free slot of its resolution (oldest first), copies
// the frames in, releases each resolution's runs, copies the records out, and enqueues a host callback that
// marks the batch finished -- so new arrivals keep joining the next batch while earlier ones are running.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

using namespace dppix;

namespace {

double now_us() {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

uint64_t a256(uint64_t x) { return (x + 255ull) & ~255ull; }

int sfail(int code, const char *fmt, ...) {
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return set_last_error(code, buf);
}

struct SrvClass {
    int32_t M = 0, N = 0;
    dp_pix_plan_t plan = nullptr;
    uint64_t frame_bytes = 0, frame_stride = 0, rec_stride = 0, ws_stride = 0;
    uint32_t slots = 0;
    uint8_t *d_frames = nullptr, *d_recs = nullptr, *d_ws = nullptr;
    dp_pix_frame_key *d_keys = nullptr;
    std::vector<uint8_t> busy;
};

struct SrvReq {
    uint32_t cam = 0;
    const void *hframe = nullptr;
    void *hrec = nullptr;
    uint64_t cap = 0, fidx = 0, rec_bytes = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int status = 0;
    bool done = false;
};

struct SrvBatch {
    struct dp_pix_server_s *srv = nullptr;
    cudaStream_t stream = nullptr;
    dp_pix_frame_key *h_keys = nullptr;  // pinned, one per slot of every class
    std::vector<uint64_t> tickets;
    std::vector<std::pair<int, uint32_t>> slots;  // (class, slot) per ticket
    bool busy = false, finished = false;
    int status = 0;
};

}  // namespace

struct dp_pix_server_s {
    int device = 0;
    int C = 3;
    std::vector<SrvClass> cls;
    std::vector<int> cam_class;
    std::vector<uint64_t> cam_count;
    std::vector<uint64_t> key_base;  // per class: offset of its slots in a batch's h_keys
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, SrvReq> reqs;
    std::vector<SrvBatch> batches;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    uint64_t in_flight = 0;
    dp_pix_server_stats st{};
    uint64_t batch_frames_total = 0;
};

namespace {

// Runs on the CUDA callback thread once the batch's record copies are done: no CUDA calls here.
void CUDART_CB batch_done(void *p) {
    SrvBatch *b = static_cast<SrvBatch *>(p);
    dp_pix_server_s *s = b->srv;
    // notify while holding the lock: once it is released this callback touches nothing of the server, which
    // may then be destroyed
    std::lock_guard<std::mutex> lk(s->mu);
    b->finished = true;
    s->cv.notify_all();
}

// Under s->mu: completes the requests of finished batches and frees their slots.
void retire(dp_pix_server_s *s) {
    bool any = false;
    const double t = now_us();
    for (SrvBatch &b : s->batches) {
        if (!b.busy || !b.finished) continue;
        for (size_t k = 0; k < b.tickets.size(); ++k) {
            SrvReq &r = s->reqs[b.tickets[k]];
            r.t_done = t;
            r.status = b.status;
            uint64_t total = 0;
            if (b.status == DP_PIX_OK) memcpy(&total, static_cast<const uint8_t *>(r.hrec) + 96, sizeof(total));
            r.rec_bytes = total;
            r.done = true;
            s->cls[b.slots[k].first].busy[b.slots[k].second] = 0;
        }
        s->in_flight -= b.tickets.size();
        s->st.completed += b.tickets.size();
        b.tickets.clear();
        b.slots.clear();
        b.busy = b.finished = false;
        any = true;
    }
    if (any) s->cv_done.notify_all();
}

// Under s->mu: fills batch b with every queued request that finds a free slot (oldest first).
void admit(dp_pix_server_s *s, SrvBatch &b) {
    const double t = now_us();
    for (auto it = s->pending.begin(); it != s->pending.end();) {
        SrvReq &r = s->reqs[*it];
        const int c = s->cam_class[r.cam];
        SrvClass &k = s->cls[c];
        uint32_t slot = k.slots;
        for (uint32_t i = 0; i < k.slots; ++i)
            if (!k.busy[i]) {
                slot = i;
                break;
            }
        if (slot == k.slots) {
            ++it;
            continue;
        }
        k.busy[slot] = 1;
        r.t_admit = t;
        b.tickets.push_back(*it);
        b.slots.emplace_back(c, slot);
        it = s->pending.erase(it);
    }
}

// Issues the copies, the keyed releases (one per run of consecutive slots of a resolution) and the callback.
// Called without s->mu; the batch's requests are not touched by other threads until it finishes.
int launch(dp_pix_server_s *s, SrvBatch &b, const std::vector<SrvReq> &rq) {
    cudaStream_t st = b.stream;
    const size_t n = b.tickets.size();
    std::vector<size_t> ord(n);
    for (size_t i = 0; i < n; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return b.slots[x] < b.slots[y]; });
    for (size_t i = 0; i < n; ++i) {
        const auto [c, slot] = b.slots[i];
        const SrvClass &k = s->cls[c];
        dp_pix_frame_key &key = b.h_keys[s->key_base[c] + slot];
        key.frame_idx = rq[i].fidx;
        key.stream_id = rq[i].cam;
        key.reserved = 0;
        const cudaError_t e = cudaMemcpyAsync(k.d_frames + slot * k.frame_stride, rq[i].hframe, k.frame_bytes,
                                              cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return sfail(DP_PIX_E_CUDA, "server frame copy: %s", cudaGetErrorString(e));
    }
    size_t i = 0;
    while (i < n) {
        const auto [c, slot0] = b.slots[ord[i]];
        size_t j = i + 1;
        while (j < n && b.slots[ord[j]].first == c && b.slots[ord[j]].second == slot0 + (j - i)) ++j;
        const uint32_t cnt = (uint32_t)(j - i);
        const SrvClass &k = s->cls[c];
        cudaError_t e = cudaMemcpyAsync(k.d_keys + slot0, b.h_keys + s->key_base[c] + slot0,
                                        cnt * sizeof(dp_pix_frame_key), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return sfail(DP_PIX_E_CUDA, "server key copy: %s", cudaGetErrorString(e));
        const int rc = dp_pix_release_keyed(k.plan, k.d_frames + slot0 * k.frame_stride, (int64_t)k.frame_stride,
                                            nullptr, 0, 0, cnt, k.d_keys + slot0, k.d_recs + slot0 * k.rec_stride,
                                            (int64_t)k.rec_stride, k.d_ws + slot0 * k.ws_stride,
                                            (uint64_t)cnt * k.ws_stride, st);
        if (rc) return rc;
        ++s->st.launches;
        i = j;
    }
    for (size_t q = 0; q < n; ++q) {
        const auto [c, slot] = b.slots[q];
        const SrvClass &k = s->cls[c];
        const cudaError_t e = cudaMemcpyAsync(rq[q].hrec, k.d_recs + slot * k.rec_stride, k.rec_stride,
                                              cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return sfail(DP_PIX_E_CUDA, "server record copy: %s", cudaGetErrorString(e));
    }
    return DP_PIX_OK;
}

void worker_main(dp_pix_server_s *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        retire(s);
        SrvBatch *fb = nullptr;
        bool busy = false;
        for (SrvBatch &b : s->batches) {
            if (b.busy) busy = true;
            else if (!fb) fb = &b;
        }
        if (s->stop && s->pending.empty() && !busy) break;
        if (fb && !s->pending.empty()) {
            admit(s, *fb);
            if (!fb->tickets.empty()) {
                fb->busy = true;
                fb->finished = false;
                fb->status = DP_PIX_OK;
                s->in_flight += fb->tickets.size();
                s->st.frames_in_flight_max = std::max(s->st.frames_in_flight_max, s->in_flight);
                ++s->st.batches;
                s->batch_frames_total += fb->tickets.size();
                std::vector<SrvReq> rq;
                rq.reserve(fb->tickets.size());
                for (uint64_t t : fb->tickets) rq.push_back(s->reqs[t]);
                lk.unlock();
                int rc = launch(s, *fb, rq);
                cudaError_t e = cudaLaunchHostFunc(fb->stream, batch_done, fb);
                lk.lock();
                if (rc == DP_PIX_OK && e != cudaSuccess) rc = DP_PIX_E_CUDA;
                fb->status = rc;
                if (e != cudaSuccess) fb->finished = true;  // nothing will call back: retire on the next pass
                continue;
            }
        }
        s->cv.wait(lk);
    }
}

}  // namespace

namespace {

int class_layout(const dp_pix_desc *common, int32_t M, int32_t N, SrvClass &k, Geom &g) {
    dp_pix_desc d = *common;
    d.M = M;
    d.N = N;
    d.row_pitch = (int64_t)N * common->C;
    const int rc = plan_geometry(&d, g);
    if (rc) return rc;
    k.M = M;
    k.N = N;
    k.frame_bytes = (uint64_t)M * N * common->C;
    k.frame_stride = a256(k.frame_bytes);
    k.rec_stride = a256(g.record_cap);
    k.ws_stride = a256(g.ws_per_frame);
    return DP_PIX_OK;
}

uint64_t slot_bytes(const SrvClass &k) { return k.frame_stride + k.rec_stride + k.ws_stride + sizeof(dp_pix_frame_key); }

void free_server(dp_pix_server_s *s) {
    for (SrvBatch &b : s->batches) {
        if (b.stream) cudaStreamDestroy(b.stream);
        if (b.h_keys) cudaFreeHost(b.h_keys);
    }
    for (SrvClass &k : s->cls)
        if (k.plan) dp_pix_plan_destroy(k.plan);
    delete s;
}

}  // namespace

extern "C" {

int dp_pix_server_sizes(const dp_pix_desc *common, int32_t M, int32_t N, uint64_t *slot_b, uint64_t *record_b) {
    if (!common) return sfail(DP_PIX_E_INVALID_ARG, "desc is NULL");
    SrvClass k;
    Geom g;
    const int rc = class_layout(common, M, N, k, g);
    if (rc) return rc;
    if (slot_b) *slot_b = slot_bytes(k) + 256;
    if (record_b) *record_b = k.rec_stride;
    return DP_PIX_OK;
}

int dp_pix_server_create(const dp_pix_desc *common, const int32_t *M, const int32_t *N, uint32_t n_cameras,
                         uint32_t n_streams, void *d_arena, uint64_t arena_bytes, dp_pix_server_t *out) {
    if (!common || !M || !N || !out) return sfail(DP_PIX_E_INVALID_ARG, "null argument");
    *out = nullptr;
    if (n_cameras < 1 || n_cameras > (1u << 24)) return sfail(DP_PIX_E_INVALID_ARG, "cameras must be 1..2^24");
    if (n_streams < 1 || n_streams > 8) return sfail(DP_PIX_E_INVALID_ARG, "n_streams must be 1..8");
    if (common->region_source != DP_PIX_SRC_VARIANCE)
        return sfail(DP_PIX_E_UNSUPPORTED, "the server releases VARIANCE-class frames (no per-frame side input)");
    if (!d_arena || (uintptr_t)d_arena % 256) return sfail(DP_PIX_E_INVALID_ARG, "arena must be 256-byte aligned");
    int rc = cuda_device_ok();
    if (rc) return rc;
    dp_pix_server_s *s = new dp_pix_server_s();
    cudaGetDevice(&s->device);
    s->C = common->C;
    s->cam_class.resize(n_cameras);
    s->cam_count.assign(n_cameras, 0);
    // resolution classes and their share of the arena (in proportion to their cameras' frame bytes)
    std::vector<double> weight;
    for (uint32_t c = 0; c < n_cameras; ++c) {
        int found = -1;
        for (size_t i = 0; i < s->cls.size(); ++i)
            if (s->cls[i].M == M[c] && s->cls[i].N == N[c]) found = (int)i;
        if (found < 0) {
            SrvClass k;
            Geom g;
            rc = class_layout(common, M[c], N[c], k, g);
            if (rc) {
                free_server(s);
                return rc;
            }
            dp_pix_desc d = *common;
            d.M = M[c];
            d.N = N[c];
            d.row_pitch = (int64_t)N[c] * common->C;
            rc = dp_pix_plan(&d, &k.plan, nullptr);
            if (rc) {
                free_server(s);
                return rc;
            }
            s->cls.push_back(k);
            weight.push_back(0.0);
            found = (int)s->cls.size() - 1;
        }
        s->cam_class[c] = found;
        weight[found] += (double)s->cls[found].frame_bytes;
    }
    double wsum = 0;
    for (double w : weight) wsum += w;
    uint8_t *p = static_cast<uint8_t *>(d_arena);
    uint64_t used = 0, key_total = 0;
    for (size_t i = 0; i < s->cls.size(); ++i) {
        SrvClass &k = s->cls[i];
        const uint64_t share = (uint64_t)((double)arena_bytes * weight[i] / wsum);
        const uint64_t per = slot_bytes(k);
        uint32_t n = (uint32_t)std::min<uint64_t>(share > 1024 ? (share - 1024) / per : 0, 1u << 16);
        if (n < 1) {
            free_server(s);
            return sfail(DP_PIX_E_BUFFER_TOO_SMALL, "arena leaves no slot for %dx%d frames (%llu bytes each)", k.M,
                         k.N, (unsigned long long)per);
        }
        k.slots = n;
        k.busy.assign(n, 0);
        k.d_frames = p + used;
        used = a256(used + (uint64_t)n * k.frame_stride);
        k.d_recs = p + used;
        used = a256(used + (uint64_t)n * k.rec_stride);
        k.d_ws = p + used;
        used = a256(used + (uint64_t)n * k.ws_stride);
        k.d_keys = reinterpret_cast<dp_pix_frame_key *>(p + used);
        used = a256(used + (uint64_t)n * sizeof(dp_pix_frame_key));
        s->key_base.push_back(key_total);
        key_total += n;
    }
    if (used > arena_bytes) {
        free_server(s);
        return sfail(DP_PIX_E_BUFFER_TOO_SMALL, "arena layout exceeds the arena");
    }
    s->batches.resize(n_streams);
    for (SrvBatch &b : s->batches) {
        b.srv = s;
        cudaError_t e = cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&b.h_keys), key_total * sizeof(dp_pix_frame_key),
                                                cudaHostAllocDefault);
        if (e != cudaSuccess) {
            free_server(s);
            return sfail(DP_PIX_E_CUDA, "server streams: %s", cudaGetErrorString(e));
        }
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return DP_PIX_OK;
}

int dp_pix_server_submit(dp_pix_server_t s, uint32_t camera, const void *host_frame, void *host_record,
                         uint64_t record_cap, uint64_t *ticket) {
    if (!s || !host_frame || !host_record || !ticket) return sfail(DP_PIX_E_INVALID_ARG, "null argument");
    if (camera >= s->cam_class.size()) return sfail(DP_PIX_E_INVALID_ARG, "no camera %u", camera);
    const SrvClass &k = s->cls[s->cam_class[camera]];
    if (record_cap < k.rec_stride)
        return sfail(DP_PIX_E_BUFFER_TOO_SMALL, "record_cap %llu < %llu", (unsigned long long)record_cap,
                     (unsigned long long)k.rec_stride);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return sfail(DP_PIX_E_INVALID_ARG, "server is stopping");
        const uint64_t t = s->next_ticket++;
        SrvReq &r = s->reqs[t];
        r.cam = camera;
        r.hframe = host_frame;
        r.hrec = host_record;
        r.cap = record_cap;
        r.fidx = s->cam_count[camera]++;
        r.t_submit = now_us();
        s->pending.push_back(t);
        ++s->st.submitted;
        *ticket = t;
    }
    s->cv.notify_all();
    return DP_PIX_OK;
}

int dp_pix_server_wait(dp_pix_server_t s, uint64_t ticket, int timeout_ms, dp_pix_server_result *res) {
    if (!s || !res) return sfail(DP_PIX_E_INVALID_ARG, "null argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return sfail(DP_PIX_E_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    auto ready = [&] { return s->reqs[ticket].done; };
    if (timeout_ms < 0) s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return DP_PIX_E_TIMEOUT;
    const SrvReq &r = s->reqs[ticket];
    res->ticket = ticket;
    res->frame_idx = r.fidx;
    res->record_bytes = r.rec_bytes;
    res->camera = r.cam;
    res->status = r.status;
    res->queue_us = r.t_admit - r.t_submit;
    res->latency_us = r.t_done - r.t_submit;
    s->reqs.erase(ticket);
    return DP_PIX_OK;
}

int dp_pix_server_stats_get(dp_pix_server_t s, dp_pix_server_stats *st) {
    if (!s || !st) return sfail(DP_PIX_E_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *st = s->st;
    st->mean_batch_frames = s->st.batches ? (double)s->batch_frames_total / (double)s->st.batches : 0.0;
    return DP_PIX_OK;
}

int dp_pix_server_slots(dp_pix_server_t s, uint32_t camera, uint32_t *slots) {
    if (!s || !slots || camera >= s->cam_class.size()) return sfail(DP_PIX_E_INVALID_ARG, "bad argument");
    *slots = s->cls[s->cam_class[camera]].slots;
    return DP_PIX_OK;
}

int dp_pix_server_destroy(dp_pix_server_t s) {
    if (!s) return DP_PIX_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (SrvBatch &b : s->batches)
        if (b.stream) cudaStreamSynchronize(b.stream);
    free_server(s);
    return DP_PIX_OK;
}

}  // extern "C"
