// server.cu -- the serving loop: frames of many cameras, continuously batched onto the GPU.
//
// Requests are queued by any thread; one worker thread owned by the server issues every CUDA call after
// creation.  Whenever one of the n_streams batch contexts is free, the worker admits the queued requests,
// oldest first, that the arena has room for, copies their frames in, releases each resolution's frames in
// one keyed launch (optionally with the reconstruction), copies the results out, and enqueues a host
// callback that marks the batch finished -- so new arrivals keep joining the next batch while earlier ones
// are running.
//
// Memory: one caller-owned arena.  Its head holds each camera's next frame index (device memory) and each
// batch context's key table; the rest is handed out per batch by a first-fit allocator: every resolution
// present in a batch gets one block for its frames, records, workspaces (and reconstructions), freed when
// the batch retires.  A request is therefore admitted whenever the free memory holds it, whatever its
// resolution: a burst of large frames can use memory that small frames are not using.
//
// Noise keys: frame f of camera c is released with stream_id c and frame_idx f, where f counts that
// camera's frames from the first index given at creation.  The counters live on the device; for every
// batch a one-block kernel on the server's key stream (one stream, so batches take their indices in the
// order they were formed) turns the batch's (camera, rank among the camera's frames in this batch) table
// into keys and advances the counters.  dp_pix_server_counters reads them back, so a restarted server can
// continue every camera's count instead of drawing the same noise again (parallel composition, Thm 1,
// holds for independent draws only).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "common.cuh"

using namespace dppix;

namespace {

constexpr uint32_t kMaxBatch = 256;  // frames per batch

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

// Keys of one batch: on entry key i holds (rank of the frame among its camera's frames in this batch,
// camera, 1 if it is the camera's last frame in this batch); on exit (counter + rank, camera, 0), and the
// camera's counter has moved past the batch's frames.  One block: each thread handles the same keys in
// both phases, and the barrier separates the counter reads from the writes.
__global__ void k_server_keys(uint64_t *__restrict__ counters, dp_pix_frame_key *__restrict__ keys, uint32_t n,
                              uint32_t n_cameras, int32_t *status) {
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint32_t cam = keys[i].stream_id;
        if (cam < n_cameras) {
            keys[i].frame_idx += counters[cam];
        } else {
            keys[i].stream_id = 1u << 24;  // the release flags this key and leaves its record undefined
            if (status) atomicCAS(status, 0, DP_PIX_E_DEVICE);
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        if (keys[i].reserved) {
            const uint32_t cam = keys[i].stream_id;
            if (cam < n_cameras) counters[cam] = keys[i].frame_idx + 1;
            keys[i].reserved = 0;
        }
    }
}

// First-fit allocator over [0, size) in 256-byte units; free blocks are kept coalesced.
struct Heap {
    std::map<uint64_t, uint64_t> free;  // offset -> bytes
    uint64_t used = 0, used_max = 0;

    void init(uint64_t size) {
        free.clear();
        if (size) free[0] = size;
    }
    uint64_t largest() const {
        uint64_t m = 0;
        for (const auto &kv : free) m = std::max(m, kv.second);
        return m;
    }
    bool alloc(uint64_t bytes, uint64_t *off) {
        bytes = a256(bytes);
        for (auto it = free.begin(); it != free.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const uint64_t rest = it->second - bytes, at = it->first + bytes;
            free.erase(it);
            if (rest) free[at] = rest;
            used += bytes;
            used_max = std::max(used_max, used);
            return true;
        }
        return false;
    }
    void release(uint64_t off, uint64_t bytes) {
        bytes = a256(bytes);
        used -= bytes;
        auto next = free.lower_bound(off);
        if (next != free.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free.erase(next);
        }
        if (next != free.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free[off] = bytes;
    }
};

struct SrvClass {
    int32_t M = 0, N = 0;
    dp_pix_plan_t plan = nullptr;
    uint64_t frame_bytes = 0, frame_stride = 0, rec_stride = 0, ws_stride = 0;
    uint64_t per_frame(bool recon) const { return frame_stride + rec_stride + ws_stride + (recon ? frame_stride : 0); }
};

struct SrvReq {
    uint32_t cam = 0;
    const void *hframe = nullptr;
    void *hrec = nullptr;
    void *hout = nullptr;
    uint64_t cap = 0, fidx = 0, rec_bytes = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int status = 0;
    bool done = false;
};

// The frames of one resolution in one batch: one arena block, one keyed launch.
struct SrvRun {
    int cls = 0;
    uint32_t n = 0, key0 = 0;
    bool recon = false;
    uint64_t off = 0, bytes = 0;
};

struct SrvBatch {
    struct dp_pix_server_s *srv = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t keys_ready = nullptr;
    dp_pix_frame_key *h_keys = nullptr;  // pinned, kMaxBatch
    dp_pix_frame_key *d_keys = nullptr;  // in the arena head, kMaxBatch
    std::vector<uint64_t> tickets;       // grouped by run, in admission order within a run
    std::vector<SrvRun> runs;
    bool busy = false, finished = false;
    int status = 0;
};

}  // namespace

struct dp_pix_server_s {
    int device = 0;
    int C = 3;
    uint32_t n_cameras = 0;
    std::vector<SrvClass> cls;
    std::vector<int> cam_class;
    uint8_t *arena = nullptr;
    uint64_t heap_base = 0;
    uint64_t *d_counters = nullptr;
    uint64_t *h_counters = nullptr;  // pinned staging for dp_pix_server_counters
    cudaStream_t key_stream = nullptr;
    Heap heap;
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

// Runs on the CUDA callback thread once the batch's copies are done: no CUDA calls here.
void CUDART_CB batch_done(void *p) {
    SrvBatch *b = static_cast<SrvBatch *>(p);
    dp_pix_server_s *s = b->srv;
    // notify while holding the lock: once it is released this callback touches nothing of the server, which
    // may then be destroyed
    std::lock_guard<std::mutex> lk(s->mu);
    b->finished = true;
    s->cv.notify_all();
}

// Under s->mu: completes the requests of finished batches and returns their memory.
void retire(dp_pix_server_s *s) {
    bool any = false;
    const double t = now_us();
    for (SrvBatch &b : s->batches) {
        if (!b.busy || !b.finished) continue;
        for (uint64_t tk : b.tickets) {
            SrvReq &r = s->reqs[tk];
            r.t_done = t;
            r.status = b.status;
            uint64_t total = 0, fidx = 0;
            if (b.status == DP_PIX_OK) {
                const uint8_t *h = static_cast<const uint8_t *>(r.hrec);
                memcpy(&fidx, h + 72, sizeof(fidx));
                memcpy(&total, h + 96, sizeof(total));
            }
            r.fidx = fidx;
            r.rec_bytes = total;
            r.done = true;
        }
        for (const SrvRun &run : b.runs) s->heap.release(run.off, run.bytes);
        s->in_flight -= b.tickets.size();
        s->st.completed += b.tickets.size();
        b.tickets.clear();
        b.runs.clear();
        b.busy = b.finished = false;
        any = true;
    }
    if (any) s->cv_done.notify_all();
}

// Under s->mu: fills batch b with the queued requests, oldest first, that fit in the free memory: for
// each resolution (in the order of its oldest request) as many of its queued frames as one free block
// holds.  A camera's frames stay in arrival order: a resolution's candidates are taken as a prefix.  When
// the oldest request finds no room, nothing is admitted until memory comes back, so a large frame is not
// starved by a stream of small ones.
void admit(dp_pix_server_s *s, SrvBatch &b) {
    const double t = now_us();
    std::vector<std::vector<uint64_t>> cand(s->cls.size());
    std::vector<int> order;
    size_t total = 0;
    for (uint64_t tk : s->pending) {
        if (total == kMaxBatch) break;
        const int c = s->cam_class[s->reqs[tk].cam];
        if (cand[c].empty()) order.push_back(c);
        cand[c].push_back(tk);
        ++total;
    }
    std::unordered_set<uint64_t> taken;
    uint32_t key = 0;
    for (int c : order) {
        const SrvClass &k = s->cls[c];
        const std::vector<uint64_t> &v = cand[c];
        bool recon = false;
        for (uint64_t tk : v) recon = recon || s->reqs[tk].hout != nullptr;
        uint32_t n = (uint32_t)std::min<uint64_t>(v.size(), s->heap.largest() / k.per_frame(recon));
        if (n == 0 && c == order[0]) break;
        if (n == 0) continue;
        recon = false;
        for (uint32_t i = 0; i < n; ++i) recon = recon || s->reqs[v[i]].hout != nullptr;
        SrvRun run;
        run.cls = c;
        run.n = n;
        run.key0 = key;
        run.recon = recon;
        run.bytes = (uint64_t)n * k.per_frame(recon);
        if (!s->heap.alloc(run.bytes, &run.off)) continue;  // cannot happen: the largest block holds it
        b.runs.push_back(run);
        for (uint32_t i = 0; i < n; ++i) {
            s->reqs[v[i]].t_admit = t;
            b.tickets.push_back(v[i]);
            taken.insert(v[i]);
        }
        key += n;
    }
    if (taken.empty()) return;
    std::deque<uint64_t> rest;
    for (uint64_t tk : s->pending)
        if (!taken.count(tk)) rest.push_back(tk);
    s->pending.swap(rest);
}

// Issues the copies, the key kernel, the keyed releases and the callback for batch b.  Called without
// s->mu; the batch's requests are not touched by other threads until it finishes.
int launch(dp_pix_server_s *s, SrvBatch &b, const std::vector<SrvReq> &rq) {
    ApiRange range("dp_pix_server batch");
    cudaStream_t st = b.stream;
    const uint32_t n = (uint32_t)b.tickets.size();
    // key table: rank among the camera's frames in this batch, and a flag on the camera's last one
    std::unordered_map<uint32_t, uint32_t> seen, last;
    for (uint32_t i = 0; i < n; ++i) {
        dp_pix_frame_key &kk = b.h_keys[i];
        kk.frame_idx = seen[rq[i].cam]++;
        kk.stream_id = rq[i].cam;
        kk.reserved = 0;
        last[rq[i].cam] = i;
    }
    for (const auto &kv : last) b.h_keys[kv.second].reserved = 1;
    cudaError_t e = cudaMemcpyAsync(b.d_keys, b.h_keys, n * sizeof(dp_pix_frame_key), cudaMemcpyHostToDevice,
                                    s->key_stream);
    if (e != cudaSuccess) return sfail(DP_PIX_E_CUDA, "server key copy: %s", cudaGetErrorString(e));
    k_server_keys<<<1, 256, 0, s->key_stream>>>(s->d_counters, b.d_keys, n, s->n_cameras, status_word());
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(b.keys_ready, s->key_stream);
    if (e != cudaSuccess) return sfail(DP_PIX_E_CUDA, "server key kernel: %s", cudaGetErrorString(e));
    // frames in while the keys are made
    uint32_t i = 0;
    for (const SrvRun &run : b.runs) {
        const SrvClass &k = s->cls[run.cls];
        uint8_t *frames = s->arena + s->heap_base + run.off;
        for (uint32_t j = 0; j < run.n; ++j, ++i) {
            e = cudaMemcpyAsync(frames + j * k.frame_stride, rq[i].hframe, k.frame_bytes, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return sfail(DP_PIX_E_CUDA, "server frame copy: %s", cudaGetErrorString(e));
        }
    }
    e = cudaStreamWaitEvent(st, b.keys_ready, 0);
    if (e != cudaSuccess) return sfail(DP_PIX_E_CUDA, "server key wait: %s", cudaGetErrorString(e));
    i = 0;
    for (const SrvRun &run : b.runs) {
        const SrvClass &k = s->cls[run.cls];
        uint8_t *frames = s->arena + s->heap_base + run.off;
        uint8_t *recs = frames + (uint64_t)run.n * k.frame_stride;
        uint8_t *ws = recs + (uint64_t)run.n * k.rec_stride;
        uint8_t *out = ws + (uint64_t)run.n * k.ws_stride;
        const uint64_t wsb = (uint64_t)run.n * k.ws_stride;
        const int64_t pitch = (int64_t)k.N * s->C;
        const int rc = run.recon
                           ? dp_pix_release_reconstruct_keyed(k.plan, frames, (int64_t)k.frame_stride, nullptr, 0, 0,
                                                              run.n, b.d_keys + run.key0, recs, (int64_t)k.rec_stride,
                                                              out, (int64_t)k.frame_stride, pitch, DP_PIX_OUT_U8, ws,
                                                              wsb, st)
                           : dp_pix_release_keyed(k.plan, frames, (int64_t)k.frame_stride, nullptr, 0, 0, run.n,
                                                  b.d_keys + run.key0, recs, (int64_t)k.rec_stride, ws, wsb, st);
        if (rc) return rc;
        ++s->st.launches;
        for (uint32_t j = 0; j < run.n; ++j, ++i) {
            e = cudaMemcpyAsync(rq[i].hrec, recs + j * k.rec_stride, k.rec_stride, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && rq[i].hout)
                e = cudaMemcpyAsync(rq[i].hout, out + j * k.frame_stride, k.frame_bytes, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) return sfail(DP_PIX_E_CUDA, "server result copy: %s", cudaGetErrorString(e));
        }
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
                s->st.arena_bytes_in_use_max = std::max(s->st.arena_bytes_in_use_max, s->heap.used_max);
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

void free_server(dp_pix_server_s *s) {
    for (SrvBatch &b : s->batches) {
        if (b.stream) cudaStreamDestroy(b.stream);
        if (b.keys_ready) cudaEventDestroy(b.keys_ready);
        if (b.h_keys) cudaFreeHost(b.h_keys);
    }
    if (s->key_stream) cudaStreamDestroy(s->key_stream);
    if (s->h_counters) cudaFreeHost(s->h_counters);
    for (SrvClass &k : s->cls)
        if (k.plan) dp_pix_plan_destroy(k.plan);
    delete s;
}

// Makes `dev` current on this thread for the life of the object and restores the previous device.
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceScope() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

int dp_pix_server_sizes(const dp_pix_desc *common, int32_t M, int32_t N, uint64_t *slot_b, uint64_t *record_b,
                        uint64_t *recon_b) {
    clear_last_error();
    if (!common) return sfail(DP_PIX_E_INVALID_ARG, "desc is NULL");
    SrvClass k;
    Geom g;
    const int rc = class_layout(common, M, N, k, g);
    if (rc) return rc;
    if (slot_b) *slot_b = k.per_frame(false);
    if (record_b) *record_b = k.rec_stride;
    if (recon_b) *recon_b = k.frame_stride;
    return DP_PIX_OK;
}

int dp_pix_server_create(const dp_pix_desc *common, const int32_t *M, const int32_t *N, uint32_t n_cameras,
                         const uint64_t *first_frame, uint32_t n_streams, void *d_arena, uint64_t arena_bytes,
                         dp_pix_server_t *out) {
    DPPIX_RANGE();
    clear_last_error();
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
    s->n_cameras = n_cameras;
    s->cam_class.resize(n_cameras);
    uint64_t need_one = 0;  // the largest single frame (with its reconstruction) must fit the empty heap
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
            need_one = std::max(need_one, k.per_frame(true));
            s->cls.push_back(k);
            found = (int)s->cls.size() - 1;
        }
        s->cam_class[c] = found;
    }
    // arena head: counters, then one key table per batch context; the heap is the rest
    s->arena = static_cast<uint8_t *>(d_arena);
    s->d_counters = reinterpret_cast<uint64_t *>(s->arena);
    uint64_t head = a256((uint64_t)n_cameras * sizeof(uint64_t));
    s->batches.resize(n_streams);
    for (SrvBatch &b : s->batches) {
        b.srv = s;
        b.d_keys = reinterpret_cast<dp_pix_frame_key *>(s->arena + head);
        head = a256(head + kMaxBatch * sizeof(dp_pix_frame_key));
    }
    if (arena_bytes < head || arena_bytes - head < need_one) {
        free_server(s);
        return sfail(DP_PIX_E_BUFFER_TOO_SMALL, "arena of %llu bytes holds no frame of the largest resolution (%llu "
                     "bytes with its reconstruction, after %llu bytes of counters and key tables)",
                     (unsigned long long)arena_bytes, (unsigned long long)need_one, (unsigned long long)head);
    }
    s->heap_base = head;
    s->heap.init((arena_bytes - head) & ~255ull);
    cudaError_t e = cudaStreamCreateWithFlags(&s->key_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaHostAlloc(reinterpret_cast<void **>(&s->h_counters), (uint64_t)n_cameras * sizeof(uint64_t),
                          cudaHostAllocDefault);
    for (SrvBatch &b : s->batches) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.keys_ready, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaHostAlloc(reinterpret_cast<void **>(&b.h_keys), kMaxBatch * sizeof(dp_pix_frame_key),
                              cudaHostAllocDefault);
    }
    if (e == cudaSuccess) {
        for (uint32_t c = 0; c < n_cameras; ++c) s->h_counters[c] = first_frame ? first_frame[c] : 0;
        e = cudaMemcpyAsync(s->d_counters, s->h_counters, (uint64_t)n_cameras * sizeof(uint64_t),
                            cudaMemcpyHostToDevice, s->key_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->key_stream);
    }
    if (e != cudaSuccess) {
        free_server(s);
        return sfail(DP_PIX_E_CUDA, "server set-up: %s", cudaGetErrorString(e));
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return DP_PIX_OK;
}

int dp_pix_server_submit(dp_pix_server_t s, uint32_t camera, const void *host_frame, void *host_record,
                         uint64_t record_cap, void *host_out, uint64_t *ticket) {
    clear_last_error();
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
        r.hout = host_out;
        r.cap = record_cap;
        r.t_submit = now_us();
        s->pending.push_back(t);
        ++s->st.submitted;
        *ticket = t;
    }
    s->cv.notify_all();
    return DP_PIX_OK;
}

int dp_pix_server_wait(dp_pix_server_t s, uint64_t ticket, int timeout_ms, dp_pix_server_result *res) {
    clear_last_error();
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

int dp_pix_server_counters(dp_pix_server_t s, uint64_t *next_frame, uint32_t n) {
    DPPIX_RANGE();
    clear_last_error();
    if (!s || !next_frame) return sfail(DP_PIX_E_INVALID_ARG, "null argument");
    if (n > s->n_cameras) return sfail(DP_PIX_E_INVALID_ARG, "n %u > cameras %u", n, s->n_cameras);
    std::unique_lock<std::mutex> lk(s->mu);
    // every submitted frame has its key once nothing is queued or in flight; holding the lock from here
    // keeps the worker from forming another batch until the counters are read
    s->cv_done.wait(lk, [&] { return s->pending.empty() && s->in_flight == 0; });
    DeviceScope dev(s->device);
    cudaError_t e = cudaMemcpyAsync(s->h_counters, s->d_counters, (uint64_t)n * sizeof(uint64_t),
                                    cudaMemcpyDeviceToHost, s->key_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->key_stream);
    if (e != cudaSuccess) return sfail(DP_PIX_E_CUDA, "server counters: %s", cudaGetErrorString(e));
    memcpy(next_frame, s->h_counters, (uint64_t)n * sizeof(uint64_t));
    return DP_PIX_OK;
}

int dp_pix_server_stats_get(dp_pix_server_t s, dp_pix_server_stats *st) {
    clear_last_error();
    if (!s || !st) return sfail(DP_PIX_E_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *st = s->st;
    st->mean_batch_frames = s->st.batches ? (double)s->batch_frames_total / (double)s->st.batches : 0.0;
    st->arena_heap_bytes = s->heap.used + [&] {
        uint64_t f = 0;
        for (const auto &kv : s->heap.free) f += kv.second;
        return f;
    }();
    return DP_PIX_OK;
}

int dp_pix_server_destroy(dp_pix_server_t s) {
    DPPIX_RANGE();
    if (!s) return DP_PIX_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    {
        DeviceScope dev(s->device);
        for (SrvBatch &b : s->batches)
            if (b.stream) cudaStreamSynchronize(b.stream);
        if (s->key_stream) cudaStreamSynchronize(s->key_stream);
        free_server(s);
    }
    return DP_PIX_OK;
}

}  // extern "C"
