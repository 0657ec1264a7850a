// serve.cu -- request loop for viewport decoding with continuous batching.
//
// Clients (simulated headsets, players) submit viewport requests at any time
// from any thread.  A worker thread owns a set of slots; each slot is a CUDA
// stream with its own batch context.  Whenever a slot is free and requests
// are pending, the worker forms a batch from the oldest pending requests,
// admits as many as fit the device-memory limit, makes their streams resident
// and launches the batch on the slot's CUDA stream.  Requests that arrive
// while other batches are on the GPU therefore join the next batch on the
// next free slot, and batches of different slots overlap on the device.  A
// host callback enqueued after each batch stamps the completion time of its
// requests and frees the slot.
//
// Coded streams are registered once (host bytes kept in pinned memory) and
// are device-resident on demand: a stream is uploaded the first time a batch
// needs it and stays resident while the cache budget allows; when a new
// stream does not fit, the least recently used streams that no batch in
// flight references are evicted.  Paper counterpart: the asynchronous
// loading of the next frames while the current one is shown (Sec. 3.5) --
// here the unit kept resident is a whole coded group.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "wv_impl.h"

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct SvStream {
    char *host = nullptr;      // pinned copy of the coded bytes
    size_t n = 0;
    int num_frames = 0;
    size_t dev_bytes = 0;      // device bytes when resident
    wv_stream *s = nullptr;    // resident stream, or null
    int refs = 0;              // batches in flight that read it
    double last_use = 0.0;
};

struct SvReq {
    wv_server_request r;
    double t_submit = 0.0, t_done = 0.0;
    int state = 0;             // 0 pending, 1 in flight, 2 done, < 0 error code
};

struct Slot;

}  // namespace

struct wv_server {
    wv_server_config cfg;
    int device = 0;
    std::mutex m;
    std::condition_variable cv;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, SvReq> reqs;
    std::deque<SvStream> streams;   // deque: references stay valid as streams are added
    std::vector<Slot *> slots;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    size_t resident_bytes = 0;
    wv_server_stats st;
    std::vector<double> lat;   // latencies (ms) of completed requests, completion order
};

namespace {

struct Slot {
    wv_server *sv = nullptr;
    cudaStream_t cs = nullptr;
    wv_batch *b = nullptr;
    bool busy = false;
    std::vector<uint64_t> tickets;
    std::vector<int> stream_ids;
    size_t arena = 0;          // device bytes the slot's batch context holds
};

void CUDART_CB on_batch_done(void *p) {
    Slot *sl = (Slot *)p;
    wv_server *sv = sl->sv;
    const double t = now_ms();
    std::lock_guard<std::mutex> lock(sv->m);
    for (uint64_t tk : sl->tickets) {
        auto it = sv->reqs.find(tk);
        if (it == sv->reqs.end()) continue;
        it->second.state = 2;
        it->second.t_done = t;
        sv->lat.push_back(t - it->second.t_submit);
        sv->st.completed += 1;
    }
    for (int id : sl->stream_ids) sv->streams[id].refs -= 1;
    sl->tickets.clear();
    sl->stream_ids.clear();
    sl->busy = false;
    sv->cv.notify_all();
}

// Make stream `id` resident (called without the lock; the worker is the only
// thread that loads or evicts).  Returns WV_OK, or WV_ERR_OOM when the cache
// budget cannot hold it even after evicting every unreferenced stream.
int make_resident(wv_server *sv, int id, cudaStream_t cs) {
    SvStream &S = sv->streams[id];
    if (S.s) return WV_OK;
    if (sv->cfg.cache_bytes) {
        for (;;) {
            size_t used;
            int victim = -1;
            {
                std::lock_guard<std::mutex> lock(sv->m);
                used = sv->resident_bytes;
                double oldest = 1e300;
                for (size_t k = 0; k < sv->streams.size(); ++k) {
                    const SvStream &o = sv->streams[k];
                    if (o.s && o.refs == 0 && (int)k != id && o.last_use < oldest) {
                        oldest = o.last_use;
                        victim = (int)k;
                    }
                }
            }
            if (used + S.dev_bytes <= sv->cfg.cache_bytes) break;
            if (victim < 0) return WV_ERR_OOM;
            wv_close_stream(sv->streams[victim].s);
            std::lock_guard<std::mutex> lock(sv->m);
            sv->streams[victim].s = nullptr;
            sv->resident_bytes -= sv->streams[victim].dev_bytes;
            sv->st.evictions += 1;
        }
    }
    wv_stream *s = nullptr;
    const int rc = wv_open_stream(S.host, S.n, nullptr, 0, cs, &s);
    if (rc != WV_OK) return rc;
    // the upload is complete; later calls on the stream object (close) must
    // not name a slot's CUDA stream, which the server may destroy first
    wv_set_cuda_stream(s, nullptr);
    std::lock_guard<std::mutex> lock(sv->m);
    S.s = s;
    sv->resident_bytes += S.dev_bytes;
    sv->st.uploads += 1;
    return WV_OK;
}

void fail_tickets(wv_server *sv, const std::vector<uint64_t> &tk, int code) {
    std::lock_guard<std::mutex> lock(sv->m);
    for (uint64_t t : tk) {
        auto it = sv->reqs.find(t);
        if (it != sv->reqs.end()) it->second.state = code;
        sv->st.failed += 1;
    }
    sv->cv.notify_all();
}

wv_request to_request(const SvReq &q, wv_stream *s) {
    wv_request r;
    memset(&r, 0, sizeof(r));
    r.s = s;
    r.frame = q.r.frame;
    r.yaw = q.r.yaw;
    r.pitch = q.r.pitch;
    r.fov = q.r.fov;
    r.out = q.r.out;
    r.fovea = q.r.fovea;
    r.gaze_x = q.r.gaze_x;
    r.gaze_y = q.r.gaze_y;
    r.r1 = q.r.r1;
    r.r2 = q.r.r2;
    r.eye = q.r.eye;
    return r;
}

void worker_loop(wv_server *sv) {
    cudaSetDevice(sv->device);
    for (;;) {
        Slot *sl = nullptr;
        std::vector<uint64_t> cand;
        {
            std::unique_lock<std::mutex> lock(sv->m);
            sv->cv.wait(lock, [&] {
                if (sv->stop) return true;
                if (sv->pending.empty()) return false;
                for (Slot *s : sv->slots)
                    if (!s->busy) return true;
                return false;
            });
            if (sv->stop) return;
            for (Slot *s : sv->slots)
                if (!s->busy) {
                    sl = s;
                    break;
                }
            // the oldest pending requests, at most max_batch
            for (size_t i = 0; i < sv->pending.size() && (int)cand.size() < sv->cfg.max_batch; ++i)
                cand.push_back(sv->pending[i]);
        }
        // residency of the streams the candidates read; a stream made
        // resident for this batch is pinned (not evictable) until the launch
        std::vector<uint64_t> ready, failed;
        std::vector<int> pinned;
        for (uint64_t tk : cand) {
            int id;
            {
                std::lock_guard<std::mutex> lock(sv->m);
                id = sv->reqs[tk].r.stream_id;
            }
            const bool have = std::find(pinned.begin(), pinned.end(), id) != pinned.end();
            const int rc = have ? WV_OK : make_resident(sv, id, sl->cs);
            if (rc == WV_OK) {
                ready.push_back(tk);
                if (!have) {
                    std::lock_guard<std::mutex> lock(sv->m);
                    sv->streams[id].refs += 1;
                    pinned.push_back(id);
                }
            } else if (rc != WV_ERR_OOM) {
                failed.push_back(tk);
            }
            // WV_ERR_OOM: stays pending until streams in flight are released
        }
        auto unpin = [&] {
            std::lock_guard<std::mutex> lock(sv->m);
            for (int id : pinned) sv->streams[id].refs -= 1;
            pinned.clear();
            sv->cv.notify_all();
        };
        if (!failed.empty()) {
            {
                std::lock_guard<std::mutex> lock(sv->m);
                for (uint64_t tk : failed)
                    sv->pending.erase(std::find(sv->pending.begin(), sv->pending.end(), tk));
            }
            fail_tickets(sv, failed, WV_ERR_CUDA);
        }
        if (ready.empty()) {
            unpin();
            std::unique_lock<std::mutex> lock(sv->m);
            // nothing could be made resident: wait for a batch to release streams
            sv->cv.wait_for(lock, std::chrono::milliseconds(1));
            continue;
        }
        std::vector<wv_request> rq;
        {
            std::lock_guard<std::mutex> lock(sv->m);
            for (uint64_t tk : ready) {
                SvReq &q = sv->reqs[tk];
                rq.push_back(to_request(q, sv->streams[q.r.stream_id].s));
            }
        }
        // admission by device memory: the largest prefix whose batch fits
        size_t limit;
        {
            size_t free_b = 0, total_b = 0;
            cudaMemGetInfo(&free_b, &total_b);
            size_t others = 0;
            for (Slot *s : sv->slots)
                if (s != sl) others += s->arena;
            if (sv->cfg.arena_bytes)
                limit = sv->cfg.arena_bytes > others ? sv->cfg.arena_bytes - others : 0;
            else
                limit = free_b + sl->arena > sv->cfg.reserve_bytes ? free_b + sl->arena - sv->cfg.reserve_bytes : 0;
        }
        int k = (int)rq.size();
        size_t need = 0;
        while (k > 0) {
            if (wv_batch_device_bytes(sl->b, rq.data(), k, &need) == WV_OK && need <= limit) break;
            k = k > 1 ? k / 2 : 0;
        }
        if (k == 0) {
            unpin();
            bool idle = true;
            {
                std::lock_guard<std::mutex> lock(sv->m);
                for (Slot *s : sv->slots) idle = idle && !s->busy;
            }
            if (idle) {   // a single request never fits: it cannot be served
                std::vector<uint64_t> one(1, ready[0]);
                {
                    std::lock_guard<std::mutex> lock(sv->m);
                    sv->pending.erase(std::find(sv->pending.begin(), sv->pending.end(), ready[0]));
                }
                fail_tickets(sv, one, WV_ERR_OOM);
            } else {
                std::unique_lock<std::mutex> lock(sv->m);
                sv->cv.wait_for(lock, std::chrono::milliseconds(1));
            }
            continue;
        }
        {
            std::lock_guard<std::mutex> lock(sv->m);
            const double t = now_ms();
            for (int i = 0; i < k; ++i) {
                const uint64_t tk = ready[i];
                sv->pending.erase(std::find(sv->pending.begin(), sv->pending.end(), tk));
                SvReq &q = sv->reqs[tk];
                q.state = 1;
                sl->tickets.push_back(tk);
                sl->stream_ids.push_back(q.r.stream_id);
                sv->streams[q.r.stream_id].refs += 1;
                sv->streams[q.r.stream_id].last_use = t;
            }
            for (int id : pinned) sv->streams[id].refs -= 1;   // the batch's own refs now hold them
            pinned.clear();
            sl->busy = true;
            sv->st.batches += 1;
            sv->st.batched_requests += k;
            sv->st.max_batch_bytes = std::max<unsigned long long>(sv->st.max_batch_bytes, need);
        }
        int rc = wv_batch_decode(sl->b, rq.data(), k);
        if (rc == WV_OK) {
            sl->arena = wv::batch_held_bytes(sl->b);
            if (cudaLaunchHostFunc(sl->cs, on_batch_done, sl) != cudaSuccess) rc = WV_ERR_CUDA;
        }
        if (rc != WV_OK) {
            std::vector<uint64_t> tk;
            {
                std::lock_guard<std::mutex> lock(sv->m);
                tk = sl->tickets;
                for (int id : sl->stream_ids) sv->streams[id].refs -= 1;
                sl->tickets.clear();
                sl->stream_ids.clear();
                sl->busy = false;
            }
            fail_tickets(sv, tk, rc);
        }
    }
}

}  // namespace

extern "C" {

int wv_server_create(const wv_server_config *cfg, wv_server **out) {
    if (!cfg || !out || cfg->slots < 1 || cfg->slots > 16 || cfg->max_batch < 1) return WV_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return WV_ERR_CUDA;
    }
    wv_server *sv = new (std::nothrow) wv_server();
    if (!sv) return WV_ERR_OOM;
    sv->cfg = *cfg;
    memset(&sv->st, 0, sizeof(sv->st));
    cudaGetDevice(&sv->device);
    for (int i = 0; i < cfg->slots; ++i) {
        Slot *sl = new Slot();
        sl->sv = sv;
        sv->slots.push_back(sl);
        if (cudaStreamCreateWithFlags(&sl->cs, cudaStreamNonBlocking) != cudaSuccess ||
            wv_batch_create(sl->cs, &sl->b) != WV_OK) {
            cudaGetLastError();
            wv_server_close(sv);
            return WV_ERR_CUDA;
        }
    }
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return WV_OK;
}

int wv_server_add_stream(wv_server *sv, const void *bytes, size_t n, int *stream_id) {
    if (!sv || !bytes || !stream_id) return WV_ERR_ARG;
    size_t need = 0;
    wv_stream_desc d;
    const int rc = wv_stream_query(bytes, n, &d, &need);
    if (rc != WV_OK) return rc;
    SvStream S;
    if (cudaHostAlloc((void **)&S.host, n, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return WV_ERR_OOM;
    }
    memcpy(S.host, bytes, n);
    S.n = n;
    S.num_frames = d.num_frames;
    S.dev_bytes = need;
    std::lock_guard<std::mutex> lock(sv->m);
    *stream_id = (int)sv->streams.size();
    sv->streams.push_back(S);
    return WV_OK;
}

int wv_server_submit(wv_server *sv, const wv_server_request *r, uint64_t *ticket) {
    if (!sv || !r || !ticket) return WV_ERR_ARG;
    std::lock_guard<std::mutex> lock(sv->m);
    if (r->stream_id < 0 || r->stream_id >= (int)sv->streams.size()) return WV_ERR_ARG;
    const wv_image &o = r->out;
    if (!o.dptr || o.width <= 0 || o.height <= 0 || o.pitch_bytes < (size_t)o.width * 4 ||
        !(r->fov > 0.f && r->fov < 3.14159f) || r->frame < 0 ||
        r->frame >= sv->streams[r->stream_id].num_frames)
        return WV_ERR_ARG;
    SvReq q;
    q.r = *r;
    q.t_submit = now_ms();
    const uint64_t tk = sv->next_ticket++;
    sv->reqs[tk] = q;
    sv->pending.push_back(tk);
    sv->st.submitted += 1;
    *ticket = tk;
    sv->cv.notify_all();
    return WV_OK;
}

int wv_server_poll(wv_server *sv, uint64_t ticket, double *latency_ms) {
    if (!sv) return WV_ERR_ARG;
    std::lock_guard<std::mutex> lock(sv->m);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return WV_ERR_ARG;
    const int state = it->second.state;
    if (state == 0 || state == 1) return 1;
    if (latency_ms) *latency_ms = it->second.t_done - it->second.t_submit;
    sv->reqs.erase(it);
    return state == 2 ? WV_OK : state;
}

int wv_server_wait(wv_server *sv, uint64_t ticket, double timeout_ms, double *latency_ms) {
    if (!sv) return WV_ERR_ARG;
    std::unique_lock<std::mutex> lock(sv->m);
    auto done = [&] {
        auto it = sv->reqs.find(ticket);
        return it == sv->reqs.end() || it->second.state >= 2 || it->second.state < 0;
    };
    if (!sv->cv.wait_for(lock, std::chrono::duration<double, std::milli>(timeout_ms), done))
        return WV_ERR_TIMEOUT;
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return WV_ERR_ARG;
    const int state = it->second.state;
    if (latency_ms) *latency_ms = it->second.t_done - it->second.t_submit;
    sv->reqs.erase(it);
    return state == 2 ? WV_OK : state;
}

int wv_server_drain(wv_server *sv, double timeout_ms) {
    if (!sv) return WV_ERR_ARG;
    std::unique_lock<std::mutex> lock(sv->m);
    auto idle = [&] {
        if (!sv->pending.empty()) return false;
        for (Slot *s : sv->slots)
            if (s->busy) return false;
        return true;
    };
    return sv->cv.wait_for(lock, std::chrono::duration<double, std::milli>(timeout_ms), idle)
               ? WV_OK
               : WV_ERR_TIMEOUT;
}

int wv_server_get_stats(wv_server *sv, wv_server_stats *out) {
    if (!sv || !out) return WV_ERR_ARG;
    std::lock_guard<std::mutex> lock(sv->m);
    *out = sv->st;
    out->resident_bytes = sv->resident_bytes;
    unsigned long long arena = 0;
    for (Slot *s : sv->slots) arena += s->arena;
    out->arena_bytes = arena;
    return WV_OK;
}

int wv_server_latencies(wv_server *sv, double *out, int cap, int *n) {
    if (!sv || !n || cap < 0 || (cap > 0 && !out)) return WV_ERR_ARG;
    std::lock_guard<std::mutex> lock(sv->m);
    const int k = std::min<int>(cap, (int)sv->lat.size());
    for (int i = 0; i < k; ++i) out[i] = sv->lat[i];
    *n = (int)sv->lat.size();
    return WV_OK;
}

int wv_server_reset_stats(wv_server *sv) {
    if (!sv) return WV_ERR_ARG;
    std::lock_guard<std::mutex> lock(sv->m);
    memset(&sv->st, 0, sizeof(sv->st));
    sv->lat.clear();
    return WV_OK;
}

void wv_server_close(wv_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lock(sv->m);
        sv->stop = true;
        sv->cv.notify_all();
    }
    if (sv->worker.joinable()) sv->worker.join();
    // batches in flight (and their completion callbacks) finish first
    for (Slot *sl : sv->slots)
        if (sl->cs) cudaStreamSynchronize(sl->cs);
    for (SvStream &S : sv->streams) {
        if (S.s) wv_close_stream(S.s);
        if (S.host) cudaFreeHost(S.host);
    }
    for (Slot *sl : sv->slots) {
        if (sl->b) wv_batch_close(sl->b);
        if (sl->cs) cudaStreamDestroy(sl->cs);
        delete sl;
    }
    delete sv;
}

}  // extern "C"
