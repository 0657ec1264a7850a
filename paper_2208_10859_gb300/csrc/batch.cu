// batch.cu -- batched viewport decoding: many requests over several streams
// of uneven size, field of view and foveation in one CUDA graph.
//
// One batch is one graph on the batch's CUDA stream: the upload of the job
// tables (one copy from pinned host memory) and the clearing of the work
// counters, then per wave of decode targets:
//   1. clearing of the wave's tile stamps;
//   2. footprint of every request of the wave (k_footprint_batch, one grid
//      slice each);
//   3. tile lists of every decode target of the wave (k_select_batch);
//   4. per decode class (wavelet, number of coefficient frames the
//      inter-frame rebuild reads) one persistent tile-decode launch over all
//      coarse, then all fine tiles of its targets (k_tiles_batch);
//   5. reprojection of every request of the wave (k_resample_batch).
// Requests of the same stream and frame without foveation share one decode
// target ("surface"), so a tile that several viewports need is decoded once.
// A foveated request (Sec. 3.7) has a surface of its own, since the details
// it drops depend on its gaze.  Surfaces are grouped, in request order, into
// waves whose planes fit the context's memory limit; every wave reuses the
// same device region, so the arena stays bounded however many requests a
// batch holds, and the requests of an early wave are complete before the
// later waves run.  The instantiated graph is kept and relaunched while the
// batch keeps its shape (counts, sizes, arena); between launches only the
// job tables change.
//
// Tile shapes (output tiles 64 x 64, 128 x 128, 256 x 64 or 256 x 128
// samples, coarse tile 32 or 64 samples of LL_2) are chosen per (wavelet,
// levels, frame size) by an autotuner that times the batch with each shape
// (wv_batch_autotune).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "wv_impl.h"

using namespace wv;

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

using TuneKey = std::array<int, 4>;   // wavelet, levels, width, height

struct Shape {
    int tw, th, ctile;   // output tile (plane samples), coarse tile (LL_2 samples)
    bool operator==(const Shape &o) const { return tw == o.tw && th == o.th && ctile == o.ctile; }
};
constexpr Shape kDefaultShape = {kTile, kTile, kCoarseTile};
// Output tiles the batch decoder takes: the fine pass's shared arrays of a
// 256 x 128 tile (levels 2 and 1, 9/7) are about 174 KB, of 256 x 256 about
// 340 KB (too large).
bool shape_ok(int tw, int th, int ctile) {
    const bool out = (tw == 64 && th == 64) || (tw == 128 && th == 128) || (tw == 256 && (th == 64 || th == 128));
    return out && (ctile == 32 || ctile == 64);
}

struct Surface {
    wv_stream *s;
    int frame;
    bool foveated;
    Geom g;
    int cls;
    bool strip;     // fine tiles are strips (k_strip_batch), else square tiles
    bool pair;      // reconstruction chroma held as alternating Cb, Cr groups of 4
    int wave;
    size_t bytes;   // device bytes of its stamps, list entries and planes
    size_t recon[3], ll2[3], fmask, stamp;   // arena offsets (inside the wave region)
};

// Arena word holding the bounded wait's poll limit (inside the 256 bytes
// before the job tables; the error word is at offset 0).
constexpr size_t kWaitWord = 64;

// A wave: surfaces [s0, s1) and the rows [r0, r1) of the request table (the
// table lists requests by wave, in caller order inside a wave).
struct Wave {
    int s0, s1, r0, r1;
    size_t ctr;            // its counters (kBatchCtr + 2 (s1 - s0) ints)
    size_t stamps, stamp_bytes;
    size_t lists_c[kClasses], lists_f[kClasses], lists_s[kClasses];
    int smem[kClasses];    // dynamic shared memory of each class's decode (0: class absent)
    bool strip[kClasses];  // the class has strip surfaces in this wave
    int max_cx, max_cy, max_stamps, max_w, max_h;
};

struct Plan {
    std::vector<Surface> surf;
    std::vector<int> req_surface;   // per request (caller order)
    std::vector<int> order;         // request table row -> request index
    std::vector<Wave> waves;
    size_t err, jobs, reqs, ctr, region, total;
    size_t ctr_bytes;               // counters of all waves, cleared every launch
    int n_ctr;
    size_t job_bytes;
};

}  // namespace

struct wv_batch {
    int device = 0;
    cudaStream_t cs = nullptr;         // stream of the last launch
    cudaStream_t cap = nullptr;        // private stream for graph capture
    char *dmem = nullptr;
    size_t dbytes = 0;
    char *host = nullptr;              // pinned job-table staging
    size_t hbytes = 0;
    cudaEvent_t staged = nullptr;      // the last launch's upload has finished
    cudaEvent_t done = nullptr;        // the last launch has finished
    bool launched = false;
    bool use_graph = true;
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> shape;      // key of the instantiated graph
    std::map<TuneKey, Shape> tuned;
    int *err = nullptr;
    // statistics of the last launch (read back on request)
    int last_requests = 0, last_surfaces = 0;
    int *ctr_dev = nullptr;
    int n_ctr = 0;
    std::vector<int> ctr_base;         // first counter of each wave of the last launch
    std::vector<int> req_wave;         // wave of each request of the last launch
    // per-step timing of the last launch (direct mode only): a start event,
    // then 5 per wave (after the stamp clear, footprint, lists, decode,
    // reprojection)
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    bool share = true;                 // unfoveated requests of one (stream, frame) share a surface
    int wait_polls = kBatchWaitPolls;  // polls of the tile decode's bounded wait (arena word at kWaitWord)
    size_t wave_bytes = kBatchWaveBytes;   // device bytes of one wave's surfaces (0: one wave)
    bool strips = true;                // fine levels of eligible targets as strips
};

namespace {

int check_request(const wv_request &r) {
    if (!r.s) return WV_ERR_ARG;
    if (r.s->g.quant != 0) return WV_ERR_ARG;   // the paper-format quantiser has no batched kernel
    if (r.frame < 0 || r.frame >= r.s->g.num_frames) return WV_ERR_ARG;
    if (!(r.fov > 0.f && r.fov < 3.14159f) || !isfinite(r.yaw) || !isfinite(r.pitch)) return WV_ERR_ARG;
    const wv_image *o = &r.out;
    if (!o->dptr || o->width <= 0 || o->height <= 0 || o->pitch_bytes < (size_t)o->width * 4 ||
        (o->pitch_bytes % 4) != 0 || ((uintptr_t)o->dptr % 4) != 0)
        return WV_ERR_ARG;
    if (r.fovea != 0 && r.fovea != 1) return WV_ERR_ARG;
    int row0, rows;
    if (eye_view(r.s->g, r.eye, &row0, &rows) != WV_OK) return WV_ERR_ARG;
    if (r.fovea && (!isfinite(r.gaze_x) || !isfinite(r.gaze_y) || isnan(r.r1) || isnan(r.r2)))
        return WV_ERR_ARG;
    return WV_OK;
}

Shape tile_shape(const wv_batch *b, const Geom &g) {
    auto it = b->tuned.find(TuneKey{g.wavelet, g.levels, g.p[0].w, g.p[0].h});
    return it == b->tuned.end() ? kDefaultShape : it->second;
}

// Device bytes of a surface's own data: stamps, worst-case list entries,
// reconstruction and LL_2 planes, foveation cell bits (each 256-aligned).
size_t surface_bytes(const Surface &S) {
    size_t o = sizeof(uint32_t) * (S.g.total_tiles + S.g.total_ctiles);
    o += sizeof(uint2) * ((S.strip ? 2 : 1) * S.g.total_tiles + S.g.total_ctiles) + 768;
    for (int p = 0; p < S.g.planes; ++p) {
        o += align256((size_t)S.g.p[p].w * S.g.p[p].h);
        if (S.g.levels >= 3) o += align256((size_t)S.g.p[p].ll2_pitch * (S.g.p[p].h >> 2) * 4);
    }
    if (S.foveated) o += align256((size_t)S.g.cells_x * S.g.cells_y);
    return o;
}

int plan_batch(const wv_batch *b, const wv_request *reqs, int n, Plan &P) {
    std::map<std::pair<const wv_stream *, int>, int> shared;
    P.surf.clear();
    P.waves.clear();
    P.req_surface.assign(n, -1);
    for (int i = 0; i < n; ++i) {
        const wv_request &r = reqs[i];
        if (!r.fovea && b->share) {
            auto it = shared.find({r.s, r.frame});
            if (it != shared.end()) {
                P.req_surface[i] = it->second;
                continue;
            }
        }
        Surface S{};
        S.s = r.s;
        S.frame = r.frame;
        S.foveated = r.fovea != 0;
        const Geom &sg = r.s->g;
        const Shape ts = tile_shape(b, sg);
        // strip tiles for the fine levels where the batched strip pass has
        // the class (the tuned square shape then only sets the coarse tile)
        S.strip = b->strips && strip_eligible(r.s->desc, r.s->n_payload) &&
                  strip_batch_supported(sg.wavelet, 1 + sg.tlevels, sg.dz_t);
        const int gr = S.strip ? build_geom_strip(r.s->desc, &S.g, kStripH, ts.ctile)
                               : build_geom_rect(r.s->desc, &S.g, ts.tw, ts.th, ts.ctile);
        if (gr != WV_OK) return WV_ERR_ARG;
        S.g.dz_t = sg.dz_t;   // the code form of the stream's device payload
        S.g.n_blocks = sg.n_blocks;
        // 1 + tlevels coefficient frames
        const int group = S.g.dz_t ? 4 + (S.foveated ? 1 : 0) : 2 * S.g.wavelet + (S.foveated ? 1 : 0);
        S.cls = kMaxBands * group + S.g.tlevels;
        S.bytes = surface_bytes(S);
        P.req_surface[i] = (int)P.surf.size();
        if (!r.fovea) shared[{r.s, r.frame}] = (int)P.surf.size();
        P.surf.push_back(S);
    }
    const int m = (int)P.surf.size();
    // waves: surfaces in order while their bytes fit the limit (a surface
    // larger than the limit forms a wave of its own)
    {
        size_t acc = 0;
        int s0 = 0;
        for (int i = 0; i < m; ++i) {
            if (i > s0 && b->wave_bytes && acc + P.surf[i].bytes > b->wave_bytes) {
                P.waves.push_back(Wave{s0, i});
                s0 = i;
                acc = 0;
            }
            acc += P.surf[i].bytes;
            P.surf[i].wave = (int)P.waves.size();
        }
        if (m > 0) P.waves.push_back(Wave{s0, m});
    }
    // request table: by wave, caller order inside a wave
    P.order.clear();
    for (Wave &W : P.waves) {
        W.r0 = (int)P.order.size();
        for (int i = 0; i < n; ++i)
            if (P.req_surface[i] >= W.s0 && P.req_surface[i] < W.s1) P.order.push_back(i);
        W.r1 = (int)P.order.size();
    }
    // arena: error word | job tables | counters of every wave | wave region
    // (stamps | lists | per-surface planes, reused by every wave).  The error
    // word stays at offset 0 for every plan.
    P.err = 0;
    size_t o = 256;
    P.jobs = o;
    o = align256(o + sizeof(SurfaceJob) * m);
    P.reqs = o;
    o = align256(o + sizeof(RequestJob) * n);
    P.job_bytes = o;
    P.ctr = o;
    P.n_ctr = 0;
    for (Wave &W : P.waves) {
        W.ctr = P.ctr + sizeof(int) * P.n_ctr;
        P.n_ctr += kBatchCtr + 2 * (W.s1 - W.s0);
    }
    P.ctr_bytes = sizeof(int) * P.n_ctr;
    P.region = align256(P.ctr + P.ctr_bytes);
    P.total = P.region;
    for (Wave &W : P.waves) {
        o = P.region;
        W.stamps = o;
        size_t tiles[kClasses] = {}, ctiles[kClasses] = {}, stiles[kClasses] = {};
        W.max_cx = W.max_cy = W.max_stamps = W.max_w = W.max_h = 0;
        for (int si = W.s0; si < W.s1; ++si) {
            Surface &S = P.surf[si];
            S.stamp = o;
            o += sizeof(uint32_t) * (S.g.total_tiles + S.g.total_ctiles);
            (S.strip ? stiles : tiles)[S.cls] += (S.strip ? 2 : 1) * (size_t)S.g.total_tiles;
            ctiles[S.cls] += S.g.total_ctiles;
            W.max_cx = std::max(W.max_cx, S.g.cells_x);
            W.max_cy = std::max(W.max_cy, S.g.cells_y);
            W.max_stamps = std::max(W.max_stamps, S.g.total_tiles + S.g.total_ctiles);
        }
        W.stamp_bytes = o - W.stamps;
        o = align256(o);
        for (int c = 0; c < kClasses; ++c) {
            W.lists_c[c] = o;
            o = align256(o + sizeof(uint2) * std::max<size_t>(ctiles[c], 1));
            W.lists_f[c] = o;
            o = align256(o + sizeof(uint2) * std::max<size_t>(tiles[c], 1));
            W.lists_s[c] = o;
            o = align256(o + sizeof(uint2) * std::max<size_t>(stiles[c], 1));
            W.strip[c] = stiles[c] > 0;
        }
        for (int si = W.s0; si < W.s1; ++si) {
            Surface &S = P.surf[si];
            for (int p = 0; p < 3; ++p) {
                S.recon[p] = o;
                if (p < S.g.planes) o = align256(o + (size_t)S.g.p[p].w * S.g.p[p].h);
            }
            // chroma as alternating Cb, Cr groups of 4: strip targets whose
            // two chroma planes are back to back
            S.pair = S.strip && S.g.planes == 3 && S.recon[2] == S.recon[1] + (size_t)S.g.p[1].w * S.g.p[1].h;
            for (int p = 0; p < 3; ++p) {
                S.ll2[p] = o;
                if (p < S.g.planes && S.g.levels >= 3)
                    o = align256(o + (size_t)S.g.p[p].ll2_pitch * (S.g.p[p].h >> 2) * 4);
            }
            S.fmask = o;
            if (S.foveated) o = align256(o + (size_t)S.g.cells_x * S.g.cells_y);
        }
        P.total = std::max(P.total, o);
        for (int k = W.r0; k < W.r1; ++k) {
            W.max_w = std::max(W.max_w, reqs[P.order[k]].out.width);
            W.max_h = std::max(W.max_h, reqs[P.order[k]].out.height);
        }
        for (int c = 0; c < kClasses; ++c) W.smem[c] = 0;
    }
    return WV_OK;
}

TileArgs pass_args(const Surface &S, char *base, int *err, bool coarse) {
    TileArgs a;
    memset(&a, 0, sizeof(a));
    a.g = S.g;
    a.payload = S.s->payload;
    a.table = S.s->table;
    a.bands = frame_bands(S.g, S.frame);
    a.err = err;
    a.f32_plane = -1;
    a.fmask = S.foveated ? (const uint8_t *)(base + S.fmask) : nullptr;
    if (kChecked) a.n_slots = S.g.n_blocks;
    const bool split = S.g.levels >= 3;
    if (coarse) {
        a.l_top = S.g.levels;
        a.l_bot = 3;
        a.tw = a.th = S.g.ctile;
        for (int p = 0; p < S.g.planes; ++p) {
            a.ll_out[p] = (float *)(base + S.ll2[p]);
            a.ll_out_pitch[p] = S.g.p[p].ll2_pitch;
        }
    } else {
        a.l_top = split ? 2 : S.g.levels;
        a.l_bot = 1;
        a.tw = S.g.tw;
        a.th = S.g.th;
        for (int p = 0; p < S.g.planes; ++p) {
            a.out_u8[p] = (uint8_t *)(base + S.recon[p]);
            if (split) {
                a.ll_in[p] = (const float *)(base + S.ll2[p]);
                a.ll_in_pitch[p] = S.g.p[p].ll2_pitch;
            }
        }
    }
    fill_tile_scales(a);
    return a;
}

// Fill the host job tables (pinned staging) for the planned arena.
void fill_jobs(wv_batch *b, const wv_request *reqs, int n, Plan &P) {
    char *base = b->dmem;
    int *err = (int *)(base + P.err);
    SurfaceJob *sj = (SurfaceJob *)(b->host + P.jobs);
    RequestJob *rj = (RequestJob *)(b->host + P.reqs);
    *(int *)(b->host + kWaitWord) = b->wait_polls;
    for (size_t i = 0; i < P.surf.size(); ++i) {
        const Surface &S = P.surf[i];
        SurfaceJob J;
        memset(&J, 0, sizeof(J));
        J.fine = pass_args(S, base, err, false);
        if (S.g.levels >= 3) J.coarse = pass_args(S, base, err, true);
        J.stamp = (uint32_t *)(base + S.stamp);
        J.fmask = S.foveated ? (uint8_t *)(base + S.fmask) : nullptr;
        J.cls = S.cls;
        J.strip = S.strip ? 1 : 0;
        if (S.pair) {   // chroma as alternating Cb, Cr groups of 4 (chroma planes adjacent)
            J.fine.out_pair = 1;
            J.fine.out_u8[2] = J.fine.out_u8[1] + 4;
        }
        // the class's tile decode takes only the coarse tiles of strip surfaces
        int need = S.strip ? 0 : (J.fine.a_floats + J.fine.p_floats) * 4;
        if (S.g.levels >= 3) need = std::max(need, (J.coarse.a_floats + J.coarse.p_floats) * 4);
        int &sm = P.waves[S.wave].smem[S.cls];
        sm = std::max(sm, need);
        memcpy(&sj[i], &J, sizeof(J));
    }
    for (int k = 0; k < n; ++k) {
        const int i = P.order[k];
        const wv_request &r = reqs[i];
        const Surface &S = P.surf[P.req_surface[i]];
        RequestJob R;
        memset(&R, 0, sizeof(R));
        int row0, rows;
        eye_view(S.g, r.eye, &row0, &rows);   // validated by check_request
        R.v = make_view(r.yaw, r.pitch, r.fov, r.out.width, r.out.height, S.g.p[0].w, rows, row0);
        R.f = make_frustum(R.v);
        R.fov.on = r.fovea;
        R.fov.gx = r.gaze_x;
        R.fov.gy = r.gaze_y;
        R.fov.r1 = r.r1;
        R.fov.r2 = r.r2;
        R.surface = P.req_surface[i] - P.waves[S.wave].s0;   // index within the wave
        R.rs.v = R.v;
        for (int p = 0; p < 3; ++p) {
            const bool has = p < S.g.planes;
            R.rs.plane[p] = has ? (const uint8_t *)(base + S.recon[p]) : nullptr;
            R.rs.w[p] = has ? S.g.p[p].w : 0;
            R.rs.h[p] = has ? S.g.p[p].h : 0;
        }
        R.rs.planes = S.g.planes;
        R.rs.c420 = S.g.c420;
        R.rs.c_pair = S.pair ? 1 : 0;
        R.rs.err = err;
        R.rs.uv = nullptr;
        R.rs.out = (uint8_t *)r.out.dptr;
        R.rs.pitch = r.out.pitch_bytes;
        memcpy(&rj[k], &R, sizeof(R));
    }
}

// Enqueue the batch on cs (captured into a graph, or run directly with
// events between the steps when timed).
cudaError_t enqueue(wv_batch *b, const Plan &P, int n, cudaStream_t cs, bool timed) {
    char *base = b->dmem;
    const SurfaceJob *surfs = (const SurfaceJob *)(base + P.jobs);
    const RequestJob *rq = (const RequestJob *)(base + P.reqs);
    if (timed) cudaEventRecord(b->ev[0], cs);
    // the wait limit word, then the job tables (the error word at 0 stays)
    cudaError_t e = cudaMemcpyAsync(base + kWaitWord, b->host + kWaitWord, P.job_bytes - kWaitWord,
                                    cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return e;
    e = cs == b->cap ? cudaEventRecordWithFlags(b->staged, cs, cudaEventRecordExternal) : cudaEventRecord(b->staged, cs);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(base + P.ctr, 0, P.ctr_bytes, cs);
    if (e != cudaSuccess) return e;
    for (size_t w = 0; w < P.waves.size(); ++w) {
        const Wave &W = P.waves[w];
        cudaEvent_t *ev = timed ? &b->ev[1 + 5 * w] : nullptr;
        const int m = W.s1 - W.s0, nr = W.r1 - W.r0;
        int *ctr = (int *)(base + W.ctr);
        e = cudaMemsetAsync(base + W.stamps, 0, W.stamp_bytes, cs);
        if (e != cudaSuccess) return e;
        if (timed) cudaEventRecord(ev[0], cs);
        launch_footprint_batch(rq + W.r0, surfs + W.s0, nr, W.max_cx, W.max_cy, cs);
        if (timed) cudaEventRecord(ev[1], cs);
        BatchLists lists;
        for (int c = 0; c < kClasses; ++c) {
            lists.coarse[c] = (uint2 *)(base + W.lists_c[c]);
            lists.fine[c] = (uint2 *)(base + W.lists_f[c]);
            lists.strip[c] = (uint2 *)(base + W.lists_s[c]);
        }
        launch_select_batch(surfs + W.s0, m, W.max_stamps, lists, ctr, cs);
        if (timed) cudaEventRecord(ev[2], cs);
        for (int c = 0; c < kClasses; ++c) {
            if (!W.smem[c]) continue;
            const int group = c / kMaxBands;
            e = launch_decode_batch(group >= 4 ? WV_WAVELET_97 : group / 2, c % kMaxBands + 1, group % 2 == 1,
                                    group >= 4, surfs + W.s0, lists.coarse[c], lists.fine[c], ctr + 4 * c,
                                    ctr + kBatchCtr, (int *)(base + P.err), (const int *)(base + kWaitWord),
                                    W.smem[c], cs);
            if (e != cudaSuccess) return e;
        }
        // the strip tiles, once their class's coarse tiles are done
        for (int c = 0; c < kClasses; ++c) {
            if (!W.strip[c]) continue;
            const int group = c / kMaxBands;
            e = launch_decode_strips_batch(group >= 4 ? WV_WAVELET_97 : group / 2, c % kMaxBands + 1, group % 2 == 1,
                                           group >= 4, surfs + W.s0, lists.strip[c], ctr + 4 * c + 3, cs);
            if (e != cudaSuccess) return e;
        }
        if (timed) cudaEventRecord(ev[3], cs);
        launch_resample_batch(rq + W.r0, nr, W.max_w, W.max_h, cs);
        if (timed) cudaEventRecord(ev[4], cs);
    }
    return cudaGetLastError();
}

std::vector<long long> shape_key(const wv_batch *b, const Plan &P, int n) {
    std::vector<long long> k = {n, (long long)P.surf.size(), (long long)(uintptr_t)b->dmem,
                                (long long)(uintptr_t)b->host, (long long)P.job_bytes,
                                (long long)P.ctr_bytes, (long long)P.waves.size()};
    for (const Wave &W : P.waves) {
        for (long long v : {(long long)W.s0, (long long)W.s1, (long long)W.r0, (long long)W.r1, (long long)W.ctr,
                            (long long)W.stamps, (long long)W.stamp_bytes, (long long)W.max_cx,
                            (long long)W.max_cy, (long long)W.max_stamps, (long long)W.max_w, (long long)W.max_h})
            k.push_back(v);
        for (int c = 0; c < kClasses; ++c) {
            k.push_back(W.smem[c]);
            k.push_back((long long)W.lists_c[c]);
            k.push_back((long long)W.lists_f[c]);
            k.push_back((long long)W.lists_s[c]);
            k.push_back(W.strip[c] ? 1 : 0);
        }
    }
    return k;
}

// Events of a timed launch: one start event and five per wave.
int ensure_events(wv_batch *b, size_t waves) {
    while (b->ev.size() < 1 + 5 * waves) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return WV_ERR_CUDA;
        }
        b->ev.push_back(e);
    }
    return WV_OK;
}

int ensure_memory(wv_batch *b, const Plan &P) {
    if (P.total > b->dbytes) {
        if (b->launched) cudaEventSynchronize(b->done);
        if (b->dmem) cudaFree(b->dmem);
        b->dmem = nullptr;
        b->dbytes = 0;
        const size_t want = P.total + P.total / 4;
        if (dev_alloc((void **)&b->dmem, want) != cudaSuccess) {
            cudaGetLastError();
            return WV_ERR_OOM;
        }
        b->dbytes = want;
        cudaMemset(b->dmem + P.err, 0, 64);
    }
    if (P.job_bytes > b->hbytes) {
        if (b->launched) cudaEventSynchronize(b->done);
        if (b->host) cudaFreeHost(b->host);
        b->host = nullptr;
        b->hbytes = 0;
        const size_t want = P.job_bytes + P.job_bytes / 4;
        if (cudaHostAlloc((void **)&b->host, want, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return WV_ERR_OOM;
        }
        b->hbytes = want;
    }
    return WV_OK;
}

int run_batch(wv_batch *b, const wv_request *reqs, int n, cudaStream_t cs) {
    if (!b || n < 0 || (n > 0 && !reqs)) return WV_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        const int rc = check_request(reqs[i]);
        if (rc != WV_OK) return rc;
    }
    if (n == 0) return WV_OK;
    Plan P;
    int rc = plan_batch(b, reqs, n, P);
    if (rc != WV_OK) return rc;
    rc = ensure_memory(b, P);
    if (rc != WV_OK) return rc;
    if (b->timing && (rc = ensure_events(b, P.waves.size())) != WV_OK) return rc;
    // the previous launch must have consumed the staging before it is rewritten
    if (b->launched) cudaEventSynchronize(b->staged);
    fill_jobs(b, reqs, n, P);
    // a launch on another CUDA stream than the previous one waits for it
    if (b->launched && cs != b->cs) cudaStreamWaitEvent(cs, b->done, 0);
    b->err = (int *)(b->dmem + P.err);
    b->ctr_dev = (int *)(b->dmem + P.ctr);
    b->n_ctr = P.n_ctr;
    b->last_requests = n;
    b->last_surfaces = (int)P.surf.size();
    b->ctr_base.clear();
    for (const Wave &W : P.waves) b->ctr_base.push_back((int)((W.ctr - P.ctr) / sizeof(int)));
    b->req_wave.assign(n, 0);
    for (int i = 0; i < n; ++i) b->req_wave[i] = P.surf[P.req_surface[i]].wave;
    cudaError_t e;
    if (b->use_graph && !b->timing) {
        const std::vector<long long> key = shape_key(b, P, n);
        if (!b->exec || key != b->shape) {
            if (b->exec) cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) {
                const cudaError_t e1 = enqueue(b, P, n, b->cap, false);
                e = cudaStreamEndCapture(b->cap, &graph);
                if (e1 != cudaSuccess) e = e1;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                cudaGetLastError();
                b->exec = nullptr;
                return WV_ERR_CUDA;
            }
            b->shape = key;
        }
        e = cudaGraphLaunch(b->exec, cs);
    } else {
        e = enqueue(b, P, n, cs, b->timing);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->done, cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return WV_ERR_CUDA;
    }
    b->cs = cs;
    b->launched = true;
    return WV_OK;
}

}  // namespace

namespace wv {
size_t batch_held_bytes(const wv_batch *b) { return b ? b->dbytes : 0; }
}  // namespace wv

namespace {

std::mutex g_default_mutex;
std::map<int, wv_batch *> g_default;   // per device: the context of wv_decode_batch

}  // namespace

extern "C" {

int wv_batch_create(void *cuda_stream, wv_batch **out) {
    if (!out) return WV_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return WV_ERR_CUDA;
    }
    wv_batch *b = new (std::nothrow) wv_batch();
    if (!b) return WV_ERR_OOM;
    cudaGetDevice(&b->device);
    b->cs = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        wv_batch_close(b);
        return WV_ERR_CUDA;
    }
    *out = b;
    return WV_OK;
}

void wv_batch_close(wv_batch *b) {
    if (!b) return;
    if (b->launched) cudaEventSynchronize(b->done);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->dmem) cudaFree(b->dmem);
    if (b->host) cudaFreeHost(b->host);
    if (b->staged) cudaEventDestroy(b->staged);
    if (b->done) cudaEventDestroy(b->done);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

int wv_batch_decode(wv_batch *b, const wv_request *reqs, int n) {
    if (!b) return WV_ERR_ARG;
    return run_batch(b, reqs, n, b->cs);
}

int wv_batch_set_cuda_stream(wv_batch *b, void *cuda_stream) {
    if (!b) return WV_ERR_ARG;
    if (b->launched && (cudaStream_t)cuda_stream != b->cs)
        cudaStreamWaitEvent((cudaStream_t)cuda_stream, b->done, 0);
    b->cs = (cudaStream_t)cuda_stream;
    return WV_OK;
}

int wv_batch_device_bytes(wv_batch *b, const wv_request *reqs, int n, size_t *bytes) {
    if (!b || !bytes || n < 0 || (n > 0 && !reqs)) return WV_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (check_request(reqs[i]) != WV_OK) return WV_ERR_ARG;
    Plan P;
    const int rc = plan_batch(b, reqs, n, P);
    if (rc != WV_OK) return rc;
    *bytes = P.total;
    return WV_OK;
}

int wv_batch_sync_status(wv_batch *b) {
    if (!b) return WV_ERR_ARG;
    if (!b->launched) return WV_OK;
    if (cudaEventSynchronize(b->done) != cudaSuccess) return WV_ERR_CUDA;
    int err = 0;
    if (cudaMemcpy(&err, b->err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return WV_ERR_CUDA;
    if (err) cudaMemset(b->err, 0, 4);
    return err;
}

int wv_batch_stats(wv_batch *b, wv_batch_info *info) {
    if (!b || !info) return WV_ERR_ARG;
    memset(info, 0, sizeof(*info));
    if (!b->launched) return WV_OK;
    if (cudaEventSynchronize(b->done) != cudaSuccess) return WV_ERR_CUDA;
    std::vector<int> c(b->n_ctr);
    if (cudaMemcpy(c.data(), b->ctr_dev, sizeof(int) * b->n_ctr, cudaMemcpyDeviceToHost) != cudaSuccess)
        return WV_ERR_CUDA;
    info->requests = b->last_requests;
    info->surfaces = b->last_surfaces;
    info->waves = (int)b->ctr_base.size();
    for (int c0 : b->ctr_base)
        for (int k = 0; k < kClasses; ++k) {
            info->coarse_tiles += c[c0 + 4 * k + 1];
            info->fine_tiles += c[c0 + 4 * k + 2] + c[c0 + 4 * k + 3];
        }
    info->bytes = b->dbytes;
    if (b->timing) {
        float ms = 0.f;
        for (size_t w = 0; w < b->ctr_base.size(); ++w)
            for (int i = 0; i < 4; ++i) {
                cudaEventElapsedTime(&ms, b->ev[1 + 5 * w + i], b->ev[1 + 5 * w + i + 1]);
                info->ms[i] += ms;
            }
    }
    return WV_OK;
}

int wv_batch_completion_ms(wv_batch *b, double *ms, int n) {
    if (!b || !ms || n < 0) return WV_ERR_ARG;
    if (!b->launched || !b->timing || n != b->last_requests || b->ev.size() < 1 + 5 * b->ctr_base.size())
        return WV_ERR_ARG;
    if (cudaEventSynchronize(b->done) != cudaSuccess) return WV_ERR_CUDA;
    for (int i = 0; i < n; ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, b->ev[0], b->ev[1 + 5 * b->req_wave[i] + 4]) != cudaSuccess) return WV_ERR_CUDA;
        ms[i] = t;
    }
    return WV_OK;
}

int wv_batch_set_memory_limit(wv_batch *b, size_t bytes) {
    if (!b) return WV_ERR_ARG;
    b->wave_bytes = bytes;
    return WV_OK;
}

int wv_batch_set_wait_limit(wv_batch *b, int polls) {
    if (!b || polls < 0) return WV_ERR_ARG;
    b->wait_polls = std::min(polls, kBatchWaitPolls);
    return WV_OK;
}

int wv_batch_set_sharing(wv_batch *b, int on) {
    if (!b || on < 0 || on > 1) return WV_ERR_ARG;
    b->share = on != 0;
    return WV_OK;
}

int wv_batch_set_strips(wv_batch *b, int on) {
    if (!b || on < 0 || on > 1) return WV_ERR_ARG;
    b->strips = on != 0;
    return WV_OK;
}

int wv_batch_set_timing(wv_batch *b, int on) {
    if (!b || on < 0 || on > 1) return WV_ERR_ARG;
    b->timing = on != 0;
    return WV_OK;
}

int wv_batch_set_tile_shape(wv_batch *b, int wavelet, int levels, int width, int height,
                            int tile_w, int tile_h, int ctile) {
    if (!b || !shape_ok(tile_w, tile_h, ctile)) return WV_ERR_ARG;
    b->tuned[TuneKey{wavelet, levels, width, height}] = Shape{tile_w, tile_h, ctile};
    return WV_OK;
}

int wv_batch_tile_shape(wv_batch *b, int wavelet, int levels, int width, int height, int *tile_w,
                        int *tile_h, int *ctile) {
    if (!b || !tile_w || !tile_h || !ctile) return WV_ERR_ARG;
    auto it = b->tuned.find(TuneKey{wavelet, levels, width, height});
    const Shape sh = it == b->tuned.end() ? kDefaultShape : it->second;
    *tile_w = sh.tw;
    *tile_h = sh.th;
    *ctile = sh.ctile;
    return WV_OK;
}

int wv_batch_autotune(wv_batch *b, const wv_request *reqs, int n, int reps) {
    if (!b || n <= 0 || !reqs || reps < 1) return WV_ERR_ARG;
    std::vector<TuneKey> keys;
    for (int i = 0; i < n; ++i) {
        if (check_request(reqs[i]) != WV_OK) return WV_ERR_ARG;
        const Geom &g = reqs[i].s->g;
        const TuneKey k{g.wavelet, g.levels, g.p[0].w, g.p[0].h};
        if (std::find(keys.begin(), keys.end(), k) == keys.end()) keys.push_back(k);
    }
    const Shape cand[] = {{128, 128, 64}, {128, 128, 32}, {64, 64, 64}, {64, 64, 32}, {256, 64, 64}, {256, 128, 64}};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return WV_ERR_CUDA;
    int rc = WV_OK;
    const bool timing = b->timing;
    b->timing = false;
    for (const TuneKey &k : keys) {
        float best = 1e30f;
        Shape pick = cand[0];
        for (const auto &c : cand) {
            b->tuned[k] = c;
            rc = run_batch(b, reqs, n, b->cs);   // warm-up (captures the graph)
            if (rc != WV_OK) break;
            cudaEventRecord(e0, b->cs);
            for (int r = 0; r < reps && rc == WV_OK; ++r) rc = run_batch(b, reqs, n, b->cs);
            cudaEventRecord(e1, b->cs);
            if (rc != WV_OK || cudaEventSynchronize(e1) != cudaSuccess) {
                rc = rc != WV_OK ? rc : WV_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                pick = c;
            }
        }
        b->tuned[k] = pick;
        if (rc != WV_OK) break;
    }
    b->timing = timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int wv_decode_batch(const wv_request *reqs, int n, void *cuda_stream) {
    if (n < 0 || (n > 0 && !reqs)) return WV_ERR_ARG;
    if (n == 0) return WV_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return WV_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_default_mutex);
    wv_batch *&b = g_default[dev];
    if (!b) {
        const int rc = wv_batch_create(cuda_stream, &b);
        if (rc != WV_OK) {
            b = nullptr;
            return rc;
        }
    }
    return run_batch(b, reqs, n, (cudaStream_t)cuda_stream);
}

void wv_release_default_batch(void) {
    std::lock_guard<std::mutex> lock(g_default_mutex);
    for (auto &kv : g_default) wv_batch_close(kv.second);
    g_default.clear();
}

}  // extern "C"
