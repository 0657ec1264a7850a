// api.cu -- C ABI of the decoder: stream parsing and upload, decode
// orchestration, inspection hooks and per-kernel event timing.
//
// Stream layout (little endian):
//   header (128 bytes)  magic "WVS1", version 1, luma width/height, planes,
//                       chroma_420, levels, wavelet, num_frames, tlevels,
//                       block, quantiser, step, blocks per frame, number of
//                       stored blocks, byte offsets of table and payload.
//                       (Sec. 3.4: the header gives the number of frames, the
//                       frame size and the number of wavelet levels.)
//   block table         int32 [num_frames][blocks per frame]: slot of the
//                       block's coefficients in the payload, -1 when the block
//                       is all zero (the per-block BlockEnd pointers of Sec.
//                       3.4, here one fixed-size slot per stored block).
//   payload             int16 [slots][block][block], row-major blocks.
// Blocks of one coefficient frame: plane by plane; in each plane LL_L, then
// for l = L..1 the subbands HL_l, LH_l, HH_l (level-wise from the lowest
// frequency, Sec. 3.4), each cut into block x block tiles in row-major order.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "wv_impl.h"

using namespace wv;

namespace {

enum Kernel { kKFootprint = 0, kKTiles = 1, kKCoarse = 2, kKFine = 3, kKResample = 4 };

// Geometry of the stream's viewport and whole-plane decodes in its current
// decode mode: 0 = the default geometry (strip tiles for the streams the
// strip kernel decodes), 1 and 2 = square tiles.
const Geom &active_geom(const wv_stream *s) { return s->decode_mode == 0 ? s->g : s->gsq; }
// Strip fine pass (levels 2 and 1 streamed down strips, strip.cu).
bool strip_mode(const wv_stream *s) { return s->decode_mode == 0 && s->g.strip; }
// Coarse pass (levels L..3 into LL_2 planes) before the fine pass.
bool split_mode(const wv_stream *s) { return s->decode_mode != 1 && s->g.levels >= 3; }

// Coefficient frames of `frame` with the byte quantiser's parameters of the
// paper-faithful format (quant 1).
Bands stream_bands(const wv_stream *s, int frame) {
    Bands b = frame_bands(s->g, frame);
    if (s->g.quant == 1)
        for (int k = 0; k < b.n; ++k)
            for (int p = 0; p < 3; ++p)
                for (int c = 0; c < 2; ++c)
                    for (int e = 0; e < 2; ++e)
                        b.qp[k][p][c][e] = s->qp_host[(((size_t)b.t[k] * 3 + p) * 2 + c) * 2 + e];
    return b;
}

// Generation stamp of the next viewport (0 is never used: the stamp arrays
// start zeroed).
uint32_t next_gen(wv_stream *s) {
    s->gen = s->gen + 1 == 0 ? 1 : s->gen + 1;
    return s->gen;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int parse(const void *bytes, size_t n, wv_stream_desc *d, StreamHeader *h) {
    if (!bytes || n < kHeaderBytes) return WV_ERR_FORMAT;
    memcpy(h, bytes, sizeof(StreamHeader));
    if (memcmp(h->magic, "WVS1", 4) != 0 || h->version != 1) return WV_ERR_FORMAT;
    d->width = (int)h->width;
    d->height = (int)h->height;
    d->planes = (int)h->planes;
    d->chroma_420 = (int)h->c420;
    d->levels = (int)h->levels;
    d->wavelet = (int)h->wavelet;
    d->num_frames = (int)h->num_frames;
    d->tlevels = (int)h->tlevels;
    d->block = (int)h->block;
    d->quant = (int)h->quant;
    d->step = h->step;
    d->stereo = (int)h->reserved0;
    Geom g;
    if (build_geom(*d, &g) != WV_OK) return WV_ERR_FORMAT;
    if ((int)h->nbpf != g.nbpf) return WV_ERR_FORMAT;
    const uint64_t tbytes = (uint64_t)g.num_frames * g.nbpf * 4;
    const uint64_t bsz = (uint64_t)g.block * g.block * 2;
    if (h->table_off < kHeaderBytes || h->table_off + tbytes > n) return WV_ERR_FORMAT;
    if (h->payload_off % 2 || h->payload_off < h->table_off + tbytes) return WV_ERR_FORMAT;
    if (h->n_payload > (n - std::min<uint64_t>(n, h->payload_off)) / bsz) return WV_ERR_FORMAT;
    const int32_t *tab = reinterpret_cast<const int32_t *>((const char *)bytes + h->table_off);
    for (uint64_t i = 0; i < (uint64_t)g.num_frames * g.nbpf; ++i) {
        int32_t s;
        memcpy(&s, tab + i, 4);
        if (s < -1 || (int64_t)s >= (int64_t)h->n_payload) return WV_ERR_FORMAT;
    }
    return WV_OK;
}

// Both geometries of a stream: square tiles always, strip tiles where the
// strip kernel applies (else a copy of the square geometry).
int stream_geoms(const wv_stream_desc &d, uint64_t n_payload, Geom *g, Geom *gsq) {
    const int rc = build_geom(d, gsq);
    if (rc != WV_OK) return rc;
    gsq->n_blocks = (int)std::min<uint64_t>(n_payload, 0x7fffffff);
    if (strip_eligible(d, n_payload)) {
        const int rs = build_geom_strip(d, g);
        g->n_blocks = gsq->n_blocks;
        return rs;
    }
    *g = *gsq;
    return WV_OK;
}

struct Layout {
    size_t payload, table, recon[3], ll2[3], mask, tiles, ctiles, tile_gen, ctile_gen, counters, err;
    size_t ll2_1[3], tiles1, ctiles1, counters1, recon1[3], total;   // the second per-viewport set
};

// Device layout of a stream; tile lists and stamps hold the larger tile count
// of the two geometries.
Layout layout(const Geom &g0, const Geom &gsq, uint64_t n_payload) {
    Geom g = g0;
    g.total_tiles = std::max(g0.total_tiles, gsq.total_tiles);
    // tile lists: an edge strip is listed as two half strips
    const size_t list_tiles = std::max<size_t>(2 * (size_t)g0.total_tiles, gsq.total_tiles);
    Layout L;
    size_t o = 0;
    L.payload = o;
    o = align256(o + n_payload * g.block * g.block * 2);
    L.table = o;
    o = align256(o + (size_t)g.num_frames * g.nbpf * 4);
    for (int p = 0; p < 3; ++p) {
        L.recon[p] = o;
        if (p < g.planes) o = align256(o + (size_t)g.p[p].w * g.p[p].h);
    }
    for (int p = 0; p < 3; ++p) {
        L.ll2[p] = o;
        if (p < g.planes && g.levels >= 3)
            o = align256(o + (size_t)g.p[p].ll2_pitch * (g.p[p].h >> 2) * 4);
    }
    L.mask = o;
    o = align256(o + (size_t)g.cells_x * g.cells_y);
    L.tiles = o;
    o = align256(o + list_tiles * 4);
    L.ctiles = o;
    o = align256(o + (size_t)(g.total_ctiles > 0 ? g.total_ctiles : 1) * 4);
    L.tile_gen = o;
    o = align256(o + (size_t)g.total_tiles * 4);
    L.ctile_gen = o;
    o = align256(o + (size_t)(g.total_ctiles > 0 ? g.total_ctiles : 1) * 4);
    L.counters = o;
    o = align256(o + 64);
    L.err = o;
    o = align256(o + 64);
    for (int p = 0; p < 3; ++p) {
        L.ll2_1[p] = o;
        if (p < g.planes && g.levels >= 3)
            o = align256(o + (size_t)g.p[p].ll2_pitch * (g.p[p].h >> 2) * 4);
    }
    L.tiles1 = o;
    o = align256(o + list_tiles * 4);
    L.ctiles1 = o;
    o = align256(o + (size_t)(g.total_ctiles > 0 ? g.total_ctiles : 1) * 4);
    L.counters1 = o;
    o = align256(o + 64);
    for (int p = 0; p < 3; ++p) {
        L.recon1[p] = o;
        if (p < g.planes) o = align256(o + (size_t)g.p[p].w * g.p[p].h);
    }
    L.total = o;
    return L;
}

int cuda_err(cudaError_t e) { return e == cudaSuccess ? WV_OK : WV_ERR_CUDA; }

std::atomic<int> g_fail_allocs{0};   // device allocations still to fail (test hook)

void prof_begin(wv_stream *s, int kind) {
    if (!s->prof) return;
    if (s->ev_used + 2 > s->ev_pool.size()) {
        for (int i = 0; i < 64; ++i) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            s->ev_pool.push_back(e);
        }
    }
    cudaEventRecord(s->ev_pool[s->ev_used], s->cs);
    s->ev_kind.push_back(kind);
}

void prof_end(wv_stream *s) {
    if (!s->prof) return;
    cudaEventRecord(s->ev_pool[s->ev_used + 1], s->cs);
    s->ev_used += 2;
}

int check_image(const wv_image *o) {
    if (!o || !o->dptr || o->width <= 0 || o->height <= 0 ||
        o->pitch_bytes < (size_t)o->width * 4 || (o->pitch_bytes % 4) != 0 ||
        ((uintptr_t)o->dptr % 4) != 0)
        return WV_ERR_ARG;
    return WV_OK;
}

// Tile decode of the selected tiles: a coarse pass (levels L..3 into LL_2
// planes) followed by a fine pass (levels 2 and 1), or all levels in one
// pass when the stream has fewer than three levels or mode 1 is set.
// The fine pass (levels 2 and 1) of the listed tiles: strips, or square tiles
// reading LL_2 from the planes.
cudaError_t launch_fine(wv_stream *s, const Bands &b, const float *const *ll2, uint8_t *const *out_u8,
                        float *f32, int f32_plane, const uint32_t *tiles, int *counters,
                        cudaStream_t cs) {
    const Geom &g = active_geom(s);
    if (strip_mode(s)) {
        // into the stream's reconstruction planes: chroma in alternating Cb, Cr groups
        const bool own = (out_u8[1] == s->recon[1] && out_u8[2] == s->recon[2]) ||
                         (out_u8[1] == s->recon1[1] && out_u8[2] == s->recon1[2]);
        const bool pairs = own && recon_pairs(s);
        uint8_t *const outs[3] = {out_u8[0], out_u8[1], pairs ? out_u8[1] + 4 : out_u8[2]};
        return launch_decode_strips(g, s->payload, s->table, b, ll2, s->ll2_pitch, outs, f32, f32_plane, tiles,
                                    counters, s->err, cs, pairs);
    }
    return launch_decode_fine(g, s->payload, s->table, b, ll2, s->ll2_pitch, out_u8, f32, f32_plane, tiles,
                              counters, s->err, cs);
}

cudaError_t run_decode(wv_stream *s, const Bands &b, uint8_t *const *out_u8, float *f32,
                       int f32_plane) {
    const Geom &g = active_geom(s);
    cudaError_t e;
    if (split_mode(s)) {
        prof_begin(s, kKCoarse);
        e = launch_decode_coarse(g, s->payload, s->table, b, s->ll2, s->ll2_pitch, s->ctiles,
                                 s->counters + 1, s->err, s->cs);
        prof_end(s);
        if (e != cudaSuccess) return e;
        const float *ll2c[3] = {s->ll2[0], s->ll2[1], s->ll2[2]};
        prof_begin(s, kKFine);
        e = launch_fine(s, b, ll2c, out_u8, f32, f32_plane, s->tiles, s->counters, s->cs);
        prof_end(s);
        return e;
    }
    prof_begin(s, kKFine);
    e = launch_decode_tiles(g, s->payload, s->table, b, out_u8, f32, f32_plane, s->tiles, s->counters, s->err,
                            s->cs);
    prof_end(s);
    return e;
}

}  // namespace

namespace wv {

// Steps 1-3 of a viewport decode: footprint, tile lists and the tile decode
// of the region an out_w x out_h viewport reads (into the stream's
// reconstruction planes).
int eye_view(const Geom &g, int eye, int *row0, int *rows) {
    if (eye < 0 || eye > (g.stereo ? 1 : 0)) return WV_ERR_ARG;
    *rows = g.stereo ? g.p[0].h / 2 : g.p[0].h;
    *row0 = eye * *rows;
    return WV_OK;
}

// The internal stream and events of the overlapped viewport path (created on
// first use; the stream has the highest priority so that its small kernels
// take SMs as soon as the running fine pass or resampling frees them).
cudaError_t ensure_aux(wv_stream *s) {
    if (s->aux) return cudaSuccess;
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->aux, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->fs, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&s->ev_ready[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_fine[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_free[k], cudaEventDisableTiming);
    }
    return e;
}

// A stream that is ever captured into a CUDA graph decodes serially from
// then on: the internal stream is not part of a capture, and graph replays
// must not race with overlapped calls.
void check_capture(wv_stream *s) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s->cs, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        s->overlap = false;
    }
}

// After work on cs that used the per-viewport buffers of set 0 (or both):
// later overlapped viewports wait for it before reusing either set.
void mark_sets_used(wv_stream *s) {
    check_capture(s);
    if (!s->aux || !s->overlap) return;
    cudaEventRecord(s->ev_free[0], s->cs);
    cudaEventRecord(s->ev_free[1], s->cs);
}

// Overlapped viewport decode into buffer set k, three stages on three
// streams: footprint, selection and coarse pass on aux (once the fine pass
// of two viewports ago and every cs use of set k are done), the fine pass
// into set k's reconstruction on fs (once the coarse pass is done and the
// resampling of two viewports ago has read that reconstruction), and cs
// waits for the fine pass; the caller's resampling then runs on cs while
// the next viewport's fine pass writes the other set.
int decode_region_overlapped(wv_stream *s, const View &v, const Bands &b, uint32_t gen) {
    const Geom &g = active_geom(s);
    const int k = s->slot;
    s->slot ^= 1;
    uint32_t *tiles = k ? s->tiles1 : s->tiles, *ctiles = k ? s->ctiles1 : s->ctiles;
    int *counters = k ? s->counters1 : s->counters;
    float *ll2[3] = {k ? s->ll2_1[0] : s->ll2[0], k ? s->ll2_1[1] : s->ll2[1], k ? s->ll2_1[2] : s->ll2[2]};
    uint8_t *const *recon = k ? s->recon1 : s->recon;
    cudaError_t e = cudaStreamWaitEvent(s->aux, s->ev_fine[k], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->aux, s->ev_free[k], 0);
    if (e != cudaSuccess) return WV_ERR_CUDA;
    launch_footprint(g, v, s->mask, s->tile_gen, s->ctile_gen, gen, counters, s->aux);
    launch_select_tiles(g, s->tile_gen, s->ctile_gen, gen, tiles, ctiles, counters, s->aux);
    e = launch_decode_coarse(g, s->payload, s->table, b, ll2, s->ll2_pitch, ctiles, counters + 1, s->err, s->aux);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev_ready[k], s->aux);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->fs, s->ev_ready[k], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->fs, s->ev_free[k], 0);
    const float *ll2c[3] = {ll2[0], ll2[1], ll2[2]};
    if (e == cudaSuccess) e = launch_fine(s, b, ll2c, recon, nullptr, -1, tiles, counters, s->fs);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev_fine[k], s->fs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->cs, s->ev_fine[k], 0);
    s->cur = k;
    s->pending = true;
    return e == cudaSuccess ? WV_OK : WV_ERR_CUDA;
}

int decode_region(wv_stream *s, int frame, float yaw, float pitch, float fov, int out_w, int out_h, int eye) {
    const Geom &g = active_geom(s);
    int row0, rows;
    if (eye_view(g, eye, &row0, &rows) != WV_OK) return WV_ERR_ARG;
    const View v = make_view(yaw, pitch, fov, out_w, out_h, g.p[0].w, rows, row0);
    const Bands b = stream_bands(s, frame);
    const uint32_t gen = next_gen(s);
    check_capture(s);
    if (split_mode(s) && !s->prof && s->overlap && ensure_aux(s) == cudaSuccess)
        return decode_region_overlapped(s, v, b, gen);
    prof_begin(s, kKFootprint);
    launch_footprint(g, v, s->mask, s->tile_gen, s->ctile_gen, gen, s->counters, s->cs);
    prof_end(s);
    prof_begin(s, kKTiles);
    launch_select_tiles(g, s->tile_gen, s->ctile_gen, gen, s->tiles, s->ctiles, s->counters, s->cs);
    prof_end(s);
    const cudaError_t e = run_decode(s, b, s->recon, nullptr, -1);
    mark_sets_used(s);
    s->cur = 0;
    s->pending = true;
    return e == cudaSuccess ? WV_OK : WV_ERR_CUDA;
}

uint8_t *const *recon_planes(const wv_stream *s) { return s->cur ? s->recon1 : s->recon; }

void release_recon(wv_stream *s, bool again) {
    if (!s->pending && !again) return;
    s->pending = false;
    if (s->aux && s->overlap) cudaEventRecord(s->ev_free[s->cur], s->cs);
}

}  // namespace wv

namespace {

int decode_viewport(wv_stream *s, int frame, float yaw, float pitch, float fov,
                    const wv_image *out, int eye = 0) {
    if (!s) return WV_ERR_ARG;
    if (frame < 0 || frame >= s->g.num_frames) return WV_ERR_ARG;
    if (!(fov > 0.f && fov < 3.14159f) || !isfinite(yaw) || !isfinite(pitch)) return WV_ERR_ARG;
    if (check_image(out) != WV_OK) return WV_ERR_ARG;
    const Geom &g = s->g;
    int row0, rows;
    if (eye_view(g, eye, &row0, &rows) != WV_OK) return WV_ERR_ARG;
    const int rc = wv::decode_region(s, frame, yaw, pitch, fov, out->width, out->height, eye);
    if (rc != WV_OK) return rc;
    const View v = make_view(yaw, pitch, fov, out->width, out->height, g.p[0].w, rows, row0);
    prof_begin(s, kKResample);
    launch_resample(g, v, recon_planes(s), nullptr, (uint8_t *)out->dptr, out->pitch_bytes, s->cs, nullptr,
                    nullptr, nullptr, recon_pairs(s), s->err);
    prof_end(s);
    release_recon(s);
    return cuda_err(cudaGetLastError());
}

// ---- host-side dependency cone (accounting only) ----

void dilate_axis(const std::vector<uint8_t> &in, std::vector<uint8_t> &out, int w, int h,
                 bool along_x, int wavelet) {
    out.assign(in.size(), 0);
    const int n = along_x ? w : h;
    auto refl = [n](int i) {
        if (n == 1) return 0;
        const int period = 2 * (n - 1);
        i %= period;
        if (i < 0) i += period;
        return i >= n ? period - i : i;
    };
    // synthesis output i reads interleaved inputs i-3..i+3 (even i) or i-4..i+4
    // (odd i) for 9/7, i-1..i+1 or i-2..i+2 for 5/3
    const int se = wavelet == WV_WAVELET_97 ? 3 : 1;
    const int so = wavelet == WV_WAVELET_97 ? 4 : 2;
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            if (!in[(size_t)y * w + x]) continue;
            const int i = along_x ? x : y;
            const int r = (i & 1) ? so : se;
            for (int o = -r; o <= r; ++o) {
                const int j = refl(i + o);
                if (along_x) out[(size_t)y * w + j] = 1;
                else out[(size_t)j * w + x] = 1;
            }
        }
    }
}

// fbits: optional foveation bits per mask cell (bit l - 1 keeps the details
// of level l = 1, 2); dropped coefficients are not read.
unsigned long long cone_bytes(const wv_stream *s, int frame, const uint8_t *mask,
                              const uint8_t *fbits = nullptr, unsigned long long *fine_part = nullptr) {
    const Geom &g = s->g;
    const Bands b = frame_bands(g, frame);
    unsigned long long total = 0, fine = 0;
    for (int p = 0; p < g.planes; ++p) {
        const PlaneGeom &pg = g.p[p];
        int w = pg.w, h = pg.h;
        const int cell = kCell / pg.sub;
        std::vector<uint8_t> R((size_t)w * h), X, tmp;
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x)
                R[(size_t)y * w + x] = mask[(size_t)(y / cell) * g.cells_x + x / cell] ? 1 : 0;
        auto count = [&](int level, int sub, int kx, int ky) {
            if (fbits && level <= 2 && sub != 0) {
                const int X = (kx << level) * pg.sub, Y = (ky << level) * pg.sub;
                if (!((fbits[(size_t)(Y / kCell) * g.cells_x + X / kCell] >> (level - 1)) & 1)) return;
            }
            const int bid = pg.base[level][sub] + (ky >> g.log2b) * pg.nbx[level] + (kx >> g.log2b);
            for (int k = 0; k < b.n; ++k)
                if (s->table_host[(size_t)b.t[k] * g.nbpf + bid] >= 0) {
                    total += 2;
                    if (level <= 2 && (sub != 0 || level < g.levels || g.levels <= 2)) fine += 2;
                }
        };
        for (int l = 1; l <= g.levels; ++l) {
            dilate_axis(R, tmp, w, h, true, g.wavelet);
            dilate_axis(tmp, X, w, h, false, g.wavelet);
            std::vector<uint8_t> next((size_t)(w / 2) * (h / 2));
            for (int y = 0; y < h; ++y)
                for (int x = 0; x < w; ++x) {
                    if (!X[(size_t)y * w + x]) continue;
                    const int sub = (x & 1) + 2 * (y & 1);
                    if (sub == 0) next[(size_t)(y >> 1) * (w / 2) + (x >> 1)] = 1;
                    else count(l, sub, x >> 1, y >> 1);
                }
            R.swap(next);
            w /= 2;
            h /= 2;
        }
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x)
                if (R[(size_t)y * w + x]) count(g.levels, 0, x, y);
    }
    if (fine_part) *fine_part = fine;
    return total;
}

// Foveation bits of every mask cell in double precision (the same definition
// as the device footprint: cell centre direction, viewer angles, max norm).
void fovea_bits_host(const Geom &g, double yaw, double pitch, const wv_request &r,
                     std::vector<uint8_t> &out) {
    const double pi = 3.14159265358979323846;
    const double cy = cos(yaw), sy = sin(yaw), cp = cos(pitch), sp = sin(pitch);
    const double R[9] = {cy, -sy * sp, sy * cp, 0.0, cp, sp, -sy, -cy * sp, cy * cp};
    out.assign((size_t)g.cells_x * g.cells_y, 0);
    for (int j = 0; j < g.cells_y; ++j)
        for (int i = 0; i < g.cells_x; ++i) {
            const double lon = 2.0 * pi * ((i + 0.5) * kCell / g.p[0].w - 0.5);
            const double lat = pi * (0.5 - (j + 0.5) * kCell / g.p[0].h);
            const double d[3] = {cos(lat) * sin(lon), sin(lat), cos(lat) * cos(lon)};
            const double x = R[0] * d[0] + R[3] * d[1] + R[6] * d[2];
            const double y = R[1] * d[0] + R[4] * d[1] + R[7] * d[2];
            const double z = R[2] * d[0] + R[5] * d[1] + R[8] * d[2];
            if (!(z > 0.0)) continue;
            const double dist = std::max(fabs(atan2(x, z) - r.gaze_x), fabs(atan2(y, z) - r.gaze_y));
            out[(size_t)j * g.cells_x + i] = (uint8_t)((dist <= r.r1 ? 1 : 0) | (dist <= r.r2 ? 2 : 0));
        }
}

}  // namespace

// ---------------------------------------------------------------------------
// geometry helpers
// ---------------------------------------------------------------------------

namespace wv {

cudaError_t dev_alloc(void **p, size_t bytes) {
    int n = g_fail_allocs.load();
    while (n > 0) {
        if (g_fail_allocs.compare_exchange_weak(n, n - 1)) return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t opt_in_smem(const void *fn, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> opted;   // (kernel, device) -> bytes set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    int &have = opted[std::make_pair(fn, dev)];
    if (bytes <= have) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

bool recon_pairs(const wv_stream *s) { return s->pair_ok && s->decode_mode == 0 && s->g.strip; }

namespace {

// Common geometry of both tile organisations: output tiles tw x th (plane
// pixels, multiples of the 32-pixel mask cell, and of 16 chroma pixels) and
// coarse tiles of ctile LL_2 samples.
int build_geom_tiles(const wv_stream_desc &d, Geom *g, int tw, int th, int strip, int ctile) {
    memset(g, 0, sizeof(*g));
    if (tw % kCell || th % kCell || tw <= 0 || th <= 0 || (ctile != 32 && ctile != 64)) return WV_ERR_ARG;
    if (d.planes != 1 && d.planes != 3) return WV_ERR_ARG;
    if (d.chroma_420 != 0 && d.chroma_420 != 1) return WV_ERR_ARG;
    if (d.levels < 1 || d.levels > kMaxLevels) return WV_ERR_ARG;
    if (d.wavelet != WV_WAVELET_53 && d.wavelet != WV_WAVELET_97) return WV_ERR_ARG;
    if (d.tlevels < 0 || d.tlevels > kMaxBands - 1) return WV_ERR_ARG;
    if (d.num_frames < 1 || d.num_frames % (1 << d.tlevels)) return WV_ERR_ARG;
    if (d.block < 16 || d.block > 256 || (d.block & (d.block - 1))) return WV_ERR_ARG;
    if (d.quant != 0 && d.quant != 1) return WV_ERR_ARG;
    if (d.quant == 1 && (d.wavelet != WV_WAVELET_97 || d.block != 32)) return WV_ERR_ARG;
    if (!(d.step > 0.f) || !isfinite(d.step)) return WV_ERR_ARG;
    if (d.wavelet == WV_WAVELET_53 && (d.step != floorf(d.step) || d.step > 65536.f))
        return WV_ERR_ARG;
    if (d.width < 2 || d.height < 2 || d.width > 16384 || d.height > 16384) return WV_ERR_ARG;
    if (d.stereo != 0 && d.stereo != 1) return WV_ERR_ARG;
    if (d.stereo && d.height % (2 * kCell)) return WV_ERR_ARG;
    if (d.width % kCell || d.height % kCell) return WV_ERR_ARG;
    g->planes = d.planes;
    g->c420 = d.planes == 3 ? d.chroma_420 : 0;
    g->levels = d.levels;
    g->wavelet = d.wavelet;
    g->num_frames = d.num_frames;
    g->tlevels = d.tlevels;
    g->block = d.block;
    g->log2b = 0;
    while ((1 << g->log2b) < d.block) ++g->log2b;
    g->step = d.step;
    g->quant = d.quant;
    g->stereo = d.stereo;
    g->cells_x = d.width / kCell;
    g->cells_y = d.height / kCell;
    g->tw = tw;
    g->th = th;
    g->strip = strip;
    g->ctile = ctile;
    // LL_2 window of an output tile: the square tile kernel's fine pass reads
    // its LL_2 window q t - 3 .. q t + q + 2 (q = tile / 4, the 9/7 halo of
    // two levels); a strip's level-2 lanes read LL_2 columns X0/4 - 4 ..
    // X0/4 + 59 and its level-2 row pairs LL_2 rows Y0/4 - 3 .. Y0/4 + th/4 + 2
    g->wx0 = strip ? -4 : -3;
    g->wx1 = strip ? 59 : tw / 4 + 2;
    g->wy0 = -3;
    g->wy1 = th / 4 + 2;
    int id = 0;
    g->total_tiles = 0;
    g->total_ctiles = 0;
    for (int p = 0; p < d.planes; ++p) {
        PlaneGeom &pg = g->p[p];
        pg.sub = (p > 0 && g->c420) ? 2 : 1;
        pg.w = d.width / pg.sub;
        pg.h = d.height / pg.sub;
        if (pg.w % (1 << d.levels) || pg.h % (1 << d.levels)) return WV_ERR_ARG;
        if ((pg.w >> d.levels) < 2 || (pg.h >> d.levels) < 2) return WV_ERR_ARG;
        for (int l = 1; l <= d.levels; ++l) {
            const int sw = pg.w >> l, sh = pg.h >> l;
            pg.nbx[l] = (sw + d.block - 1) / d.block;
            pg.nby[l] = (sh + d.block - 1) / d.block;
        }
        const int L = d.levels;
        pg.base[L][0] = id;
        id += pg.nbx[L] * pg.nby[L];
        for (int l = L; l >= 1; --l)
            for (int s = 1; s <= 3; ++s) {
                pg.base[l][s] = id;
                id += pg.nbx[l] * pg.nby[l];
            }
        pg.tiles_x = (pg.w + tw - 1) / tw;
        pg.tiles_y = (pg.h + th - 1) / th;
        g->total_tiles += pg.tiles_x * pg.tiles_y;
        pg.ll2_pitch = (((pg.w >> 2) + 7) / 8) * 8;
        if (d.levels >= 3) {
            pg.ctiles_x = ((pg.w >> 2) + ctile - 1) / ctile;
            pg.ctiles_y = ((pg.h >> 2) + ctile - 1) / ctile;
        }
        g->total_ctiles += pg.ctiles_x * pg.ctiles_y;
    }
    g->nbpf = id;
    return WV_OK;
}

}  // namespace

int build_geom(const wv_stream_desc &d, Geom *g, int tile, int ctile) {
    if (tile != 64 && tile != 128) {
        memset(g, 0, sizeof(*g));
        return WV_ERR_ARG;
    }
    return build_geom_tiles(d, g, tile, tile, 0, ctile);
}

int build_geom_rect(const wv_stream_desc &d, Geom *g, int tw, int th, int ctile) {
    if (tw < 64 || tw > 256 || th < 64 || th > 256) {
        memset(g, 0, sizeof(*g));
        return WV_ERR_ARG;
    }
    return build_geom_tiles(d, g, tw, th, 0, ctile);
}

// The strip kernel decodes levels 2 and 1 of dead-zone streams of three or
// more levels (LL_2 from the coarse pass; taking it from the LL band of
// two-level streams in the same loop cost 5 % in spilled registers) and
// addresses the payload with 32-bit element offsets.
bool strip_eligible(const wv_stream_desc &d, uint64_t n_payload) {
    return d.levels >= 3 && d.quant == 0 &&
           n_payload * (uint64_t)d.block * (uint64_t)d.block < (1ull << 32);
}

int build_geom_strip(const wv_stream_desc &d, Geom *g, int th, int ctile) {
    if (th % kCell || th < 32 || th > 256) {
        memset(g, 0, sizeof(*g));
        return WV_ERR_ARG;
    }
    return build_geom_tiles(d, g, kStripW, th, 1, ctile);
}

Bands frame_bands(const Geom &g, int frame) {
    Bands b;
    memset(&b, 0, sizeof(b));
    const int k = g.tlevels, n = 1 << k;
    const int set = frame / n, fl = frame % n;
    b.n = 1 + k;
    b.t[0] = set * n;
    b.bit[0] = 0;
    int idx = 1;
    for (int j = k; j >= 1; --j, ++idx) {
        b.t[idx] = set * n + (1 << (k - j)) + (fl >> j);
        b.bit[idx] = (fl >> (j - 1)) & 1;
    }
    for (; idx < kMaxBands; ++idx) {
        b.t[idx] = 0;
        b.bit[idx] = 0;
    }
    return b;
}

Frustum make_frustum(const View &v) {
    // camera-space normals of x <= T z, x >= -T z, y <= T z, y >= -T z
    const double T = v.t, nrm = 1.0 / sqrt(1.0 + T * T);
    const double m[4][3] = {{-nrm, 0.0, T * nrm}, {nrm, 0.0, T * nrm},
                            {0.0, -nrm, T * nrm}, {0.0, nrm, T * nrm}};
    Frustum f;
    for (int k = 0; k < 4; ++k)
        for (int i = 0; i < 3; ++i)
            f.n[k][i] = (float)(v.r[3 * i + 0] * m[k][0] + v.r[3 * i + 1] * m[k][1] +
                                v.r[3 * i + 2] * m[k][2]);
    return f;
}

View make_view(float yaw, float pitch, float fov, int out_w, int out_h, int eq_w, int eq_h, int row0) {
    const double cy = cos((double)yaw), sy = sin((double)yaw);
    const double cp = cos((double)pitch), sp = sin((double)pitch);
    // R = R_y(yaw) R_x(pitch); R_x: (x, y, z) -> (x, y cp + z sp, -y sp + z cp)
    const double R[9] = {cy, -sy * sp, sy * cp,
                         0.0, cp, sp,
                         -sy, -cy * sp, cy * cp};
    View v;
    for (int i = 0; i < 9; ++i) v.r[i] = (float)R[i];
    v.t = (float)tan((double)fov / 2.0);
    v.sx = (float)(2.0 / out_w);
    v.sy = (float)(2.0 / out_h);
    const double pi = 3.14159265358979323846;
    v.ku = (float)(eq_w / (2.0 * pi));
    v.cu = (float)(0.5 * eq_w - 0.5);
    v.kv = (float)(-eq_h / pi);
    v.cv = (float)(0.5 * eq_h - 0.5 + row0);
    v.out_w = out_w;
    v.out_h = out_h;
    v.row0 = row0;
    v.rows = eq_h;
    return v;
}

}  // namespace wv

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

const char *wv_strerror(int code) {
    switch (code) {
    case WV_OK: return "ok";
    case WV_ERR_ARG: return "invalid argument";
    case WV_ERR_FORMAT: return "malformed or unsupported stream";
    case WV_ERR_OOM: return "out of memory or buffer too small";
    case WV_ERR_CUDA: return "CUDA error or no CUDA device";
    case WV_ERR_RANGE: return "value out of range";
    case WV_ERR_TIMEOUT: return "device wait timed out";
    case WV_ERR_DEVICE: return "kernel reported an inconsistency";
    default: return "unknown error";
    }
}

int wv_stream_query(const void *bytes, size_t n, wv_stream_desc *desc, size_t *device_bytes) {
    return wv_stream_query_ex(bytes, n, 0, desc, device_bytes);
}

int wv_stream_query_ex(const void *bytes, size_t n, int flags, wv_stream_desc *desc, size_t *device_bytes) {
    if (flags & ~WV_OPEN_HOST_PAYLOAD) return WV_ERR_ARG;
    const bool host_payload = (flags & WV_OPEN_HOST_PAYLOAD) != 0;
    wv_stream_desc d;
    StreamHeader h;
    if (is_paper_stream(bytes, n)) {
        PaperInfo info;
        const int rc = paper_parse(bytes, n, &d, &info);
        if (rc != WV_OK) return rc;
        if (desc) *desc = d;
        if (device_bytes) {
            Geom g, gsq;
            stream_geoms(d, info.n_slots, &g, &gsq);
            *device_bytes = layout(g, gsq, host_payload ? 0 : info.n_slots).total;
        }
        return WV_OK;
    }
    const int rc = parse(bytes, n, &d, &h);
    if (rc != WV_OK) return rc;
    if (desc) *desc = d;
    if (device_bytes) {
        Geom g, gsq;
        stream_geoms(d, h.n_payload, &g, &gsq);
        *device_bytes = layout(g, gsq, host_payload ? 0 : h.n_payload).total;
    }
    return WV_OK;
}

int wv_open_stream(const void *bytes, size_t n, void *device_mem, size_t device_bytes,
                   void *cuda_stream, wv_stream **out) {
    return wv_open_stream_ex(bytes, n, device_mem, device_bytes, cuda_stream, 0, out);
}

int wv_open_stream_ex(const void *bytes, size_t n, void *device_mem, size_t device_bytes,
                      void *cuda_stream, int flags, wv_stream **out) {
    if (!out) return WV_ERR_ARG;
    *out = nullptr;
    if (flags & ~WV_OPEN_HOST_PAYLOAD) return WV_ERR_ARG;
    const bool host_payload = (flags & WV_OPEN_HOST_PAYLOAD) != 0;
    wv_stream_desc d;
    StreamHeader h;
    PaperInfo paper;
    const bool is_paper = is_paper_stream(bytes, n);
    int rc = is_paper ? paper_parse(bytes, n, &d, &paper) : parse(bytes, n, &d, &h);
    if (rc != WV_OK) return rc;
    if (is_paper) {
        memset(&h, 0, sizeof(h));
        h.n_payload = paper.n_slots;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return WV_ERR_CUDA;
    wv_stream *s = new (std::nothrow) wv_stream();
    if (!s) return WV_ERR_OOM;
    stream_geoms(d, h.n_payload, &s->g, &s->gsq);
    s->desc = d;
    cudaGetDevice(&s->device);
    s->cs = (cudaStream_t)cuda_stream;
    s->n_payload = h.n_payload;
    const Layout L = layout(s->g, s->gsq, host_payload ? 0 : h.n_payload);
    const size_t payload_bytes = (size_t)h.n_payload * s->g.block * s->g.block * 2;
    if (host_payload && payload_bytes) {
        // the coefficient store in pinned, device-mapped host memory: the
        // tile decoder reads the blocks a viewport needs from there (on a
        // Grace-Blackwell node over NVLink-C2C) instead of an HBM copy
        if (cudaHostAlloc(&s->host_payload, payload_bytes, cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return WV_ERR_OOM;
        }
        void *dp = nullptr;
        if (cudaHostGetDevicePointer(&dp, s->host_payload, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeHost(s->host_payload);
            delete s;
            return WV_ERR_CUDA;
        }
        s->payload = (int16_t *)dp;
    }
    if (device_mem) {
        if (device_bytes < L.total || ((uintptr_t)device_mem % 256)) {
            if (s->host_payload) cudaFreeHost(s->host_payload);
            delete s;
            return WV_ERR_OOM;
        }
        s->dmem = device_mem;
    } else {
        if (dev_alloc(&s->dmem, L.total) != cudaSuccess) {
            cudaGetLastError();
            if (s->host_payload) cudaFreeHost(s->host_payload);
            delete s;
            return WV_ERR_OOM;
        }
        s->owns = true;
    }
    s->dbytes = L.total;
    char *base = (char *)s->dmem;
    if (!host_payload) s->payload = (int16_t *)(base + L.payload);
    s->table = (int32_t *)(base + L.table);
    for (int p = 0; p < 3; ++p) s->recon[p] = p < s->g.planes ? (uint8_t *)(base + L.recon[p]) : nullptr;
    for (int p = 0; p < 3; ++p) s->recon1[p] = p < s->g.planes ? (uint8_t *)(base + L.recon1[p]) : nullptr;
    s->pair_ok = s->g.planes == 3 && L.recon[2] == L.recon[1] + (size_t)s->g.p[1].w * s->g.p[1].h &&
                 L.recon1[2] == L.recon1[1] + (size_t)s->g.p[1].w * s->g.p[1].h;
    s->mask = (uint8_t *)(base + L.mask);
    s->tiles = (uint32_t *)(base + L.tiles);
    s->ctiles = (uint32_t *)(base + L.ctiles);
    s->tile_gen = (uint32_t *)(base + L.tile_gen);
    s->ctile_gen = (uint32_t *)(base + L.ctile_gen);
    for (int p = 0; p < 3; ++p) {
        const bool has = p < s->g.planes && s->g.levels >= 3;
        s->ll2[p] = has ? (float *)(base + L.ll2[p]) : nullptr;
        s->ll2_pitch[p] = has ? s->g.p[p].ll2_pitch : 0;
    }
    s->counters = (int *)(base + L.counters);
    s->err = (int *)(base + L.err);
    for (int p = 0; p < 3; ++p) s->ll2_1[p] = s->ll2[p] ? (float *)(base + L.ll2_1[p]) : nullptr;
    s->tiles1 = (uint32_t *)(base + L.tiles1);
    s->ctiles1 = (uint32_t *)(base + L.ctiles1);
    s->counters1 = (int *)(base + L.counters1);
    const size_t tcount = (size_t)s->g.num_frames * s->g.nbpf;
    s->table_host.resize(tcount);
    if (is_paper) {
        memcpy(s->table_host.data(), paper.table.data(), tcount * 4);
        s->qp_host = paper.qp;
    } else {
        memcpy(s->table_host.data(), (const char *)bytes + h.table_off, tcount * 4);
    }
    cudaError_t e = cudaMemcpyAsync(s->table, s->table_host.data(), tcount * 4,
                                    cudaMemcpyHostToDevice, s->cs);
    if (e == cudaSuccess && is_paper)
        e = paper_transcode(bytes, n, paper, s->payload, s->cs);
    else if (e == cudaSuccess && h.n_payload && host_payload)
        memcpy(s->host_payload, (const char *)bytes + h.payload_off, payload_bytes);
    else if (e == cudaSuccess && h.n_payload)
        e = cudaMemcpyAsync(s->payload, (const char *)bytes + h.payload_off, payload_bytes,
                            cudaMemcpyHostToDevice, s->cs);
    // 9/7 dead-zone codes become t = 2q + sign(q) on the device when every
    // |q| <= kDzTMax (the tile decoder then needs no sign logic)
    if (e == cudaSuccess && !is_paper && h.n_payload && s->g.wavelet == WV_WAVELET_97 && s->g.quant == 0) {
        const size_t count = (size_t)h.n_payload * s->g.block * s->g.block;
        int max_abs = 0;
        e = cudaMemsetAsync(s->counters + 8, 0, 4, s->cs);
        if (e == cudaSuccess) e = payload_max_abs(s->payload, count, s->counters + 8, s->cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&max_abs, s->counters + 8, 4, cudaMemcpyDeviceToHost, s->cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->cs);
        if (e == cudaSuccess && max_abs <= kDzTMax) {
            e = payload_to_deadzone_t(s->payload, count, s->cs);
            s->g.dz_t = 1;
            s->gsq.dz_t = 1;
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(base + L.recon[0], 0, L.tiles - L.recon[0], s->cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + L.recon1[0], 0, L.total - L.recon1[0], s->cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + L.tile_gen, 0, L.err + 64 - L.tile_gen, s->cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + L.ll2_1[0], 0, L.total - L.ll2_1[0], s->cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        wv_close_stream(s);
        return WV_ERR_CUDA;
    }
    *out = s;
    return WV_OK;
}

void wv_debug_fail_device_allocs(int n) { g_fail_allocs.store(n > 0 ? n : 0); }

int wv_set_cuda_stream(wv_stream *s, void *cuda_stream) {
    if (!s) return WV_ERR_ARG;
    s->cs = (cudaStream_t)cuda_stream;
    return WV_OK;
}

void wv_close_stream(wv_stream *s) {
    if (!s) return;
    cudaStreamSynchronize(s->cs);
    if (s->aux) {
        cudaStreamSynchronize(s->aux);
        cudaStreamDestroy(s->aux);
    }
    if (s->fs) {
        cudaStreamSynchronize(s->fs);
        cudaStreamDestroy(s->fs);
    }
    for (cudaEvent_t e : {s->ev_fine[0], s->ev_fine[1]})
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : {s->ev_ready[0], s->ev_ready[1], s->ev_free[0], s->ev_free[1]})
        if (e) cudaEventDestroy(e);
    if (s->host_payload) cudaFreeHost(s->host_payload);
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    if (s->owns && s->dmem) cudaFree(s->dmem);
    delete s;
}

int wv_decode_viewport(wv_stream *s, int frame, float yaw, float pitch, float fov,
                       const wv_image *out) {
    return decode_viewport(s, frame, yaw, pitch, fov, out);
}

int wv_decode_viewport_eye(wv_stream *s, int frame, int eye, float yaw, float pitch, float fov,
                           const wv_image *out) {
    return decode_viewport(s, frame, yaw, pitch, fov, out, eye);
}

int wv_decode_full(wv_stream *s, int frame, int plane, void *dptr, int as_float) {
    if (!s || frame < 0 || frame >= s->g.num_frames || plane < 0 || plane >= s->g.planes)
        return WV_ERR_ARG;
    if (!dptr && as_float) return WV_ERR_ARG;
    // the strip fine pass writes 8-bit samples only: float output runs the
    // square-tile passes (the same arithmetic per sample)
    struct ModeGuard {
        wv_stream *s;
        int saved;
        ~ModeGuard() { s->decode_mode = saved; }
    } guard{s, s->decode_mode};
    if (as_float && strip_mode(s)) s->decode_mode = 2;
    const Geom &g = active_geom(s);
    uint8_t *outs[3] = {s->recon[0], s->recon[1], s->recon[2]};
    float *f32 = nullptr;
    if (dptr) {
        if (as_float) f32 = (float *)dptr;
        else outs[plane] = (uint8_t *)dptr;
    }
    launch_all_tiles(g, plane, s->tiles, s->counters, s->cs);
    if (split_mode(s)) launch_all_ctiles(g, plane, s->ctiles, s->counters, s->cs);
    cudaError_t e = run_decode(s, stream_bands(s, frame), outs, f32, as_float ? plane : -1);
    mark_sets_used(s);
    if (!dptr) {   // set 0's reconstruction now holds the decode (for wv_resample_at)
        s->cur = 0;
        s->pending = true;
    }
    if (e != cudaSuccess) return WV_ERR_CUDA;
    return cuda_err(cudaGetLastError());
}

int wv_stream_sync_status(wv_stream *s) {
    if (!s) return WV_ERR_ARG;
    if (cudaStreamSynchronize(s->cs) != cudaSuccess) return WV_ERR_CUDA;
    int err = 0;
    if (cudaMemcpy(&err, s->err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return WV_ERR_CUDA;
    if (err) cudaMemset(s->err, 0, 4);
    return err;
}

int wv_debug_footprint(wv_stream *s, float yaw, float pitch, float fov, int out_w, int out_h,
                       uint8_t *mask_host, int *tiles) {
    if (!s || out_w <= 0 || out_h <= 0 || !(fov > 0.f && fov < 3.14159f)) return WV_ERR_ARG;
    const Geom &g = active_geom(s);
    int row0, rows;
    eye_view(g, 0, &row0, &rows);
    const View v = make_view(yaw, pitch, fov, out_w, out_h, g.p[0].w, rows, row0);
    uint8_t *m = s->mask;
    const uint32_t gen = next_gen(s);
    launch_footprint(g, v, m, s->tile_gen, s->ctile_gen, gen, s->counters, s->cs);
    launch_select_tiles(g, s->tile_gen, s->ctile_gen, gen, s->tiles, s->ctiles, s->counters, s->cs);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && mask_host)
        e = cudaMemcpyAsync(mask_host, m, (size_t)g.cells_x * g.cells_y, cudaMemcpyDeviceToHost, s->cs);
    int cnt = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, s->counters, 4, cudaMemcpyDeviceToHost, s->cs);
    mark_sets_used(s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->cs);
    if (tiles) *tiles = cnt;
    return cuda_err(e);
}

int wv_debug_project(wv_stream *s, float yaw, float pitch, float fov, int out_w, int out_h,
                     float *uv_dev) {
    if (!s || !uv_dev || out_w <= 0 || out_h <= 0 || !(fov > 0.f && fov < 3.14159f))
        return WV_ERR_ARG;
    int row0, rows;
    eye_view(s->g, 0, &row0, &rows);
    const View v = make_view(yaw, pitch, fov, out_w, out_h, s->g.p[0].w, rows, row0);
    launch_project(v, uv_dev, s->cs);
    return cuda_err(cudaGetLastError());
}

int wv_resample_at(wv_stream *s, const float *uv_dev, const wv_image *out) {
    if (!s || !uv_dev || check_image(out) != WV_OK) return WV_ERR_ARG;
    View v = make_view(0.f, 0.f, 1.f, out->width, out->height, s->g.p[0].w, s->g.p[0].h);
    launch_resample(s->g, v, recon_planes(s), uv_dev, (uint8_t *)out->dptr, out->pitch_bytes, s->cs, nullptr,
                    nullptr, nullptr, recon_pairs(s), s->err);
    release_recon(s, true);   // any number of reads of the last decode: each releases its set again
    return cuda_err(cudaGetLastError());
}

int wv_cone_bytes(wv_stream *s, int frame, const uint8_t *mask_host, unsigned long long *bytes) {
    if (!s || !mask_host || !bytes || frame < 0 || frame >= s->g.num_frames) return WV_ERR_ARG;
    *bytes = cone_bytes(s, frame, mask_host);
    return WV_OK;
}

int wv_cone_bytes_split(wv_stream *s, int frame, const uint8_t *mask_host, unsigned long long *fine,
                        unsigned long long *coarse) {
    if (!s || !mask_host || !fine || !coarse || frame < 0 || frame >= s->g.num_frames) return WV_ERR_ARG;
    const unsigned long long total = cone_bytes(s, frame, mask_host, nullptr, fine);
    *coarse = total - *fine;
    return WV_OK;
}

int wv_cone_bytes_fovea(wv_stream *s, int frame, const uint8_t *mask_host,
                        const uint8_t *fovea_host, unsigned long long *bytes) {
    if (!s || !mask_host || !bytes || frame < 0 || frame >= s->g.num_frames) return WV_ERR_ARG;
    *bytes = cone_bytes(s, frame, mask_host, fovea_host);
    return WV_OK;
}

int wv_request_bytes(const wv_request *r, unsigned long long *cone, unsigned long long *region) {
    if (!r || !r->s || !cone || !region) return WV_ERR_ARG;
    wv_stream *s = r->s;
    const Geom &g = s->g;
    if (r->frame < 0 || r->frame >= g.num_frames || r->out.width <= 0 || r->out.height <= 0)
        return WV_ERR_ARG;
    std::vector<uint8_t> mask((size_t)g.cells_x * g.cells_y);
    int tiles = 0;
    const int rc = wv_debug_footprint(s, r->yaw, r->pitch, r->fov, r->out.width, r->out.height,
                                      mask.data(), &tiles);
    if (rc != WV_OK) return rc;
    std::vector<uint8_t> fb;
    if (r->fovea) fovea_bits_host(g, r->yaw, r->pitch, *r, fb);
    *cone = cone_bytes(s, r->frame, mask.data(), r->fovea ? fb.data() : nullptr);
    unsigned long long cells = 0;
    for (uint8_t m : mask) cells += m ? 1 : 0;
    unsigned long long per_cell = 0;
    for (int p = 0; p < g.planes; ++p) per_cell += (unsigned long long)(kCell / g.p[p].sub) * (kCell / g.p[p].sub);
    *region = cells * per_cell;
    return WV_OK;
}

int wv_profile_begin(wv_stream *s) {
    if (!s) return WV_ERR_ARG;
    s->prof = true;
    s->ev_used = 0;
    s->ev_kind.clear();
    return WV_OK;
}

int wv_profile_end(wv_stream *s, wv_profile *out) {
    if (!s || !out) return WV_ERR_ARG;
    memset(out, 0, sizeof(*out));
    if (cudaStreamSynchronize(s->cs) != cudaSuccess) return WV_ERR_CUDA;
    for (size_t i = 0; i < s->ev_kind.size(); ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, s->ev_pool[2 * i], s->ev_pool[2 * i + 1]);
        const int k = s->ev_kind[i];
        out->ms[k] += ms;
        out->launches[k] += 1;
    }
    int cnt = 0;
    cudaMemcpy(&cnt, s->counters, 4, cudaMemcpyDeviceToHost);
    out->tiles = cnt;
    s->prof = false;
    s->ev_used = 0;
    s->ev_kind.clear();
    return WV_OK;
}

int wv_launches_per_viewport(const wv_stream *s) {
    if (!s) return WV_ERR_ARG;
    return split_mode(s) ? 5 : 4;
}

int wv_set_decode_mode(wv_stream *s, int mode) {
    if (!s || mode < 0 || mode > 2) return WV_ERR_ARG;
    s->decode_mode = mode;
    return WV_OK;
}

int wv_encode_sizes(const wv_stream_desc *desc, size_t *scratch_bytes, size_t *max_stream_bytes) {
    if (!desc) return WV_ERR_ARG;
    Geom g;
    if (build_geom(*desc, &g) != WV_OK) return WV_ERR_ARG;
    return encode_sizes(g, scratch_bytes, max_stream_bytes);
}

int wv_encode(const wv_stream_desc *desc, const void *const *planes_dev, void *scratch_dev,
              size_t scratch_bytes, void *out, size_t cap, size_t *out_len, void *cuda_stream) {
    if (!desc || !planes_dev || !scratch_dev || !out || !out_len || desc->quant != 0) return WV_ERR_ARG;
    Geom g;
    if (build_geom(*desc, &g) != WV_OK) return WV_ERR_ARG;
    return encode_run(g, planes_dev, scratch_dev, scratch_bytes, out, cap, out_len,
                      (cudaStream_t)cuda_stream);
}

int wv_encode_paper(const wv_stream_desc *desc, const void *const *planes_dev, void *scratch_dev,
                    size_t scratch_bytes, float alpha, float alpha_t, void *out, size_t cap, size_t *out_len,
                    void *cuda_stream) {
    if (!desc || !planes_dev || !scratch_dev || !out || !out_len || desc->quant != 1) return WV_ERR_ARG;
    if (!(alpha >= 0.f) || !(alpha_t >= 0.f) || !isfinite(alpha) || !isfinite(alpha_t)) return WV_ERR_ARG;
    Geom g;
    if (build_geom(*desc, &g) != WV_OK) return WV_ERR_ARG;
    return encode_paper(g, planes_dev, scratch_dev, scratch_bytes, alpha, alpha_t, out, cap, out_len,
                        (cudaStream_t)cuda_stream);
}

}  // extern "C"
