// wv_impl.h -- internal declarations of the GB300 wavelet viewport decoder.
//
// Device data of an open stream (all in one caller- or library-owned buffer):
//   payload   int16 [n_payload][B][B]   stored coefficient blocks, row-major
//   table     int32 [num_frames][nbpf]  slot of each block, -1 = all zero
//   recon     uint8 per plane, width x height, row-major (decoded region)
//   mask      uint8 [cells_y][cells_x]  low-resolution binary mask
//   ll2       float per plane, (w/4 rounded up to 8) x h/4: LL_2 of the
//             coarse pass (levels >= 3)
//   tiles     uint32 [max_tiles]        selected output tiles
//   tile_gen  uint32 [tiles]            generation that last selected a tile
//   ctile_gen uint32 [coarse tiles]      generation that last listed a coarse tile
//   ctiles    uint32 [coarse tiles]      coarse tiles the selected tiles need
//   counters  int32 [16]                 [0] = tile count, [1] = coarse tile count,
//                                        [2] = strip tiles taken (strip kernel)
//   err       int32                      first device-side error code
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/wv.h"

namespace wv {

constexpr int kMaxLevels = 6;
constexpr int kMaxBands = 4;    // 1 + tlevels, tlevels <= 3
constexpr int kCell = 32;       // luma pixels per mask cell (256 cells at 8192)
constexpr int kLogCell = 5;
constexpr int kTile = 128;      // default output tile side (plane pixels)
constexpr int kThreads = 256;   // threads of the tile-decode CTA
constexpr int kCoarseTile = 64; // default coarse tile side at level 2 (256 plane pixels)
constexpr int kStripW = 224;    // output columns of a strip tile (one warp: 28 lanes x 8)
#ifndef WV_STRIP_H
#define WV_STRIP_H 64
#endif
constexpr int kStripH = WV_STRIP_H;   // default output rows of a strip tile
// Strip tile entries (plane << 28 | ty << 14 | tx) with kHalfStrip set stand
// for half a strip (rows th/2), the lower half when kLowerHalf is set too:
// the tile selection splits the edge strips so, whose reflected columns
// make them the slowest.
constexpr uint32_t kHalfStrip = 1u << 31, kLowerHalf = 1u << 30;
// Interior strip: every level-1 and level-2 lane inside a plane of width w.
__host__ __device__ __forceinline__ bool strip_interior(int tx, int w) { return tx > 0 && tx * kStripW + 248 <= w; }

// Subband index inside a level: 0 = LL (level L only), 1 = HL, 2 = LH, 3 = HH.
struct PlaneGeom {
    int w, h;
    int nbx[kMaxLevels + 1];           // blocks per row of a level-l subband
    int nby[kMaxLevels + 1];
    int base[kMaxLevels + 1][4];       // first block id of (level, subband)
    int tiles_x, tiles_y;              // output tiles (Geom::tw x Geom::th samples)
    int ctiles_x, ctiles_y;            // coarse tiles (Geom::ctile samples of LL_2)
    int sub;                           // luma pixels per plane pixel (1 or 2)
    int ll2_pitch;                     // floats per row of the LL_2 plane
};

struct Geom {
    int planes, c420, levels, wavelet, num_frames, tlevels, block, log2b, nbpf;
    int quant;   // 0: dead-zone uniform quantiser (step); 1: byte quantiser of the paper format
    int stereo;  // 1: top/bottom stereo frames
    int dz_t;    // 9/7 dead zone: the device payload holds t = 2q + sign(q) (set at open)
    float step;
    PlaneGeom p[3];
    int cells_x, cells_y;
    int total_tiles;
    int total_ctiles;
    int tw, th;  // output tile width and height (plane pixels): square 64 or 128, or a strip kStripW x th
    int strip;   // 1: output tiles are strips decoded by the strip kernel (strip.cu)
    int ctile;   // coarse tile side (LL_2 samples): 32 or 64
    // LL_2 window an output tile (tx, ty) reads: columns (tw / 4) tx + wx0 ..
    // (tw / 4) tx + wx1, rows (th / 4) ty + wy0 .. (th / 4) ty + wy1 (before
    // symmetric extension); the coarse tiles holding it are decoded first
    int wx0, wx1, wy0, wy1;
    // payload blocks of the stream (table entries are below it; checked at
    // open on the host, and on the device in WV_CHECKED builds)
    int n_blocks;
};

// WV_CHECKED builds (build(checked=True)): the kernels test the indices
// their data decide (table entries, output and tap offsets, stamp indices)
// and on a violation record WV_ERR_DEVICE in the error word and skip the
// access instead of faulting.
#ifndef WV_CHECKED
#define WV_CHECKED 0
#endif
constexpr bool kChecked = WV_CHECKED != 0;

// Coefficient frames that rebuild one frame (inverse inter-frame Haar):
// t[0] is the low band L_k, t[1..] the detail bands from level k down to 1;
// bit[b] = 1 means the detail is added, 0 subtracted.
struct Bands {
    int n;
    int t[kMaxBands];
    int bit[kMaxBands];
    // byte quantiser (quant 1): per band, plane and class (0 approximation,
    // 1 details) the pair (c_min, (c_max - c_min) / 255)
    float qp[kMaxBands][3][2][2];
};

// Viewport camera: ray of pixel (i, j) is R * ((i + 1/2) sx - 1) t,
// (1 - (j + 1/2) sy) t, 1); equirectangular position
// u = lon * ku + cu, v = lat * kv + cv.
struct View {
    float r[9];
    float t, sx, sy;
    float ku, cu, kv, cv;
    int out_w, out_h;
    int row0, rows;   // luma rows of the equirect the eye sees (stereo: half the frame)
};

// Inward unit normals (world coordinates) of the viewport frustum's four
// side planes: a direction d is inside when n_k . d >= 0 for every k.
struct Frustum {
    float n[4][3];
};

// Foveated decoding (Sec. 3.7): the details of level 1 are kept only in mask
// cells whose centre lies within r1 of the gaze, those of level 2 within r2;
// distance = max(|theta_x - gx|, |theta_y - gy|) in viewer angles (theta_x =
// atan2(x, z), theta_y = atan2(y, z)), cells behind the viewer are outside.
struct Fovea {
    int on;
    float gx, gy, r1, r2;
};

struct Range {
    int lo, hi;
};

// Arguments of one tile-decode pass (levels l_top down to l_bot) over a list
// of tiles of one decode target.
struct TileArgs {
    Geom g;
    const int16_t *payload;
    const int32_t *table;
    Bands bands;
    int l_top, l_bot;        // levels synthesised: l_top down to l_bot
    int tw, th;              // output tile width and height at level l_bot - 1
    const float *ll_in[3];   // LL_{l_top} planes when l_top < levels
    int ll_in_pitch[3];
    uint8_t *out_u8[3];      // l_bot == 1: samples
    float *out_f32;          // l_bot == 1: float samples of plane f32_plane
    int f32_plane;
    float *ll_out[3];        // l_bot > 1: LL_{l_bot - 1} planes
    int ll_out_pitch[3];
    const uint8_t *fmask;    // foveation bits per mask cell (bit l-1: keep level l), or null
    const uint32_t *tiles;   // tile list (count entries)
    const int *count;
    int *work;               // strip kernel: next tile to take (zeroed before the launch)
    int *err;
    // payload blocks held (0: not checked; streams validate their table when
    // opened): a table entry at or above it reads as an absent block and
    // records WV_ERR_FORMAT
    int n_slots;
    // strip kernel: chroma (planes 1, 2) in groups of 4 samples, Cb and Cr
    // groups alternating (8 bytes per 4 positions), out_u8[2] = out_u8[1] + 4;
    // the resampler loads both planes' taps with one 8-byte load
    int out_pair;
    int a_floats, p_floats;
    // 9/7: half the dequantisation step times the synthesis band scaling
    // folded over all levels.  Synthesis scales a low band by K and a high
    // band by 1/K per axis at every level, the LL produced by level l + 1
    // included; with LL_L x K^(2L), HL_l and LH_l x K^(2(l-1)), HH_l x
    // K^(2(l-2)) the output of level l carries K^(2(l-1)), exactly the factor
    // the next finer level expects of its LL, and level 1 returns unscaled
    // samples.  (The half: the midpoint reconstruction is computed as
    // (2q + sign q) step / 2.)
    float scale[kMaxLevels + 1][4];
};

// Bilinear reprojection of one viewport from decoded planes.
struct ResampleArgs {
    View v;
    const uint8_t *plane[3];
    int w[3], h[3];
    int planes, c420;
    const float *uv;   // optional caller-given positions
    uint8_t *out;
    size_t pitch;
    // instead of RGBA: luma / 255 (float) and 8-bit Cb, Cr planes of the
    // viewport (out_w x out_h, tightly packed), for the post-filter
    float *y_plane;
    uint8_t *cb_plane, *cr_plane;
    int c_pair;   // plane[1] holds Cb and Cr in alternating 4-sample groups (plane[2] unused)
    int *err;     // WV_CHECKED builds: error word for out-of-plane taps
};

// ---- batched decoding ---------------------------------------------------------
// A batch decodes many viewport requests of several streams.  Requests of the
// same (stream, frame) without foveation share one decode target ("surface":
// its own reconstruction and LL_2 planes); a foveated request has its own.
struct SurfaceJob {
    TileArgs coarse;   // levels L..3 into LL_2 (used when levels >= 3)
    TileArgs fine;     // levels 2..1 from LL_2, or all levels when levels < 3
    uint32_t *stamp;   // tile stamps (total_tiles), then coarse stamps (total_ctiles)
    uint8_t *fmask;    // foveation cell bits (foveated surfaces), else null
    int cls;           // decode class (see kClasses)
    int strip;         // fine tiles are strips (fine: strip-pass arguments), decoded by k_strip_batch
};

// Decode classes of a batch: one persistent tile-decode launch per wavelet,
// foveation (a separately compiled kernel), code form and number of
// coefficient frames present: class = kMaxBands group + frames - 1 with
// group = 2 wavelet + foveated for codes q, 4 + foveated for 9/7 codes held
// as 2q + sign(q).
constexpr int kClasses = 6 * kMaxBands;

// Work lists of a batch, one pair per decode class.
struct BatchLists {
    uint2 *coarse[kClasses];
    uint2 *fine[kClasses];
    uint2 *strip[kClasses];   // strip tiles of the class's strip surfaces
};

struct RequestJob {
    View v;
    Frustum f;
    Fovea fov;
    int surface;
    ResampleArgs rs;
};

// Batch counters: decode class c uses [4c] next work item, [4c + 1] coarse
// items, [4c + 2] fine items, [4c + 3] strip items; surface s uses
// [kBatchCtr + 2s] coarse tiles listed and [kBatchCtr + 2s + 1] coarse
// tiles finished.
constexpr int kBatchCtr = 4 * kClasses;

struct StreamHeader {
    char magic[4];
    uint32_t version, width, height, planes, c420, levels, wavelet, num_frames,
        tlevels, block, quant, reserved0;
    float step;
    uint32_t nbpf, reserved1;
    uint64_t n_payload, table_off, payload_off;
};
static_assert(sizeof(StreamHeader) == 88, "stream header layout");
constexpr size_t kHeaderBytes = 128;

// paper-faithful stream format (paper.cu)
struct PaperInfo {
    uint64_t n_slots;              // stored blocks (blocks with records)
    std::vector<int32_t> table;    // [frame][block] slot or -1
    std::vector<uint2> src;        // per slot: byte offset of its records, count
    std::vector<float> qp;         // [frame][3][2][2] (c_min, step) per plane and class
};
bool is_paper_stream(const void *bytes, size_t n);
int paper_parse(const void *bytes, size_t n, wv_stream_desc *d, PaperInfo *info);
cudaError_t paper_transcode(const void *bytes, size_t n, const PaperInfo &info, int16_t *payload,
                            cudaStream_t cs);

// host helpers (api.cu)
int decode_region(wv_stream *s, int frame, float yaw, float pitch, float fov, int out_w, int out_h,
                  int eye = 0);
int build_geom(const wv_stream_desc &d, Geom *g, int tile = kTile, int ctile = kCoarseTile);
// Square-tile organisation with tw x th output tiles (multiples of the mask
// cell; the batch decoder's shapes).
int build_geom_rect(const wv_stream_desc &d, Geom *g, int tw, int th, int ctile);
// Strip geometry (output tiles kStripW x th, th a multiple of 32 in [32, 256])
// for streams the strip kernel decodes (strip_eligible), else WV_ERR_ARG.
int build_geom_strip(const wv_stream_desc &d, Geom *g, int th = kStripH, int ctile = kCoarseTile);
bool strip_eligible(const wv_stream_desc &d, uint64_t n_payload);
Bands frame_bands(const Geom &g, int frame);
View make_view(float yaw, float pitch, float fov, int out_w, int out_h, int eq_w, int eq_h, int row0 = 0);
int eye_view(const Geom &g, int eye, int *row0, int *rows);   // WV_ERR_ARG for an invalid eye
Frustum make_frustum(const View &v);

// kernel launchers
void launch_footprint(const Geom &g, const View &v, uint8_t *mask, uint32_t *tile_gen,
                      uint32_t *ctile_gen, uint32_t gen, int *counters, cudaStream_t cs);
void launch_select_tiles(const Geom &g, const uint32_t *tile_gen, const uint32_t *ctile_gen,
                         uint32_t gen, uint32_t *tiles, uint32_t *ctiles, int *counters,
                         cudaStream_t cs);
void launch_all_tiles(const Geom &g, int plane, uint32_t *tiles, int *counters,
                      cudaStream_t cs);
void launch_all_ctiles(const Geom &g, int plane, uint32_t *ctiles, int *counters,
                       cudaStream_t cs);
int decode_tiles_smem_bytes(const Geom &g);
int decode_tiles_grid(const Geom &g);
cudaError_t launch_decode_tiles(const Geom &g, const int16_t *payload, const int32_t *table,
                                const Bands &bands, uint8_t *const *out_u8, float *out_f32,
                                int f32_plane, const uint32_t *tiles, const int *counters,
                                int *err, cudaStream_t cs, int n_slots = 0);
cudaError_t launch_decode_coarse(const Geom &g, const int16_t *payload, const int32_t *table,
                                 const Bands &bands, float *const *ll2, const int *ll2_pitch,
                                 const uint32_t *tiles, const int *count, int *err, cudaStream_t cs);
cudaError_t launch_decode_strips(const Geom &g, const int16_t *payload, const int32_t *table,
                                 const Bands &bands, const float *const *ll2, const int *ll2_pitch,
                                 uint8_t *const *out_u8, float *out_f32, int f32_plane,
                                 const uint32_t *tiles, int *counters, int *err, cudaStream_t cs,
                                 bool chroma_pairs = false);
// Batched strip fine pass: the strip tiles (list of (surface, entry)) of the
// decode targets of one class whose coarse tiles are done; classes with up
// to two coefficient frames, 9/7 codes held as 2q + sign(q) or 5/3.
bool strip_batch_supported(int wavelet, int nb, bool dz_t);
cudaError_t launch_decode_strips_batch(int wavelet, int nb, bool fovea, bool dz_t, const SurfaceJob *surfs,
                                       const uint2 *list, const int *count, cudaStream_t cs);
cudaError_t launch_decode_fine(const Geom &g, const int16_t *payload, const int32_t *table,
                               const Bands &bands, const float *const *ll2, const int *ll2_pitch,
                               uint8_t *const *out_u8, float *out_f32, int f32_plane,
                               const uint32_t *tiles, const int *count, int *err, cudaStream_t cs);
void launch_resample(const Geom &g, const View &v, uint8_t *const *recon, const float *uv,
                     uint8_t *out, size_t pitch, cudaStream_t cs, float *y_plane = nullptr,
                     uint8_t *cb_plane = nullptr, uint8_t *cr_plane = nullptr, bool c_pair = false,
                     int *err = nullptr);
void fill_tile_scales(TileArgs &a);
void smem_needs_cached(int wavelet, int l_top, int l_bot, int tw, int th, int *a_floats, int *p_floats);

// batched kernels
void launch_footprint_batch(const RequestJob *reqs, const SurfaceJob *surfs, int n, int max_cx,
                            int max_cy, cudaStream_t cs);
void launch_select_batch(const SurfaceJob *surfs, int m, int max_stamps, const BatchLists &lists,
                         int *ctr, cudaStream_t cs);
// Largest |q| for which an opened 9/7 dead-zone stream keeps its codes as
// t = 2q + sign(q) on the device (|t| <= 16383: two bands add in 16 bits).
constexpr int kDzTMax = 8191;
cudaError_t payload_max_abs(const int16_t *payload, size_t count, int *dev_word, cudaStream_t cs);
cudaError_t payload_to_deadzone_t(int16_t *payload, size_t count, cudaStream_t cs);
cudaError_t launch_decode_batch(int wavelet, int nb, bool fovea, bool dz_t, const SurfaceJob *surfs,
                                const uint2 *coarse, const uint2 *fine, int *cls_ctr, int *surf_ctr,
                                int *err, const int *wait_polls, int smem_bytes, cudaStream_t cs);
// Polls of a batch's bounded device wait before it gives up (the default and
// the largest a batch accepts; wv_batch_set_wait_limit lowers it)
constexpr int kBatchWaitPolls = 1 << 21;
// Default device bytes of one wave of a batch's decode targets.
constexpr size_t kBatchWaveBytes = size_t(1) << 30;
// Device allocations of the library (stream stores, batch arenas): cudaMalloc,
// unless a failure was injected with wv_debug_fail_device_allocs.
cudaError_t dev_alloc(void **p, size_t bytes);
// Raises kernel fn's dynamic shared memory limit on the current device to at
// least `bytes` (never lowers it); one lock covers the check and the set, so
// concurrent launches from several host threads cannot undo each other.
cudaError_t opt_in_smem(const void *fn, int bytes);
// Whether a stream's reconstruction planes hold chroma as alternating Cb
// and Cr groups of 4 samples: the strip fine pass writes them so (decode
// mode 0), the square-tile passes plane by plane.
bool recon_pairs(const wv_stream *s);
// The reconstruction planes of the stream's last decode, and the release of
// its set once the resampling that reads them is enqueued on cs.
uint8_t *const *recon_planes(const wv_stream *s);
void release_recon(wv_stream *s, bool again = false);
void launch_resample_batch(const RequestJob *reqs, int n, int max_w, int max_h, cudaStream_t cs);
size_t batch_held_bytes(const wv_batch *b);   // device bytes a batch context holds (no sync)
void launch_project(const View &v, float *uv, cudaStream_t cs);

// encoder (encode.cu)
int encode_sizes(const Geom &g, size_t *scratch, size_t *max_stream);
int encode_run(const Geom &g, const void *const *planes, void *scratch, size_t scratch_bytes,
               void *out, size_t cap, size_t *out_len, cudaStream_t cs);
int encode_paper(const Geom &g, const void *const *planes, void *scratch, size_t scratch_bytes, float alpha,
                 float alpha_t, void *out, size_t cap, size_t *out_len, cudaStream_t cs);

}  // namespace wv

struct wv_stream {
    // g: geometry of the default decode (strip tiles when strip_eligible,
    // else square tiles); gsq: square 128-sample tiles (decode modes 1, 2)
    wv::Geom g;
    wv::Geom gsq;
    wv_stream_desc desc;
    int device = 0;
    cudaStream_t cs = nullptr;
    void *dmem = nullptr;
    bool owns = false;
    size_t dbytes = 0;
    int16_t *payload = nullptr;
    int32_t *table = nullptr;
    uint8_t *recon[3] = {nullptr, nullptr, nullptr};
    uint8_t *mask = nullptr;
    uint32_t *tiles = nullptr;
    uint32_t *tile_gen = nullptr;
    uint32_t *ctile_gen = nullptr;
    uint32_t *ctiles = nullptr;
    uint32_t gen = 0;   // viewport generation (stamps in tile_gen / ctile_gen)
    float *ll2[3] = {nullptr, nullptr, nullptr};
    int ll2_pitch[3] = {0, 0, 0};
    int decode_mode = 0;   // 0: default (strip fine pass), 1: all levels fused per square tile,
                           // 2: coarse pass + square-tile fine pass
    bool pair_ok = false;  // recon[1], recon[2] adjacent: chroma can be held in alternating groups
    int *counters = nullptr;
    int *err = nullptr;
    // A second set of per-viewport buffers (tile lists, counters, LL_2
    // planes): consecutive viewports alternate between the sets, so the
    // footprint, selection and coarse pass of a viewport (on the internal
    // stream `aux`) run while the previous viewport's fine pass and
    // resampling (on cs) are still executing.  Set 0 is the fields above.
    // The sets also hold a reconstruction each: a viewport's fine pass (on
    // the internal stream `fs`) writes one while the previous viewport's
    // resampling (on cs) reads the other.
    uint32_t *tiles1 = nullptr, *ctiles1 = nullptr;
    int *counters1 = nullptr;
    float *ll2_1[3] = {nullptr, nullptr, nullptr};
    uint8_t *recon1[3] = {nullptr, nullptr, nullptr};
    int slot = 0;
    int cur = 0;             // the set whose reconstruction holds the last decode
    bool pending = false;    // the last decode's set is released after its resampling on cs
    bool overlap = true;
    cudaStream_t aux = nullptr;
    cudaStream_t fs = nullptr;
    cudaEvent_t ev_ready[2] = {nullptr, nullptr};   // set k's coarse pass done (aux)
    cudaEvent_t ev_fine[2] = {nullptr, nullptr};    // set k's fine pass done (fs)
    cudaEvent_t ev_free[2] = {nullptr, nullptr};    // cs no longer reads set k
    uint64_t n_payload = 0;
    void *host_payload = nullptr;   // WV_OPEN_HOST_PAYLOAD: pinned, mapped coefficient store
    std::vector<int32_t> table_host;
    std::vector<float> qp_host;   // byte quantiser parameters (quant 1), [frame][3][2][2]
    // profiling: (kernel id, start, stop) event triples
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_kind;
    size_t ev_used = 0;
    int last_tiles = 0;
};

#ifdef __CUDACC__
namespace wv {

// Whole-sample symmetric extension of index i into [0, n).
__device__ __forceinline__ int reflect_idx(int i, int n) {
    if (n == 1) return 0;
    const int period = 2 * (n - 1);
    i %= period;
    if (i < 0) i += period;
    return i >= n ? period - i : i;
}

// atan2(y, x) in float32 for the projection, from a polynomial of this
// library's own fit: atan(t) = t P(t^2) on [0, 1] with P of degree 9, the
// coefficients minimising the largest relative error (Remez exchange; 2.4e-9
// in exact arithmetic, under 1.3 ulp in float32 Horner form).  Reduction:
// t = min(|x|, |y|) / max(|x|, |y|) (hardware reciprocal), then pi/2 - r
// when |y| > |x|, pi - r when x < 0, and the sign of y.  The largest error
// against fp64 over the projection's inputs is measured by the GPU tests
// (a few ulp of the result); atan2(0, 0) = 0.
__device__ __forceinline__ float wv_atan2(float y, float x) {
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    float rcp;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rcp) : "f"(mx));
    const float t = mx > 0.0f ? mn * rcp : 0.0f;
    const float u = t * t;
    float p = -0.0017539301188662648f;
    p = fmaf(p, u, 0.010726944543421268f);
    p = fmaf(p, u, -0.030804596841335297f);
    p = fmaf(p, u, 0.05755210295319557f);
    p = fmaf(p, u, -0.0837731584906578f);
    p = fmaf(p, u, 0.1094203069806099f);
    p = fmaf(p, u, -0.142619326710701f);
    p = fmaf(p, u, 0.1999826580286026f);
    p = fmaf(p, u, -0.3333328366279602f);
    p = fmaf(p, u, 1.0f);
    float r = p * t;
    if (ay > ax) r = 1.5707963267948966f - r;
    if (x < 0.0f) r = 3.141592653589793f - r;
    return copysignf(r, y);
}

// Equirectangular luma position sampled by viewport pixel (i, j).  *hxz
// receives |(dx, dz)| / |d|, the cosine of the ray's latitude: the absolute
// float32 error of the longitude grows as its inverse near the poles.
__device__ __forceinline__ void project_px(const View &v, int i, int j, float &u, float &w,
                                           float *hxz = nullptr) {
    const float xn = fmaf((float)i + 0.5f, v.sx, -1.0f) * v.t;
    const float yn = fmaf(-((float)j + 0.5f), v.sy, 1.0f) * v.t;
    const float dx = fmaf(v.r[0], xn, fmaf(v.r[1], yn, v.r[2]));
    const float dy = fmaf(v.r[3], xn, fmaf(v.r[4], yn, v.r[5]));
    const float dz = fmaf(v.r[6], xn, fmaf(v.r[7], yn, v.r[8]));
    const float h = sqrtf(fmaf(dx, dx, dz * dz));
    const float lon = wv_atan2(dx, dz);
    const float lat = wv_atan2(dy, h);
    u = fmaf(lon, v.ku, v.cu);
    w = fmaf(lat, v.kv, v.cv);
    if (hxz) *hxz = h * rsqrtf(fmaf(dy, dy, h * h));
}

// Split a coordinate into integer part and a fraction in 1/256 steps,
// rounding half up and carrying 256 into the integer part.
__device__ __forceinline__ void fixed_split(float t, int &i, int &f) {
    const float fl = floorf(t);
    i = (int)fl;
    f = (int)floorf(fmaf(t - fl, 256.0f, 0.5f));
    if (f >= 256) { f = 0; i += 1; }
}

// BT.709: Kr = 0.2126, Kb = 0.0722, Kg = 1 - Kr - Kb.
constexpr double kKr = 0.2126, kKb = 0.0722, kKg = 1.0 - kKr - kKb;
constexpr int kRCr = (int)(2.0 * (1.0 - kKr) * 65536.0 + 0.5);
constexpr int kGCb = (int)(2.0 * kKb * (1.0 - kKb) / kKg * 65536.0 + 0.5);
constexpr int kGCr = (int)(2.0 * kKr * (1.0 - kKr) / kKg * 65536.0 + 0.5);
constexpr int kBCb = (int)(2.0 * (1.0 - kKb) * 65536.0 + 0.5);

// YCbCr (8-bit, full range) -> RGBA8 with the integer BT.709 coefficients,
// rounded half up and clamped.
__device__ __forceinline__ uchar4 to_rgba(int y, int cb, int cr) {
    const int yy = y * 65536 + 32768;
    cb -= 128;
    cr -= 128;
    const int r = (yy + kRCr * cr) >> 16;
    const int g = (yy - kGCb * cb - kGCr * cr) >> 16;
    const int b = (yy + kBCb * cb) >> 16;
    return make_uchar4((unsigned char)min(max(r, 0), 255), (unsigned char)min(max(g, 0), 255),
                       (unsigned char)min(max(b, 0), 255), 255);
}

__device__ __forceinline__ void record_error(int *err, int code) {
    atomicCAS(err, 0, code);
}

// WV_CHECKED builds: whether 0 <= i < n, recording WV_ERR_DEVICE when not;
// always true in normal builds (the test compiles away).
__device__ __forceinline__ bool checked_in(long long i, long long n, int *err) {
    if constexpr (!kChecked) {
        return true;
    } else {
        if (i >= 0 && i < n) return true;
        if (err) record_error(err, WV_ERR_DEVICE);
        return false;
    }
}

}  // namespace wv
#endif
