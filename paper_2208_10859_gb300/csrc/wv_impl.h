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
//   counters  int32 [16]                 [0] = tile count, [1] = coarse tile count
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
constexpr int kTile = 128;      // output tile side (plane pixels)
constexpr int kThreads = 256;   // threads of the tile-decode CTA
constexpr int kCoarseTile = 64; // coarse tile side at level 2 (256 plane pixels)

// Subband index inside a level: 0 = LL (level L only), 1 = HL, 2 = LH, 3 = HH.
struct PlaneGeom {
    int w, h;
    int nbx[kMaxLevels + 1];           // blocks per row of a level-l subband
    int nby[kMaxLevels + 1];
    int base[kMaxLevels + 1][4];       // first block id of (level, subband)
    int tiles_x, tiles_y;
    int ctiles_x, ctiles_y;            // coarse tiles (kCoarseTile at level 2)
    int sub;                           // luma pixels per plane pixel (1 or 2)
    int ll2_pitch;                     // floats per row of the LL_2 plane
};

struct Geom {
    int planes, c420, levels, wavelet, num_frames, tlevels, block, log2b, nbpf;
    float step;
    PlaneGeom p[3];
    int cells_x, cells_y;
    int total_tiles;
    int total_ctiles;
};

// Coefficient frames that rebuild one frame (inverse inter-frame Haar):
// t[0] is the low band L_k, t[1..] the detail bands from level k down to 1;
// bit[b] = 1 means the detail is added, 0 subtracted.
struct Bands {
    int n;
    int t[kMaxBands];
    int bit[kMaxBands];
};

// Viewport camera: ray of pixel (i, j) is R * ((i + 1/2) sx - 1) t,
// (1 - (j + 1/2) sy) t, 1); equirectangular position
// u = lon * ku + cu, v = lat * kv + cv.
struct View {
    float r[9];
    float t, sx, sy;
    float ku, cu, kv, cv;
    int out_w, out_h;
};

// Inward unit normals (world coordinates) of the viewport frustum's four
// side planes: a direction d is inside when n_k . d >= 0 for every k.
struct Frustum {
    float n[4][3];
};

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

// host helpers (api.cu)
int build_geom(const wv_stream_desc &d, Geom *g);
Bands frame_bands(const Geom &g, int frame);
View make_view(float yaw, float pitch, float fov, int out_w, int out_h, int eq_w, int eq_h);
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
                                int *err, cudaStream_t cs);
cudaError_t launch_decode_coarse(const Geom &g, const int16_t *payload, const int32_t *table,
                                 const Bands &bands, float *const *ll2, const int *ll2_pitch,
                                 const uint32_t *tiles, const int *count, int *err, cudaStream_t cs);
cudaError_t launch_decode_fine(const Geom &g, const int16_t *payload, const int32_t *table,
                               const Bands &bands, const float *const *ll2, const int *ll2_pitch,
                               uint8_t *const *out_u8, float *out_f32, int f32_plane,
                               const uint32_t *tiles, const int *count, int *err, cudaStream_t cs);
void launch_resample(const Geom &g, const View &v, uint8_t *const *recon, const float *uv,
                     uint8_t *out, size_t pitch, cudaStream_t cs);
void launch_project(const View &v, float *uv, cudaStream_t cs);

// encoder (encode.cu)
int encode_sizes(const Geom &g, size_t *scratch, size_t *max_stream);
int encode_run(const Geom &g, const void *const *planes, void *scratch, size_t scratch_bytes,
               void *out, size_t cap, size_t *out_len, cudaStream_t cs);

}  // namespace wv

struct wv_stream {
    wv::Geom g;
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
    int decode_mode = 0;   // 0: coarse pass + fine pass (levels >= 3), 1: all levels fused
    int *counters = nullptr;
    int *err = nullptr;
    uint64_t n_payload = 0;
    std::vector<int32_t> table_host;
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
    const float lon = atan2f(dx, dz);
    const float lat = atan2f(dy, h);
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

__device__ __forceinline__ void record_error(int *err, int code) {
    atomicCAS(err, 0, code);
}

}  // namespace wv
#endif
