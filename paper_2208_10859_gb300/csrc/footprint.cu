// footprint.cu -- viewport footprint (low-resolution binary mask) and tile
// selection.
//
// Sec. 3.1: the region to reconstruct is defined on a low-resolution binary
// mask (256x256 for an 8k frame, i.e. 32-pixel cells) that can take any
// shape; Sec. 3.6: the mapping pass reads the reconstructed region, so the
// mask must hold every sample the mapping reads.  Here every viewport pixel
// is projected with the same arithmetic as the mapping kernel and the cells
// of its bilinear taps (luma and centre-sited chroma) are marked.  A margin
// of 1/64 pixel around each position makes the mask cover positions computed
// in higher precision as well.
#include "wv_impl.h"

namespace wv {

namespace {

constexpr float kMargin = 1.0f / 64.0f;

// Mark the cells of the bilinear taps of every position within +-mu (x) and
// +-mv (y) pixels of (u, v): columns floor(u - mu) .. floor(u + mu) + 1
// (wrapping), rows floor(v - mv) .. floor(v + mv) + 1 (clamped).
__device__ __forceinline__ void mark_taps(uint8_t *mask, int cells_x, int cells_y, float u,
                                          float v, float mu, float mv, int w, int h, int cell) {
    const int x_lo = (int)floorf(u - mu);
    const int x_hi = (int)floorf(u + mu) + 1;
    const int y_lo = min(max((int)floorf(v - mv), 0), h - 1);
    const int y_hi = min(max((int)floorf(v + mv) + 1, 0), h - 1);
    int c_lo = (x_lo >= 0 ? x_lo : x_lo - cell + 1) / cell;   // floor division
    int c_hi = (x_hi >= 0 ? x_hi : x_hi - cell + 1) / cell;
    if (c_hi - c_lo + 1 >= cells_x) {
        c_lo = 0;
        c_hi = cells_x - 1;
    }
    for (int cy = y_lo / cell; cy <= y_hi / cell && cy < cells_y; ++cy)
        for (int c = c_lo; c <= c_hi; ++c) {
            int cx = c % cells_x;
            if (cx < 0) cx += cells_x;
            mask[cy * cells_x + cx] = 1;
        }
}

__global__ void k_footprint(View v, uint8_t *__restrict__ mask, int cells_x, int cells_y,
                            int eq_w, int eq_h, int chroma, int *counters) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i == 0 && j == 0) counters[0] = 0;   // tile count of this viewport
    if (i >= v.out_w || j >= v.out_h) return;
    float u, w, hxz;
    project_px(v, i, j, u, w, &hxz);
    // longitude error bound grows as 1 / cos(latitude) toward the poles
    const float mu = fminf(kMargin + v.ku * 4e-6f / fmaxf(hxz, 1e-12f), (float)eq_w);
    mark_taps(mask, cells_x, cells_y, u, w, mu, kMargin, eq_w, eq_h, kCell);
    if (chroma) {
        const float uc = fmaf(u + 0.5f, 0.5f, -0.5f);
        const float vc = fmaf(w + 0.5f, 0.5f, -0.5f);
        mark_taps(mask, cells_x, cells_y, uc, vc, 0.5f * mu, 0.5f * kMargin, eq_w / 2, eq_h / 2,
                  kCell / 2);
    }
}

// One thread per candidate tile of every plane: a tile is selected when any
// mask cell it covers is set.  A selected tile also flags the coarse tiles
// (kCoarseTile samples of LL_2 per axis) that hold its LL_2 window
// [q t - 3, q t + q + 2] (q = kTile / 4; 9/7 halo, the 5/3 window is
// narrower), including the window's symmetric extension at the plane edges.
// The other mask buffer (used by the next viewport) is cleared on the way.
__device__ __forceinline__ bool any_cell(const Geom &g, const uint8_t *mask, const PlaneGeom &pg,
                                         int px0, int px1, int py0, int py1) {
    px1 = min(px1, pg.w);
    py1 = min(py1, pg.h);
    const int s = pg.sub;
    const int cx0 = px0 * s / kCell, cx1 = min((px1 * s - 1) / kCell, g.cells_x - 1);
    const int cy0 = py0 * s / kCell, cy1 = min((py1 * s - 1) / kCell, g.cells_y - 1);
    for (int cy = cy0; cy <= cy1; ++cy)
        for (int cx = cx0; cx <= cx1; ++cx)
            if (mask[cy * g.cells_x + cx]) return true;
    return false;
}

// Coarse tiles [c_lo, c_hi] holding LL_2 indices [lo, hi] of a subband of n2
// samples after whole-sample symmetric extension (mirrors at 0 and n2 - 1,
// one further sample toward the inside at the right end for safety).
__device__ __forceinline__ void coarse_span(int lo, int hi, int n2, int &c_lo, int &c_hi) {
    int a = max(lo, 0), b = min(hi, n2 - 1);
    if (lo < 0) b = max(b, min(-lo, n2 - 1));
    if (hi > n2 - 1) a = min(a, max(2 * (n2 - 1) - hi, 0));
    c_lo = a / kCoarseTile;
    c_hi = b / kCoarseTile;
}

__global__ void k_select_tiles(Geom g, const uint8_t *__restrict__ mask,
                               uint8_t *__restrict__ other, uint32_t *__restrict__ tiles,
                               uint8_t *__restrict__ cflags, int *counters) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int ncells = g.cells_x * g.cells_y;
    for (int c = tid; c < ncells; c += gridDim.x * blockDim.x) other[c] = 0;
    if (tid >= g.total_tiles) return;
    int plane = 0, t = tid, cbase = 0;
    while (plane < g.planes - 1 && t >= g.p[plane].tiles_x * g.p[plane].tiles_y) {
        t -= g.p[plane].tiles_x * g.p[plane].tiles_y;
        cbase += g.p[plane].ctiles_x * g.p[plane].ctiles_y;
        ++plane;
    }
    const PlaneGeom &pg = g.p[plane];
    const int tx = t % pg.tiles_x, ty = t / pg.tiles_x;
    if (!any_cell(g, mask, pg, tx * kTile, (tx + 1) * kTile, ty * kTile, (ty + 1) * kTile)) return;
    const int pos = atomicAdd(&counters[0], 1);
    tiles[pos] = ((uint32_t)plane << 28) | ((uint32_t)ty << 14) | (uint32_t)tx;
    if (pg.ctiles_x == 0) return;
    int cx0, cx1, cy0, cy1;
    const int q = kTile / 4;   // LL_2 samples per tile side
    coarse_span(q * tx - 3, q * tx + q + 2, pg.w >> 2, cx0, cx1);
    coarse_span(q * ty - 3, q * ty + q + 2, pg.h >> 2, cy0, cy1);
    for (int cy = cy0; cy <= cy1; ++cy)
        for (int cx = cx0; cx <= cx1; ++cx) cflags[cbase + cy * pg.ctiles_x + cx] = 1;
}

__global__ void k_fill(uint8_t *p, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 1;
}

__global__ void k_all_tiles(int plane, int tiles_x, int tiles_y, uint32_t *tiles,
                            int *count) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) *count = tiles_x * tiles_y;
    if (t >= tiles_x * tiles_y) return;
    tiles[t] = ((uint32_t)plane << 28) | ((uint32_t)(t / tiles_x) << 14) | (uint32_t)(t % tiles_x);
}

__global__ void k_project(View v, float *uv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= v.out_w || j >= v.out_h) return;
    float u, w;
    project_px(v, i, j, u, w);
    uv[2 * ((size_t)j * v.out_w + i)] = u;
    uv[2 * ((size_t)j * v.out_w + i) + 1] = w;
}

}  // namespace

void launch_footprint(const Geom &g, const View &v, uint8_t *mask, int *counters,
                      cudaStream_t cs) {
    dim3 block(32, 8);
    dim3 grid((v.out_w + 31) / 32, (v.out_h + 7) / 8);
    k_footprint<<<grid, block, 0, cs>>>(v, mask, g.cells_x, g.cells_y, g.p[0].w, g.p[0].h,
                                        g.planes == 3 && g.c420, counters);
}

void launch_select_tiles(const Geom &g, const uint8_t *mask, uint8_t *mask_other,
                         uint32_t *tiles, uint8_t *cflags, int *counters, cudaStream_t cs) {
    const int threads = 256;
    const int blocks = (g.total_tiles + threads - 1) / threads;
    k_select_tiles<<<blocks > 0 ? blocks : 1, threads, 0, cs>>>(g, mask, mask_other, tiles, cflags,
                                                                counters);
}

void launch_all_tiles(const Geom &g, int plane, uint32_t *tiles, int *counters,
                      cudaStream_t cs) {
    const int n = g.p[plane].tiles_x * g.p[plane].tiles_y;
    k_all_tiles<<<(n + 255) / 256, 256, 0, cs>>>(plane, g.p[plane].tiles_x, g.p[plane].tiles_y,
                                                 tiles, &counters[0]);
}

void launch_all_ctiles(const Geom &g, int plane, uint8_t *cflags, cudaStream_t cs) {
    int base = 0;
    for (int p = 0; p < plane; ++p) base += g.p[p].ctiles_x * g.p[p].ctiles_y;
    const int n = g.p[plane].ctiles_x * g.p[plane].ctiles_y;
    if (n > 0) k_fill<<<(n + 255) / 256, 256, 0, cs>>>(cflags + base, n);
}

void launch_project(const View &v, float *uv, cudaStream_t cs) {
    dim3 block(32, 8);
    dim3 grid((v.out_w + 31) / 32, (v.out_h + 7) / 8);
    k_project<<<grid, block, 0, cs>>>(v, uv);
}

}  // namespace wv
