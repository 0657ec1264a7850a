// footprint.cu -- viewport footprint (low-resolution binary mask) and tile
// selection.
//
// Sec. 3.1: the region to reconstruct is defined on a low-resolution binary
// mask (256x256 for an 8k frame, i.e. 32-pixel cells) that can take any
// shape; Sec. 3.6: the mapping pass reads the reconstructed region, so the
// mask must hold every sample the mapping reads.
#include "wv_impl.h"

namespace wv {

namespace {

// Coarse tiles [c_lo, c_hi] (ctile samples of LL_2) holding LL_2 indices
// [lo, hi] of a subband of n2 samples after whole-sample symmetric extension.
// An output tile's LL_2 window is given by the geometry (Geom::wx0 ..
// Geom::wy1: the 9/7 halo of levels 2 and 1; the 5/3 window is narrower).
__device__ __forceinline__ void coarse_span(int lo, int hi, int n2, int ctile, int &c_lo,
                                            int &c_hi) {
    int a = max(lo, 0), b = min(hi, n2 - 1);
    if (lo < 0) b = max(b, min(-lo, n2 - 1));
    if (hi > n2 - 1) a = min(a, max(2 * (n2 - 1) - hi, 0));
    c_lo = a / ctile;
    c_hi = b / ctile;
}

constexpr float kReach = 3.0f;

// Footprint: one thread per mask cell.  The viewport samples the frame at positions
// inside the image of its frustum; every bilinear tap (luma, and centre-sited
// chroma mapped to luma) lies within 2.5 luma pixels of its position.  A cell
// is therefore needed when the cell grown by kReach pixels on every side
// meets the frustum.  The grown cell is a longitude/latitude rectangle on the
// sphere; it lies inside the spherical cap around its centre direction whose
// angular radius rho is the largest angle to a corner (along a parallel or a
// meridian the angle to a fixed point has at most one interior minimum, so
// the farthest point is a corner).  The cap is tested against each of the
// four frustum side planes (inward unit normals n_k): it meets half-space k
// iff n_k . c >= -sin(rho).  Passing all four tests is necessary for meeting
// the frustum, so the mask is a superset of the needed cells (cells near the
// frustum's corners may be included without being needed).  Rows 0 and
// H/32 - 1 extend to the poles because the resampler clamps v to the frame.
__device__ __forceinline__ bool cell_needed(const Frustum &f, int eq_w, int eq_h, int cells_y,
                                            int cx, int cy) {
    // grown cell in pixel coordinates -> longitude / latitude (radians / pi)
    const float u0 = (float)(cx * kCell) - kReach, u1 = (float)((cx + 1) * kCell) + kReach;
    const float v0 = (float)(cy * kCell) - kReach, v1 = (float)((cy + 1) * kCell) + kReach;
    const float sx = 2.0f / (float)eq_w, sy = 1.0f / (float)eq_h;
    const float lon0 = fmaf(u0 + 0.5f, sx, -1.0f), lon1 = fmaf(u1 + 0.5f, sx, -1.0f);
    float lat0 = fmaf(-(v1 + 0.5f), sy, 0.5f), lat1 = fmaf(-(v0 + 0.5f), sy, 0.5f);
    if (cy == 0) lat1 = 0.5f;
    if (cy == cells_y - 1) lat0 = -0.5f;
    lat0 = fmaxf(lat0, -0.5f);
    lat1 = fminf(lat1, 0.5f);
    const float lonc = 0.5f * (lon0 + lon1), latc = 0.5f * (lat0 + lat1);
    // unit directions (x = cos lat sin lon, y = sin lat, z = cos lat cos lon)
    float sa, ca, sb, cb, sc, cc, sl0, cl0, sl1, cl1, slc, clc;
    sincospif(lat0, &sa, &ca);
    sincospif(lat1, &sb, &cb);
    sincospif(latc, &sc, &cc);
    sincospif(lon0, &sl0, &cl0);
    sincospif(lon1, &sl1, &cl1);
    sincospif(lonc, &slc, &clc);
    const float c[3] = {cc * slc, sc, cc * clc};
    // smallest cosine to the four corners
    float mincos = 1.0f;
    const float cl[2] = {cl0, cl1}, sl[2] = {sl0, sl1};
    const float clat[2] = {ca, cb}, slat[2] = {sa, sb};
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const float d = c[0] * clat[j] * sl[i] + c[1] * slat[j] + c[2] * clat[j] * cl[i];
            mincos = fminf(mincos, d);
        }
    mincos = fminf(fmaxf(mincos, -1.0f), 1.0f);
    // sin(rho), with slack for float rounding of the dot products
    const float srho = sqrtf(fmaxf(0.0f, 1.0f - mincos * mincos)) * 1.01f + 1e-5f;
    if (mincos <= -0.5f) return true;   // caps wider than 120 degrees: always keep
    bool hit = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float d = f.n[k][0] * c[0] + f.n[k][1] * c[1] + f.n[k][2] * c[2];
        hit = hit && (d >= -srho);
    }
    return hit;
}

// Stamp the tile of every plane that holds cell (cx, cy), and the coarse
// tiles that tile reads.
__device__ __forceinline__ void stamp_cell(const Geom &g, int cx, int cy, uint32_t *tile_gen,
                                           uint32_t *ctile_gen, uint32_t gen) {
    int base = 0, cbase = 0;
    for (int p = 0; p < g.planes; ++p) {
        const PlaneGeom &pg = g.p[p];
        const int cw = kCell / pg.sub;   // plane pixels per cell side (tile sides are multiples)
        const int tx = cx * cw / g.tw, ty = cy * cw / g.th;
        tile_gen[base + ty * pg.tiles_x + tx] = gen;
        if (pg.ctiles_x > 0) {
            int cx0, cx1, cy0, cy1;
            const int qx = g.tw / 4, qy = g.th / 4;   // LL_2 samples per tile side
            coarse_span(qx * tx + g.wx0, qx * tx + g.wx1, pg.w >> 2, g.ctile, cx0, cx1);
            coarse_span(qy * ty + g.wy0, qy * ty + g.wy1, pg.h >> 2, g.ctile, cy0, cy1);
            for (int y = cy0; y <= cy1; ++y)
                for (int x = cx0; x <= cx1; ++x) ctile_gen[cbase + y * pg.ctiles_x + x] = gen;
        }
        base += pg.tiles_x * pg.tiles_y;
        cbase += pg.ctiles_x * pg.ctiles_y;
    }
}

// Foveation bits of cell (cx, cy): bit 0 = level-1 details kept (centre
// within r1 of the gaze), bit 1 = level-2 details kept (within r2).  The
// centre direction is rotated into viewer coordinates by R^T.
__device__ __forceinline__ uint8_t fovea_bits(const View &v, const Fovea &fv, int eq_w, int eq_h,
                                              int cx, int cy) {
    const float lon = fmaf((float)(cx * kCell + kCell / 2), 2.0f / (float)eq_w, -1.0f);
    const float lat = fmaf(-(float)(cy * kCell + kCell / 2), 1.0f / (float)eq_h, 0.5f);
    float sl, cl, sp, cp;
    sincospif(lon, &sl, &cl);
    sincospif(lat, &sp, &cp);
    const float dx = cp * sl, dy = sp, dz = cp * cl;
    const float x = v.r[0] * dx + v.r[3] * dy + v.r[6] * dz;
    const float y = v.r[1] * dx + v.r[4] * dy + v.r[7] * dz;
    const float z = v.r[2] * dx + v.r[5] * dy + v.r[8] * dz;
    if (!(z > 0.0f)) return 0;
    const float d = fmaxf(fabsf(atan2f(x, z) - fv.gx), fabsf(atan2f(y, z) - fv.gy));
    return (uint8_t)((d <= fv.r1 ? 1 : 0) | (d <= fv.r2 ? 2 : 0));
}

// Whether cell (cx, cy) of the frame is needed by the eye's equirect (rows
// v.row0 .. v.row0 + v.rows - 1; cells of the other eye of a stereo frame
// never are).
__device__ __forceinline__ bool cell_needed_eye(const View &v, const Frustum &f, int eq_w, int cx, int cy) {
    const int c0 = v.row0 >> kLogCell, nc = v.rows >> kLogCell;
    if (cy < c0 || cy >= c0 + nc) return false;
    return cell_needed(f, eq_w, v.rows, nc, cx, cy - c0);
}

__global__ void k_footprint(View v, Frustum f, Geom g, uint8_t *__restrict__ mask,
                            uint32_t *__restrict__ tile_gen, uint32_t *__restrict__ ctile_gen,
                            uint32_t gen, int *counters) {
    const int cx = blockIdx.x * blockDim.x + threadIdx.x;
    const int cy = blockIdx.y * blockDim.y + threadIdx.y;
    if (cx == 0 && cy == 0) counters[0] = counters[1] = counters[2] = 0;   // tile counts of this viewport
    if (cx >= g.cells_x || cy >= g.cells_y) return;
    const bool hit = cell_needed_eye(v, f, g.p[0].w, cx, cy);
    mask[cy * g.cells_x + cx] = hit ? 1 : 0;
    if (hit) stamp_cell(g, cx, cy, tile_gen, ctile_gen, gen);
}

// Batch: one z-slice of the grid per request; stamps go to the request's
// surface (stamp arrays cleared before the launch, stamp value 1).
__global__ void k_footprint_batch(const RequestJob *__restrict__ reqs,
                                  const SurfaceJob *__restrict__ surfs) {
    const RequestJob &r = reqs[blockIdx.z];
    const SurfaceJob &s = surfs[r.surface];
    const Geom &g = s.fine.g;
    const int cx = blockIdx.x * blockDim.x + threadIdx.x;
    const int cy = blockIdx.y * blockDim.y + threadIdx.y;
    if (cx >= g.cells_x || cy >= g.cells_y) return;
    if (cell_needed_eye(r.v, r.f, g.p[0].w, cx, cy))
        stamp_cell(g, cx, cy, s.stamp, s.stamp + g.total_tiles, 1u);
    if (r.fov.on && s.fmask) {
        const int c0 = r.v.row0 >> kLogCell, nc = r.v.rows >> kLogCell;
        s.fmask[cy * g.cells_x + cx] =
            (cy >= c0 && cy < c0 + nc) ? fovea_bits(r.v, r.fov, g.p[0].w, r.v.rows, cx, cy - c0) : 0;
    }
}

// Tile entry: plane << 28 | ty << 14 | tx, from index t of the plane-ordered
// tile (or coarse tile) range of a geometry.
__device__ __forceinline__ uint32_t tile_entry(const Geom &g, int t, bool coarse) {
    int plane = 0;
    for (;;) {
        const PlaneGeom &pg = g.p[plane];
        const int n = coarse ? pg.ctiles_x * pg.ctiles_y : pg.tiles_x * pg.tiles_y;
        if (t < n || plane == g.planes - 1) break;
        t -= n;
        ++plane;
    }
    const int nx = coarse ? g.p[plane].ctiles_x : g.p[plane].tiles_x;
    return ((uint32_t)plane << 28) | ((uint32_t)(t / nx) << 14) | (uint32_t)(t % nx);
}

// Tile selection: one thread per tile and one per coarse tile of every
// plane; a (coarse) tile is listed when the footprint stamped it with this
// viewport's generation.  One atomic per warp reserves list positions.
__device__ __forceinline__ void append(bool sel, uint32_t entry, uint32_t *list, int *count) {
    const unsigned ballot = __ballot_sync(0xffffffffu, sel);
    if (!sel) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(ballot) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(ballot));
    base = __shfl_sync(ballot, base, leader);
    list[base + __popc(ballot & ((1u << lane) - 1u))] = entry;
}

__global__ void k_select_tiles(Geom g, const uint32_t *__restrict__ tile_gen,
                               const uint32_t *__restrict__ ctile_gen, uint32_t gen,
                               uint32_t *__restrict__ tiles, uint32_t *__restrict__ ctiles,
                               int *counters) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const bool coarse = tid >= g.total_tiles;
    const int t0 = coarse ? tid - g.total_tiles : tid;
    const bool valid = coarse ? t0 < g.total_ctiles : true;
    bool sel = valid && (coarse ? ctile_gen[t0] : tile_gen[t0]) == gen;
    uint32_t entry = sel ? tile_entry(g, t0, coarse) : 0u;
    // edge strips are listed as two half strips (their reflected columns
    // make them the slowest tiles; halves halve their latency)
    const bool split = sel && !coarse && g.strip &&
                       !strip_interior((int)(entry & 0x3fff), g.p[(entry >> 28) & 3].w) &&
                       (int)((entry >> 14) & 0x3fff) * g.th + g.th / 2 < g.p[(entry >> 28) & 3].h;
    if (split) entry |= kHalfStrip;
    // warps straddling the two ranges: every call is made by all lanes
    append(sel && !coarse, entry, tiles, &counters[0]);
    append(split, entry | kLowerHalf, tiles, &counters[0]);
    append(sel && coarse, entry, ctiles, &counters[1]);
}

__device__ __forceinline__ void append2(bool sel, uint2 entry, uint2 *list, int *count) {
    const unsigned ballot = __ballot_sync(0xffffffffu, sel);
    if (!sel) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(ballot) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(ballot));
    base = __shfl_sync(ballot, base, leader);
    list[base + __popc(ballot & ((1u << lane) - 1u))] = entry;
}

// Batch selection: row blockIdx.y of the grid covers the stamps of surface
// blockIdx.y; listed entries carry the surface index.  Coarse tiles are also
// counted per surface (the fine tiles of a surface wait for that many).
__global__ void k_select_batch(const SurfaceJob *__restrict__ surfs, BatchLists lists, int *ctr) {
    const int si = blockIdx.y;
    const SurfaceJob &s = surfs[si];
    const Geom &g = s.fine.g;
    const int total = g.total_tiles + g.total_ctiles;
    if ((int)(blockIdx.x * blockDim.x) >= total) return;   // whole block outside: uniform
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const bool is_coarse = tid >= g.total_tiles;
    const bool sel = tid < total && s.stamp[tid] != 0;
    uint2 e = make_uint2((uint32_t)si, 0u);
    if (sel) e.y = tile_entry(g, is_coarse ? tid - g.total_tiles : tid, is_coarse);
    const int c = s.cls;
    // strip surfaces: fine tiles to the strip list, edge strips as two halves
    const bool st = sel && !is_coarse && s.strip;
    const bool split = st && !strip_interior((int)(e.y & 0x3fff), g.p[(e.y >> 28) & 3].w) &&
                       (int)((e.y >> 14) & 0x3fff) * g.th + g.th / 2 < g.p[(e.y >> 28) & 3].h;
    if (split) e.y |= kHalfStrip;
    append2(st, e, lists.strip[c], &ctr[4 * c + 3]);
    append2(split, make_uint2(e.x, e.y | kLowerHalf), lists.strip[c], &ctr[4 * c + 3]);
    append2(sel && !is_coarse && !s.strip, e, lists.fine[c], &ctr[4 * c + 2]);
    const unsigned cb = __ballot_sync(0xffffffffu, sel && is_coarse);
    if (cb && (threadIdx.x & 31) == __ffs(cb) - 1) atomicAdd(&ctr[kBatchCtr + 2 * si], __popc(cb));
    append2(sel && is_coarse, e, lists.coarse[c], &ctr[4 * c + 1]);
}

__global__ void k_all_tiles(int plane, int tiles_x, int tiles_y, uint32_t *tiles,
                            int *count, int *work) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        *count = tiles_x * tiles_y;
        if (work) *work = 0;
    }
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

void launch_footprint(const Geom &g, const View &v, uint8_t *mask, uint32_t *tile_gen,
                      uint32_t *ctile_gen, uint32_t gen, int *counters, cudaStream_t cs) {
    const Frustum f = make_frustum(v);
    dim3 block(32, 8);
    dim3 grid((g.cells_x + 31) / 32, (g.cells_y + 7) / 8);
    k_footprint<<<grid, block, 0, cs>>>(v, f, g, mask, tile_gen, ctile_gen, gen, counters);
}

void launch_footprint_batch(const RequestJob *reqs, const SurfaceJob *surfs, int n, int max_cx,
                            int max_cy, cudaStream_t cs) {
    dim3 block(32, 8);
    dim3 grid((max_cx + 31) / 32, (max_cy + 7) / 8, n);
    k_footprint_batch<<<grid, block, 0, cs>>>(reqs, surfs);
}

void launch_select_batch(const SurfaceJob *surfs, int m, int max_stamps, const BatchLists &lists,
                         int *ctr, cudaStream_t cs) {
    dim3 grid((max_stamps + 255) / 256, m);
    k_select_batch<<<grid, 256, 0, cs>>>(surfs, lists, ctr);
}

void launch_select_tiles(const Geom &g, const uint32_t *tile_gen, const uint32_t *ctile_gen,
                         uint32_t gen, uint32_t *tiles, uint32_t *ctiles, int *counters,
                         cudaStream_t cs) {
    const int threads = 256;
    const int blocks = (g.total_tiles + g.total_ctiles + threads - 1) / threads;
    k_select_tiles<<<blocks > 0 ? blocks : 1, threads, 0, cs>>>(g, tile_gen, ctile_gen, gen, tiles,
                                                                ctiles, counters);
}

void launch_all_tiles(const Geom &g, int plane, uint32_t *tiles, int *counters,
                      cudaStream_t cs) {
    const int n = g.p[plane].tiles_x * g.p[plane].tiles_y;
    k_all_tiles<<<(n + 255) / 256, 256, 0, cs>>>(plane, g.p[plane].tiles_x, g.p[plane].tiles_y,
                                                 tiles, &counters[0], &counters[2]);
}

void launch_all_ctiles(const Geom &g, int plane, uint32_t *ctiles, int *counters,
                       cudaStream_t cs) {
    const int n = g.p[plane].ctiles_x * g.p[plane].ctiles_y;
    k_all_tiles<<<(n + 255) / 256 > 0 ? (n + 255) / 256 : 1, 256, 0, cs>>>(
        plane, g.p[plane].ctiles_x, g.p[plane].ctiles_y, ctiles, &counters[1], nullptr);
}

void launch_project(const View &v, float *uv, cudaStream_t cs) {
    dim3 block(32, 8);
    dim3 grid((v.out_w + 31) / 32, (v.out_h + 7) / 8);
    k_project<<<grid, block, 0, cs>>>(v, uv);
}

}  // namespace wv
