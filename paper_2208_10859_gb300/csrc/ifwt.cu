// ifwt.cu -- fused per-tile decode: coefficient gather, dequantisation,
// inverse inter-frame Haar and every level of the 2D inverse FWT in one pass.
//
// Method: Sec. 3.5 rebuilds the wavelet representation of a frame on the GPU
// (the inverse inter-frame transform of Sec. 3.2 iterates over the uploaded
// coefficients, adding log2(n) detail coefficients with sign -1 or +1) and
// then runs the 2D iFWT only over the masked region (Sec. 3.1).
//
// Design: one CTA decodes one output tile (kTile x kTile samples of one
// plane).  Working from the coarsest level down, level l needs the
// coefficients of window K_l = [floor(K_{l-1}.lo / 2) - H, floor(K_{l-1}.hi /
// 2) + H] (H = 2 for 9/7, whose synthesis reads 3 resp. 4 interleaved samples
// to each side, H = 1 for 5/3), with K_0 the tile.  The interleaved array of
// level l (LL from the previous level, HL/LH/HH gathered from global memory)
// lives in shared memory; rows are synthesised first, then columns, each line
// by one thread with a streaming (pipelined) lifting that keeps the four
// lifting stages in registers.  Positions outside the plane are filled by
// whole-sample symmetric extension at every level.  The finest level writes
// the tile straight to the plane buffer.  No tensor cores: lifting is not a
// contraction.
#include <math.h>

#include "wv_impl.h"

namespace wv {

namespace {

// CDF 9/7 lifting factorisation (Daubechies & Sweldens 1998; JPEG2000 Part 1
// irreversible wavelet): analysis lifts with alpha, beta, gamma, delta and
// scales the low band by 1/K and the high band by K.
constexpr float kAlpha = -1.586134342059924f;
constexpr float kBeta = -0.052980118572961f;
constexpr float kGamma = 0.882911075530934f;
constexpr float kDelta = 0.443506852043971f;
constexpr double kK = 1.230174104914001;

template <int WAV>
struct Traits;
template <>
struct Traits<0> {   // LeGall 5/3, reversible integer lifting
    using T = int;
    static constexpr int H = 1;
};
template <>
struct Traits<1> {   // CDF 9/7, float lifting
    using T = float;
    static constexpr int H = 2;
};

struct Win {
    int lo, hi;
};

// Streaming 1D synthesis of an interleaved line p[0..n) (stride st).  Each
// output is emitted once all of its inputs have been read, so it may
// overwrite the line in place.  Outputs closer than the synthesis support to
// the line ends are not valid (the window halo absorbs them).
template <class Emit>
__device__ __forceinline__ void synth_line(float *p, int st, int n, Emit emit) {
    float po = p[st];
    float y1p = 0.f, y2pp = 0.f, y3pp = 0.f;
    for (int k = 0; k < n / 2; ++k) {
        const float e = p[(2 * k) * st];
        const float o = p[(2 * k + 1) * st];
        const float y1k = fmaf(-kDelta, po + o, e);          // even: -delta step
        const float y2m = fmaf(-kGamma, y1p + y1k, po);      // odd:  -gamma step
        const float y3m = fmaf(-kBeta, y2pp + y2m, y1p);     // even: -beta step
        const float y4m = fmaf(-kAlpha, y3pp + y3m, y2pp);   // odd:  -alpha step
        if (k >= 2) {
            emit(2 * k - 4, y3pp);
            emit(2 * k - 3, y4m);
        }
        y3pp = y3m;
        y2pp = y2m;
        y1p = y1k;
        po = o;
    }
}

template <class Emit>
__device__ __forceinline__ void synth_line(int *p, int st, int n, Emit emit) {
    int po = p[st];
    int y1p = 0;
    for (int k = 0; k < n / 2; ++k) {
        const int e = p[(2 * k) * st];
        const int o = p[(2 * k + 1) * st];
        const int y1k = e - ((po + o + 2) >> 2);    // x[2k]   = s[k] - floor((d[k-1]+d[k]+2)/4)
        const int y2m = po + ((y1p + y1k) >> 1);    // x[2k-1] = d[k-1] + floor((x[2k-2]+x[2k])/2)
        if (k >= 1) {
            emit(2 * k - 2, y1p);
            emit(2 * k - 1, y2m);
        }
        y1p = y1k;
        po = o;
    }
}

struct DecodeArgs {
    Geom g;
    const int16_t *payload;
    const int32_t *table;
    Bands bands;
    uint8_t *out_u8[3];
    float *out_f32;
    int f32_plane;
    const uint32_t *tiles;
    const int *counters;
    int *err;
    int buf_floats[2];
    // 9/7: dequantisation step times the synthesis band scaling folded over
    // all levels.  Synthesis scales a low band by K and a high band by 1/K
    // per axis at every level, the LL produced by level l + 1 included; with
    // LL_L x K^(2L), HL_l and LH_l x K^(2(l-1)), HH_l x K^(2(l-2)) the output
    // of level l carries K^(2(l-1)), which is exactly the factor the next
    // finer level expects of its LL, and level 1 returns unscaled samples.
    float scale[kMaxLevels + 1][4];
};

// Dequantised, temporally rebuilt coefficient (sub, level, kx, ky) of a plane.
template <int WAV>
__device__ __forceinline__ typename Traits<WAV>::T gather(const DecodeArgs &a, const PlaneGeom &pg,
                                                          int level, int sub, int kx, int ky) {
    const Geom &g = a.g;
    const int lb = g.log2b, bm = g.block - 1;
    const int bid = pg.base[level][sub] + (ky >> lb) * pg.nbx[level] + (kx >> lb);
    const int off = ((ky & bm) << lb) + (kx & bm);
    const size_t bsz = (size_t)g.block * g.block;
    if constexpr (WAV == 1) {
        float acc = 0.f;
        for (int b = 0; b < a.bands.n; ++b) {
            const int slot = __ldg(&a.table[(size_t)a.bands.t[b] * g.nbpf + bid]);
            float c = 0.f;
            if (slot >= 0) {
                const int q = __ldg(&a.payload[(size_t)slot * bsz + off]);
                // dead-zone reconstruction at the interval midpoint
                if (q != 0) c = (float)q + (q > 0 ? 0.5f : -0.5f);
            }
            acc = (b == 0) ? c : (a.bands.bit[b] ? acc + c : acc - c);
        }
        return acc * a.scale[level][sub];
    } else {
        const int s = (int)a.g.step;
        int v = 0;
        for (int b = 0; b < a.bands.n; ++b) {
            const int slot = __ldg(&a.table[(size_t)a.bands.t[b] * g.nbpf + bid]);
            int c = 0;
            if (slot >= 0) {
                const int q = __ldg(&a.payload[(size_t)slot * bsz + off]);
                if (q != 0) c = q > 0 ? q * s + (s >> 1) : q * s - (s >> 1);
            }
            if (b == 0) {
                v = c;
            } else {   // S-transform inverse: a = L - floor(H/2), b = a + H
                const int lo = v - (c >> 1);
                v = a.bands.bit[b] ? lo + c : lo;
            }
        }
        return v;
    }
}

template <int WAV>
__global__ void __launch_bounds__(kThreads, 2) k_decode_tiles(DecodeArgs a) {
    using T = typename Traits<WAV>::T;
    constexpr int H = Traits<WAV>::H;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf[2] = {reinterpret_cast<T *>(smem_raw),
                 reinterpret_cast<T *>(smem_raw) + a.buf_floats[0]};
    const int count = *(volatile const int *)a.counters;
    const Geom &g = a.g;
    const int L = g.levels;

    for (int ti = blockIdx.x; ti < count; ti += gridDim.x) {
        const uint32_t e = a.tiles[ti];
        const int plane = (int)(e >> 28);
        const int ty = (int)((e >> 14) & 0x3fff), tx = (int)(e & 0x3fff);
        const PlaneGeom &pg = g.p[plane];
        const int X0 = tx * kTile, X1 = min(X0 + kTile, pg.w);
        const int Y0 = ty * kTile, Y1 = min(Y0 + kTile, pg.h);

        Win wx[kMaxLevels + 1], wy[kMaxLevels + 1];
        wx[0] = {X0, X1 - 1};
        wy[0] = {Y0, Y1 - 1};
        for (int l = 1; l <= L; ++l) {
            wx[l] = {(wx[l - 1].lo >> 1) - H, (wx[l - 1].hi >> 1) + H};
            wy[l] = {(wy[l - 1].lo >> 1) - H, (wy[l - 1].hi >> 1) + H};
        }

        for (int l = L; l >= 1; --l) {
            T *cur = buf[(L - l) & 1];
            const T *prev = buf[(L - l + 1) & 1];
            const int aw = 2 * (wx[l].hi - wx[l].lo + 1);
            const int ah = 2 * (wy[l].hi - wy[l].lo + 1);
            const int st = aw + 1;
            const int nx = pg.w >> (l - 1), ny = pg.h >> (l - 1);   // level l-1 size
            const int gx0 = 2 * wx[l].lo, gy0 = 2 * wy[l].lo;
            int pst = 0, pgx0 = 0, pgy0 = 0, pah = 0;
            if (l < L) {
                pst = 2 * (wx[l + 1].hi - wx[l + 1].lo + 1) + 1;
                pah = 2 * (wy[l + 1].hi - wy[l + 1].lo + 1);
                pgx0 = 2 * wx[l + 1].lo;
                pgy0 = 2 * wy[l + 1].lo;
            }
            // 1. build the interleaved array of level l
            for (int idx = threadIdx.x; idx < aw * ah; idx += blockDim.x) {
                const int jy = idx / aw, jx = idx - jy * aw;
                const int ry = reflect_idx(gy0 + jy, ny), rx = reflect_idx(gx0 + jx, nx);
                const int ky = ry >> 1, kx = rx >> 1;
                const int sub = (rx & 1) + 2 * (ry & 1);   // 0 LL, 1 HL, 2 LH, 3 HH
                T val;
                if (sub == 0 && l < L) {
                    const int py = ky - pgy0, px = kx - pgx0;
                    if (py < 0 || py >= pah || px < 0 || px >= pst - 1) {
                        record_error(a.err, WV_ERR_DEVICE);
                        val = T(0);
                    } else {
                        val = prev[py * pst + px];
                    }
                } else {
                    val = gather<WAV>(a, pg, l, sub, kx, ky);
                }
                cur[jy * st + jx] = val;
            }
            __syncthreads();
            // 2. horizontal synthesis, one row per thread, in place
            for (int r = threadIdx.x; r < ah; r += blockDim.x) {
                T *row = cur + r * st;
                synth_line(row, 1, aw, [&](int i, T v) { row[i] = v; });
            }
            __syncthreads();
            // 3. vertical synthesis, one column per thread
            if (l > 1) {
                for (int c = threadIdx.x; c < aw; c += blockDim.x) {
                    T *col = cur + c;
                    synth_line(col, st, ah, [&](int i, T v) { col[i * st] = v; });
                }
            } else {
                const int c0 = X0 - gx0, c1 = X1 - gx0;   // valid output columns
                const int r0 = Y0 - gy0, r1 = Y1 - gy0;
                for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
                    T *col = cur + c;
                    const int x = X0 + (c - c0);
                    if (a.out_f32 && plane == a.f32_plane) {
                        float *o = a.out_f32 + x;
                        synth_line(col, st, ah, [&](int i, T v) {
                            if (i >= r0 && i < r1) o[(size_t)(Y0 + i - r0) * pg.w] = (float)v + 128.0f;
                        });
                    } else {
                        uint8_t *o = a.out_u8[plane] + x;
                        synth_line(col, st, ah, [&](int i, T v) {
                            if (i >= r0 && i < r1) {
                                int p;
                                if constexpr (WAV == 1) p = __float2int_rd(v + 128.5f);
                                else p = v + 128;
                                o[(size_t)(Y0 + i - r0) * pg.w] = (uint8_t)min(max(p, 0), 255);
                            }
                        });
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Largest interleaved array (rows x (cols + 1)) per buffer parity.
void buffer_sizes(const Geom &g, int out[2]) {
    const int H = g.wavelet == WV_WAVELET_97 ? 2 : 1;
    out[0] = out[1] = 0;
    Win w{0, kTile - 1};
    for (int l = 1; l <= g.levels; ++l) {
        w = {(w.lo >> 1) - H, (w.hi >> 1) + H};
        const int n = 2 * (w.hi - w.lo + 1);
        const int sz = n * (n + 1);
        int &slot = out[(g.levels - l) & 1];
        if (sz > slot) slot = sz;
    }
}

}  // namespace

int decode_tiles_smem_bytes(const Geom &g) {
    int b[2];
    buffer_sizes(g, b);
    return (b[0] + b[1]) * 4;
}

int decode_tiles_grid(const Geom &g) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms * 2;
}

cudaError_t launch_decode_tiles(const Geom &g, const int16_t *payload, const int32_t *table,
                                const Bands &bands, uint8_t *const *out_u8, float *out_f32,
                                int f32_plane, const uint32_t *tiles, const int *counters,
                                int *err, cudaStream_t cs) {
    DecodeArgs a;
    a.g = g;
    a.payload = payload;
    a.table = table;
    a.bands = bands;
    for (int p = 0; p < 3; ++p) a.out_u8[p] = out_u8[p];
    a.out_f32 = out_f32;
    a.f32_plane = f32_plane;
    a.tiles = tiles;
    a.counters = counters;
    a.err = err;
    buffer_sizes(g, a.buf_floats);
    const double k2 = kK * kK;
    for (int l = 0; l <= kMaxLevels; ++l) {
        a.scale[l][0] = (float)(g.step * pow(k2, g.levels));
        a.scale[l][1] = a.scale[l][2] = (float)(g.step * pow(k2, l - 1));
        a.scale[l][3] = (float)(g.step * pow(k2, l - 2));
    }
    const int smem = (a.buf_floats[0] + a.buf_floats[1]) * 4;
    const int grid = decode_tiles_grid(g);
    cudaError_t e;
    if (g.wavelet == WV_WAVELET_97) {
        e = cudaFuncSetAttribute(k_decode_tiles<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        k_decode_tiles<1><<<grid, kThreads, smem, cs>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_decode_tiles<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        k_decode_tiles<0><<<grid, kThreads, smem, cs>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace wv
