// ifwt.cu -- tile decode: coefficient gather, dequantisation, inverse
// inter-frame Haar and the 2D inverse FWT over a range of levels in one pass.
//
// Method: Sec. 3.5 rebuilds the wavelet representation of a frame on the GPU
// (the inverse inter-frame transform of Sec. 3.2 adds log2(n) detail
// coefficients with sign -1 or +1 to the low band) and then runs the 2D iFWT
// only over the masked region (Sec. 3.1).
//
// One CTA decodes one output tile at level l_bot - 1 (l_bot = 1: samples).
// Working from level l_top down, level l needs the coefficients of the window
// K_l = [floor(K_{l-1}.lo / 2) - H, floor(K_{l-1}.hi / 2) + H] (H = 2 for 9/7,
// whose synthesis reads 3 resp. 4 interleaved samples on each side of an even
// resp. odd output; H = 1 for 5/3), where K_{l-1} is the range the level below
// needs.  Per level:
//   gather + rows: each lane owns 8 coefficient columns (16 interleaved
//     columns) of one array row: one aligned 16-byte load per subband and
//     temporal band, dequantisation and the inter-frame rebuild in registers,
//     then the horizontal lifting steps in registers with one warp shuffle per
//     step for the neighbour lane's edge value; results go to shared array A;
//   columns: every thread streams one column segment of A through the
//     vertical lifting steps (four pipelined stages in registers) and writes
//     the next level's LL window (shared P), an LL plane or the final samples.
// Positions outside the plane are filled by whole-sample symmetric extension
// at every level (edge chunks take a per-coefficient path).  Outputs within
// the synthesis support of an array edge are invalid and never used.  No
// tensor cores: lifting is not a contraction.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "codes.cuh"

namespace wv {

namespace {

template <int WAV>
struct Traits;
template <>
struct Traits<0> {   // LeGall 5/3, reversible integer lifting
    using T = int;
    static constexpr int H = 1;      // coefficient halo per level
    static constexpr int V = 2;      // invalid outputs at each line end
};
template <>
struct Traits<1> {   // CDF 9/7, float lifting
    using T = float;
    static constexpr int H = 2;
    static constexpr int V = 4;
};

__device__ __host__ __forceinline__ int floor8(int x) { return x & ~7; }

// ---- per-level geometry ----------------------------------------------------

struct LevelGeo {
    int l;
    Range ky;            // coefficient rows of the window
    int kx0, nch;        // first coefficient column (multiple of 8), 8-wide chunks
    int rows;            // interleaved array rows = 2 |ky|
    Range ox, oy;        // outputs of this level (level l-1 coordinates)
    int ja4, sa;         // A column origin (array column, multiple of 16), stride (multiple of 16)
    int nw, nh;          // subband size at level l
};

// Layout of the next level's LL window in P, written by level l's columns:
// rows oy, columns from floor8(ox.lo), stride a multiple of 8.
struct PLayout {
    int col0, stride;
};

__device__ __host__ __forceinline__ PLayout p_layout(Range ox) {
    PLayout p;
    p.col0 = floor8(ox.lo);
    p.stride = 8 * ((ox.hi + 1 - p.col0 + 7) >> 3);
    return p;
}

template <int H>
__device__ __forceinline__ LevelGeo make_level(int l, Range ox, Range oy, int pw, int ph) {
    LevelGeo G;
    G.l = l;
    G.ox = ox;
    G.oy = oy;
    const Range kx = {(ox.lo >> 1) - H, (ox.hi >> 1) + H};
    G.ky = {(oy.lo >> 1) - H, (oy.hi >> 1) + H};
    G.kx0 = floor8(kx.lo);
    G.nch = (kx.hi + 1 - G.kx0 + 7) >> 3;
    G.rows = 2 * (G.ky.hi - G.ky.lo + 1);
    G.ja4 = (ox.lo - 2 * G.kx0) & ~15;
    G.sa = ((ox.hi - 2 * G.kx0 + 1) - G.ja4 + 15) & ~15;
    G.nw = pw >> l;
    G.nh = ph >> l;
    return G;
}

// ---- dequantisation + inter-frame rebuild of 8 coefficients ----------------

template <int NB>
struct Raw {
    uint4 q[2][NB];      // [even/odd columns][band]
    bool have[2][NB];
    int keep[2];         // foveation: bit 0 keeps coefficients 0-3, bit 1 keeps 4-7
};

// QM = 2: dead-zone codes stored as t = 2q + sign(q) (transcoded when the
// stream was opened, |q| <= kDzTMax), so c = t step / 2 needs no sign logic;
// with two bands the pair L +- H is formed as 16-bit integers (|t| <= 16383:
// the sum fits) and converted once.  Results equal those of QM = 0 exactly:
// every intermediate is an integer below 2^24.
// QM = 1: the byte quantiser of the paper-faithful format (Sec. 3.3): a
// stored value v > 0 is code + 1 and decodes to c_min + code (c_max - c_min)
// / 255 of its coefficient frame, plane and class (cls 0: approximation
// band, 1: detail bands); 0 is an absent coefficient (0).
template <int WAV, int NB, int QM = 0>
__device__ __forceinline__ void combine8(const TileArgs &a, const uint4 *q, const bool *have,
                                         float s, int plane, int cls, typename Traits<WAV>::T out[8]) {
    if constexpr (WAV == 1 && QM == 2 && NB == 2) {
        const bool add = a.bands.bit[1];
        const uint32_t w0[4] = {q[0].x, q[0].y, q[0].z, q[0].w};
        const uint32_t w1[4] = {q[1].x, q[1].y, q[1].z, q[1].w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t l = have[0] ? w0[k] : 0u, h = have[1] ? w1[k] : 0u;
            float lo, hi;
            halves_to_float(add ? __vadd2(l, h) : __vsub2(l, h), lo, hi);
            out[2 * k] = lo * s;
            out[2 * k + 1] = hi * s;
        }
    } else if constexpr (WAV == 1 && QM == 2) {
        float acc[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[m] = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (!have[b] || (q[b].x | q[b].y | q[b].z | q[b].w) == 0) continue;
            const uint32_t w[4] = {q[b].x, q[b].y, q[b].z, q[b].w};
            const float sg = (b == 0 || a.bands.bit[b]) ? 1.f : -1.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float lo, hi;
                halves_to_float(w[k], lo, hi);
                acc[2 * k] = fmaf(sg, lo, acc[2 * k]);
                acc[2 * k + 1] = fmaf(sg, hi, acc[2 * k + 1]);
            }
        }
#pragma unroll
        for (int m = 0; m < 8; ++m) out[m] = acc[m] * s;
    } else if constexpr (WAV == 1 && QM == 1) {
        float acc[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[m] = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (!have[b] || (q[b].x | q[b].y | q[b].z | q[b].w) == 0) continue;
            const uint32_t w[4] = {q[b].x, q[b].y, q[b].z, q[b].w};
            const float sg = (b == 0 || a.bands.bit[b]) ? 1.f : -1.f;
            const float lo = a.bands.qp[b][plane][cls][0], d = a.bands.qp[b][plane][cls][1];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int v = (m & 1) ? hi16(w[m >> 1]) : lo16(w[m >> 1]);
                const float c = v ? fmaf((float)(v - 1), d, lo) : 0.f;
                acc[m] = fmaf(sg, c, acc[m]);
            }
        }
#pragma unroll
        for (int m = 0; m < 8; ++m) out[m] = acc[m] * s;
    } else if constexpr (WAV == 1) {
        float acc[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[m] = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            // absent block, or 8 coefficients in the dead zone: contributes 0
            if (!have[b] || (q[b].x | q[b].y | q[b].z | q[b].w) == 0) continue;
            const uint32_t w[4] = {q[b].x, q[b].y, q[b].z, q[b].w};
            const float sg = (b == 0 || a.bands.bit[b]) ? 1.f : -1.f;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int v = (m & 1) ? hi16(w[m >> 1]) : lo16(w[m >> 1]);
                // dead-zone reconstruction at the interval midpoint:
                // sign(q) (|q| + 1/2) = (2q + sign(q)) / 2
                const int t = 2 * v + min(max(v, -1), 1);
                acc[m] = fmaf(sg, (float)t, acc[m]);
            }
        }
#pragma unroll
        for (int m = 0; m < 8; ++m) out[m] = acc[m] * s;
    } else {
        const int st = (int)a.g.step;
        int v[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = 0;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (!have[b] || (q[b].x | q[b].y | q[b].z | q[b].w) == 0) continue;   // adds 0
            const uint32_t w[4] = {q[b].x, q[b].y, q[b].z, q[b].w};
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int qq = (m & 1) ? hi16(w[m >> 1]) : lo16(w[m >> 1]);
                const int c = qq == 0 ? 0 : (qq > 0 ? qq * st + (st >> 1) : qq * st - (st >> 1));
                if (b == 0) {
                    v[m] = c;
                } else {   // S-transform inverse: a = L - floor(H/2), b = a + H
                    const int lo = v[m] - (c >> 1);
                    v[m] = a.bands.bit[b] ? lo + c : lo;
                }
            }
        }
#pragma unroll
        for (int m = 0; m < 8; ++m) out[m] = v[m];
    }
}

// Foveated decoding (Sec. 3.7): whether the level-l (l = 1, 2) detail
// coefficient (kx, ky) of a plane is kept, from the foveation bits of the
// mask cell holding its nominal luma position (kx 2^l sub, ky 2^l sub).
__device__ __forceinline__ bool fovea_kept(const TileArgs &a, const PlaneGeom &pg, int l, int kx,
                                           int ky) {
    const int X = (kx << l) * pg.sub, Y = (ky << l) * pg.sub;
    return (__ldg(&a.fmask[(Y >> kLogCell) * a.g.cells_x + (X >> kLogCell)]) >> (l - 1)) & 1;
}

// Dequantised, rebuilt coefficient (scalar path for edge chunks).
template <int WAV, int NB, bool FOV, int QM = 0, bool CHK = false>
__device__ __forceinline__ typename Traits<WAV>::T coef1(const TileArgs &a, const PlaneGeom &pg, int plane,
                                                         int level, int sub, int kx, int ky) {
    const Geom &g = a.g;
    using T = typename Traits<WAV>::T;
    if (FOV && level <= 2 && sub != 0 && !fovea_kept(a, pg, level, kx, ky)) return T(0);
    const int lb = g.log2b, bm = g.block - 1;
    const int bid = pg.base[level][sub] + (ky >> lb) * pg.nbx[level] + (kx >> lb);
    const size_t off = (size_t)((ky & bm) << lb) + (kx & bm);
    const size_t bsz = (size_t)g.block * g.block;
    uint4 q[NB];
    bool have[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        int slot = __ldg(&a.table[(size_t)a.bands.t[b] * g.nbpf + bid]);
        if constexpr (CHK) {   // entries at or above the payload's block count: absent, recorded
            if (slot >= a.n_slots) {
                record_error(a.err, WV_ERR_FORMAT);
                slot = -1;
            }
        }
        have[b] = slot >= 0;
        const int v = have[b] ? (int)__ldg(&a.payload[(size_t)slot * bsz + off]) : 0;
        q[b] = make_uint4((uint32_t)(uint16_t)v, 0, 0, 0);
    }
    typename Traits<WAV>::T out[8];
    combine8<WAV, NB, QM>(a, q, have, a.scale[level][sub], plane, sub == 0 ? 0 : 1, out);
    return out[0];
}

template <class T>
__device__ __forceinline__ T from_bits(float f) {
    return reinterpret_cast<const T &>(f);
}
template <class T>
__device__ __forceinline__ float to_bits(T v) {
    return reinterpret_cast<const float &>(v);
}

// Position of column j of a row of A.  The 16-byte groups of a row are
// XOR-swizzled so that the four float4 stores of the 8 chunks a warp writes
// into one row hit 8 different bank groups, while a column keeps one
// position in every row (the vertical pass reads conflict-free).
__device__ __forceinline__ int swz(int j) {
    const int g = j >> 2;
    return ((g ^ ((g >> 3) & 3)) << 2) | (j & 3);
}

// ---- gather + horizontal synthesis ------------------------------------------

struct Task {
    bool active;
    int jy, c;           // array row, chunk
    int ky, py;          // coefficient row (after extension), row parity
    bool fast;           // chunk entirely inside the subband (no extension)
};

template <int WAV, int NB, bool FOV, bool CHK = false>
__device__ __forceinline__ void load_task(const TileArgs &a, const PlaneGeom &pg, const LevelGeo &G,
                                          const Task &t, Raw<NB> &r) {
    const Geom &g = a.g;
    const int lb = g.log2b, bm = g.block - 1;
    const size_t bsz = (size_t)g.block * g.block;
    const int kx = G.kx0 + 8 * t.c;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int sub = e ? (t.py ? 3 : 1) : (t.py ? 2 : 0);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            r.have[e][b] = false;
            r.q[e][b] = make_uint4(0, 0, 0, 0);
        }
        r.keep[e] = 3;
        if (!t.active || !t.fast || (sub == 0 && G.l < g.levels)) continue;
        // foveation: coefficients 0-3 and 4-7 of the chunk (one or two cells);
        // a chunk that keeps nothing is not loaded, a half is cleared later
        if (FOV && G.l <= 2 && sub != 0)
            r.keep[e] = (int)fovea_kept(a, pg, G.l, kx, t.ky) | ((int)fovea_kept(a, pg, G.l, kx + 4, t.ky) << 1);
        const bool any = !FOV || r.keep[e] != 0;
        const int bid = pg.base[G.l][sub] + (t.ky >> lb) * pg.nbx[G.l] + (kx >> lb);
        const size_t off = (size_t)((t.ky & bm) << lb) + (kx & bm);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            int slot = __ldg(&a.table[(size_t)a.bands.t[b] * g.nbpf + bid]);
            if constexpr (CHK) {   // entries at or above the payload's block count: absent, recorded
                if (slot >= a.n_slots) {
                    record_error(a.err, WV_ERR_FORMAT);
                    slot = -1;
                }
            }
            if (slot >= 0 && any) {
                r.have[e][b] = true;
                r.q[e][b] = __ldg(reinterpret_cast<const uint4 *>(a.payload + (size_t)slot * bsz + off));
            }
        }
    }
}

// Foveation: clear coefficients 0-3 (keep bit 0 unset) or 4-7 (bit 1 unset).
template <int NB>
__device__ __forceinline__ void clear_halves(uint4 (&q)[NB], int keep) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        if (!(keep & 1)) q[b].x = q[b].y = 0u;
        if (!(keep & 2)) q[b].z = q[b].w = 0u;
    }
}

template <int WAV, int NB, bool FOV, int QM = 0, bool CHK = false>
__device__ __forceinline__ void finish_task(const TileArgs &a, const PlaneGeom &pg, int plane,
                                            const LevelGeo &G, const Task &t, Raw<NB> &r,
                                            const float *P, int nch, float *A) {
    using T = typename Traits<WAV>::T;
    const Geom &g = a.g;
    T v[16];
    const int kx = G.kx0 + 8 * t.c;
    const int s_even = t.py ? 2 : 0;
    const int s_odd = t.py ? 3 : 1;
    if (t.active) {
        T ev[8], od[8];
        // odd columns: HL (even row) or HH (odd row)
        if (t.fast) {
            if (FOV && r.keep[1] != 3) clear_halves<NB>(r.q[1], r.keep[1]);
            combine8<WAV, NB, QM>(a, r.q[1], r.have[1], a.scale[G.l][s_odd], plane, 1, od);
        } else {
#pragma unroll
            for (int m = 0; m < 8; ++m)
                od[m] = coef1<WAV, NB, FOV, QM, CHK>(a, pg, plane, G.l, s_odd, refl_sub(kx + m, G.nw, 1), t.ky);
        }
        // even columns: LH (odd row) or LL (even row)
        if (s_even == 2 || G.l == g.levels) {
            if (t.fast) {
                if (FOV && r.keep[0] != 3) clear_halves<NB>(r.q[0], r.keep[0]);
                combine8<WAV, NB, QM>(a, r.q[0], r.have[0], a.scale[G.l][s_even], plane, s_even == 0 ? 0 : 1, ev);
            } else {
#pragma unroll
                for (int m = 0; m < 8; ++m)
                    ev[m] = coef1<WAV, NB, FOV, QM, CHK>(a, pg, plane, G.l, s_even, refl_sub(kx + m, G.nw, 0), t.ky);
            }
        } else if (G.l == a.l_top) {   // LL from a plane written by a coarser pass
            const float *src = a.ll_in[plane] + (size_t)t.ky * a.ll_in_pitch[plane];
            if (t.fast) {
                // L2 loads: in a batch the coarse pass writing these planes
                // runs in the same launch
                const float4 x0 = __ldcg(reinterpret_cast<const float4 *>(src + kx));
                const float4 x1 = __ldcg(reinterpret_cast<const float4 *>(src + kx + 4));
                const float f[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                for (int m = 0; m < 8; ++m) ev[m] = from_bits<T>(f[m]);
            } else {
#pragma unroll
                for (int m = 0; m < 8; ++m) ev[m] = from_bits<T>(__ldcg(src + refl_sub(kx + m, G.nw, 0)));
            }
        } else {                       // LL from the level above (shared P)
            const int sp = 8 * G.nch;
            const float *prow = P + (t.ky - G.ky.lo) * sp;
            if (t.fast) {
                const float4 x0 = *reinterpret_cast<const float4 *>(prow + 8 * t.c);
                const float4 x1 = *reinterpret_cast<const float4 *>(prow + 8 * t.c + 4);
                const float f[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                for (int m = 0; m < 8; ++m) ev[m] = from_bits<T>(f[m]);
            } else {
#pragma unroll
                for (int m = 0; m < 8; ++m) ev[m] = from_bits<T>(prow[refl_sub(kx + m, G.nw, 0) - G.kx0]);
            }
        }
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            v[2 * m] = ev[m];
            v[2 * m + 1] = od[m];
        }
    } else {
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = T(0);
    }
    // horizontal synthesis across the row's lanes (chunk c sits next to chunk
    // c - 1 and c + 1); lanes at the row ends use their own values, which only
    // affects the invalid columns at the array edges
    const bool has_l = t.c > 0, has_r = t.c < nch - 1;
    if constexpr (WAV == 1) {
        float L = __shfl_up_sync(0xffffffffu, v[15], 1);
        if (!has_l) L = v[1];
        v[0] = fmaf(-kDelta, L + v[1], v[0]);
#pragma unroll
        for (int m = 1; m < 8; ++m) v[2 * m] = fmaf(-kDelta, v[2 * m - 1] + v[2 * m + 1], v[2 * m]);
        float R = __shfl_down_sync(0xffffffffu, v[0], 1);
        if (!has_r) R = v[14];
#pragma unroll
        for (int m = 0; m < 7; ++m) v[2 * m + 1] = fmaf(-kGamma, v[2 * m] + v[2 * m + 2], v[2 * m + 1]);
        v[15] = fmaf(-kGamma, v[14] + R, v[15]);
        L = __shfl_up_sync(0xffffffffu, v[15], 1);
        if (!has_l) L = v[1];
        v[0] = fmaf(-kBeta, L + v[1], v[0]);
#pragma unroll
        for (int m = 1; m < 8; ++m) v[2 * m] = fmaf(-kBeta, v[2 * m - 1] + v[2 * m + 1], v[2 * m]);
        R = __shfl_down_sync(0xffffffffu, v[0], 1);
        if (!has_r) R = v[14];
#pragma unroll
        for (int m = 0; m < 7; ++m) v[2 * m + 1] = fmaf(-kAlpha, v[2 * m] + v[2 * m + 2], v[2 * m + 1]);
        v[15] = fmaf(-kAlpha, v[14] + R, v[15]);
    } else {
        int L = __shfl_up_sync(0xffffffffu, v[15], 1);
        if (!has_l) L = v[1];
        v[0] -= (L + v[1] + 2) >> 2;
#pragma unroll
        for (int m = 1; m < 8; ++m) v[2 * m] -= (v[2 * m - 1] + v[2 * m + 1] + 2) >> 2;
        int R = __shfl_down_sync(0xffffffffu, v[0], 1);
        if (!has_r) R = v[14];
#pragma unroll
        for (int m = 0; m < 7; ++m) v[2 * m + 1] += (v[2 * m] + v[2 * m + 2]) >> 1;
        v[15] += (v[14] + R) >> 1;
    }
    if (!t.active) return;
    // store the columns the vertical pass reads: A[jy][swz(j - ja4)]
    const int j0 = 16 * t.c - G.ja4;
    float *row = A + t.jy * G.sa;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = j0 + 4 * q;
        if (j >= 0 && j + 4 <= G.sa) {
            float4 w;
            w.x = to_bits<T>(v[4 * q]);
            w.y = to_bits<T>(v[4 * q + 1]);
            w.z = to_bits<T>(v[4 * q + 2]);
            w.w = to_bits<T>(v[4 * q + 3]);
            *reinterpret_cast<float4 *>(row + swz(j)) = w;
        }
    }
}

template <int WAV, int NB, bool FOV, int QM = 0, bool CHK = false>
__device__ __forceinline__ void gather_rows(const TileArgs &a, const PlaneGeom &pg, int plane, const LevelGeo &G,
                            const float *P, float *A) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int nch = G.nch;
    const int rpw = 32 / nch;               // rows per warp pass
    const int r_in = lane / nch;            // row of this lane within the pass
    const int c = lane - r_in * nch;        // chunk of this lane
    const bool lane_ok = r_in < rpw;
    const int stride = nwarps * rpw;
    const int kxc = G.kx0 + 8 * c;
    const bool fast_x = kxc >= 0 && kxc + 8 <= G.nw;
    auto make = [&](int jy) {
        Task t;
        t.jy = jy;
        t.c = c;
        t.active = lane_ok && jy < G.rows;
        int ry = t.active ? 2 * G.ky.lo + jy : 0;
        if (ry < 0 || ry >= 2 * G.nh) ry = reflect_idx(ry, 2 * G.nh);
        t.py = ry & 1;
        t.ky = ry >> 1;
        t.fast = fast_x;
        return t;
    };
    // one row task per lane and iteration: the coefficient loads are not
    // what limits this loop (it is issue-bound), and a single task in flight
    // leaves the registers to the scheduler
    for (int base = warp * rpw; base < G.rows; base += stride) {
        const Task t = make(base + r_in);
        Raw<NB> r;
        load_task<WAV, NB, FOV, CHK>(a, pg, G, t, r);
        finish_task<WAV, NB, FOV, QM, CHK>(a, pg, plane, G, t, r, P, nch, A);
    }
}

// ---- vertical synthesis -----------------------------------------------------

// Streaming synthesis of one column of A: emits array rows [r_a, r_b) (all
// valid), reading rows from r_a - V (rounded down to even) on.  Values travel
// as float bits (int bits for 5/3).  `col` is the (swizzled) column position.
template <int WAV, class Emit>
__device__ __forceinline__ void column_segment(const float *A, int sa, int col, int rows, int r_a,
                                               int r_b, Emit emit) {
    constexpr int VV = Traits<WAV>::V;
    int i = max(0, (r_a - VV) & ~1);
    const float *p = A + col;
    if constexpr (WAV == 1) {
        // pair i (rows i, i + 1) completes rows i - 4 (even) and i - 3 (odd)
        float po = p[(i + 1) * sa];
        float y1p = 0.f, y2pp = 0.f, y3pp = 0.f, y4m = 0.f;
        auto step = [&](int r) {
            const float e = p[r * sa];
            const float o = p[(r + 1) * sa];
            const float y1k = fmaf(-kDelta, po + o, e);          // even: -delta step
            const float y2m = fmaf(-kGamma, y1p + y1k, po);      // odd:  -gamma step
            const float y3m = fmaf(-kBeta, y2pp + y2m, y1p);     // even: -beta step
            y4m = fmaf(-kAlpha, y3pp + y3m, y2pp);               // odd:  -alpha step
            const float out_even = y3pp;
            y3pp = y3m;
            y2pp = y2m;
            y1p = y1k;
            po = o;
            return out_even;
        };
        for (; i < r_a + 3; i += 2) step(i);                 // warm-up: nothing valid yet
        if (i == r_a + 3) {                                  // odd r_a: only row i - 3
            step(i);
            emit(i - 3, y4m);
            i += 2;
        }
        for (; i <= r_b + 2; i += 2) {                        // rows i - 4 and i - 3
            const float ev = step(i);
            emit(i - 4, ev);
            emit(i - 3, y4m);
        }
        if (i - 4 <= r_b - 1 && i + 1 < rows) emit(i - 4, step(i));   // odd r_b: last even row
    } else {
        const int *pi = reinterpret_cast<const int *>(p);
        int po = pi[(i + 1) * sa];
        int y1p = 0, y2m = 0;
        auto step = [&](int r) {
            const int e = pi[r * sa];
            const int o = pi[(r + 1) * sa];
            const int y1k = e - ((po + o + 2) >> 2);    // x[r]   = s - floor((d_l + d_r + 2)/4)
            y2m = po + ((y1p + y1k) >> 1);              // x[r-1] = d + floor((x[r-2] + x[r])/2)
            const int out_even = y1p;
            y1p = y1k;
            po = o;
            return out_even;
        };
        // pair i completes rows i - 2 (even) and i - 1 (odd)
        for (; i < r_a + 1; i += 2) step(i);
        if (i == r_a + 1) {
            step(i);
            emit(i - 1, __int_as_float(y2m));
            i += 2;
        }
        for (; i <= r_b; i += 2) {
            const int ev = step(i);
            emit(i - 2, __int_as_float(ev));
            emit(i - 1, __int_as_float(y2m));
        }
        if (i - 2 <= r_b - 1 && i + 1 < rows) emit(i - 2, __int_as_float(step(i)));
    }
}

// Same as column_segment for two adjacent columns (col even: one 8-byte
// shared load per row for both); emit(i, v0, v1).
template <int WAV, class Emit>
__device__ __forceinline__ void column_pair(const float *A, int sa, int col, int rows, int r_a,
                                            int r_b, Emit emit) {
    constexpr int VV = Traits<WAV>::V;
    int i = max(0, (r_a - VV) & ~1);
    const float2 *p = reinterpret_cast<const float2 *>(A + col);
    const int s2 = sa / 2;
    if constexpr (WAV == 1) {
        float2 po = p[(i + 1) * s2];
        float2 y1p = {0.f, 0.f}, y2pp = {0.f, 0.f}, y3pp = {0.f, 0.f}, y4m = {0.f, 0.f};
        auto step = [&](int r) {
            const float2 e = p[r * s2];
            const float2 o = p[(r + 1) * s2];
            float2 y1k, y2m, y3m;
            y1k.x = fmaf(-kDelta, po.x + o.x, e.x);
            y1k.y = fmaf(-kDelta, po.y + o.y, e.y);
            y2m.x = fmaf(-kGamma, y1p.x + y1k.x, po.x);
            y2m.y = fmaf(-kGamma, y1p.y + y1k.y, po.y);
            y3m.x = fmaf(-kBeta, y2pp.x + y2m.x, y1p.x);
            y3m.y = fmaf(-kBeta, y2pp.y + y2m.y, y1p.y);
            y4m.x = fmaf(-kAlpha, y3pp.x + y3m.x, y2pp.x);
            y4m.y = fmaf(-kAlpha, y3pp.y + y3m.y, y2pp.y);
            const float2 out_even = y3pp;
            y3pp = y3m;
            y2pp = y2m;
            y1p = y1k;
            po = o;
            return out_even;
        };
        for (; i < r_a + 3; i += 2) step(i);
        if (i == r_a + 3) {
            step(i);
            emit(i - 3, y4m.x, y4m.y);
            i += 2;
        }
        for (; i <= r_b + 2; i += 2) {
            const float2 ev = step(i);
            emit(i - 4, ev.x, ev.y);
            emit(i - 3, y4m.x, y4m.y);
        }
        if (i - 4 <= r_b - 1 && i + 1 < rows) {
            const float2 ev = step(i);
            emit(i - 4, ev.x, ev.y);
        }
    } else {
        const int2 *pi = reinterpret_cast<const int2 *>(p);
        int2 po = pi[(i + 1) * s2];
        int2 y1p = {0, 0}, y2m = {0, 0};
        auto step = [&](int r) {
            const int2 e = pi[r * s2];
            const int2 o = pi[(r + 1) * s2];
            int2 y1k;
            y1k.x = e.x - ((po.x + o.x + 2) >> 2);
            y1k.y = e.y - ((po.y + o.y + 2) >> 2);
            y2m.x = po.x + ((y1p.x + y1k.x) >> 1);
            y2m.y = po.y + ((y1p.y + y1k.y) >> 1);
            const int2 out_even = y1p;
            y1p = y1k;
            po = o;
            return out_even;
        };
        for (; i < r_a + 1; i += 2) step(i);
        if (i == r_a + 1) {
            step(i);
            emit(i - 1, __int_as_float(y2m.x), __int_as_float(y2m.y));
            i += 2;
        }
        for (; i <= r_b; i += 2) {
            const int2 ev = step(i);
            emit(i - 2, __int_as_float(ev.x), __int_as_float(ev.y));
            emit(i - 1, __int_as_float(y2m.x), __int_as_float(y2m.y));
        }
        if (i - 2 <= r_b - 1 && i + 1 < rows) {
            const int2 ev = step(i);
            emit(i - 2, __int_as_float(ev.x), __int_as_float(ev.y));
        }
    }
}

// Decode one tile (entry: plane << 28 | ty << 14 | tx) of a pass: levels
// l_top down to l_bot; A and P are the CTA's shared arrays.
template <int WAV, int NB, bool FOV, int QM = 0, bool CHK = false>
__device__ __forceinline__ void decode_one(const TileArgs &a, uint32_t e, float *A, float *P) {
    constexpr int H = Traits<WAV>::H;
    const Geom &g = a.g;
    const int plane = (int)(e >> 28);
    const int ty = (int)((e >> 14) & 0x3fff), tx = (int)(e & 0x3fff);
    const PlaneGeom &pg = g.p[plane];
    const int nout_x = pg.w >> (a.l_bot - 1), nout_y = pg.h >> (a.l_bot - 1);
    // output ranges of every level (level l - 1 coordinates), l_bot upward
    Range ox[kMaxLevels + 2], oy[kMaxLevels + 2];
    ox[a.l_bot] = {tx * a.tw, min((tx + 1) * a.tw, nout_x) - 1};
    oy[a.l_bot] = {ty * a.th, min((ty + 1) * a.th, nout_y) - 1};
    for (int l = a.l_bot + 1; l <= a.l_top; ++l) {
        ox[l] = {(ox[l - 1].lo >> 1) - H, (ox[l - 1].hi >> 1) + H};
        oy[l] = {(oy[l - 1].lo >> 1) - H, (oy[l - 1].hi >> 1) + H};
    }
    for (int l = a.l_top; l >= a.l_bot; --l) {
        const LevelGeo G = make_level<H>(l, ox[l], oy[l], pg.w, pg.h);
        const PLayout pn = p_layout(G.ox);   // next level's LL window in P
        const bool fits = G.rows * G.sa <= a.a_floats && G.nch <= 32 &&
                          (l == a.l_bot || (G.oy.hi - G.oy.lo + 1) * pn.stride <= a.p_floats);
        if (!fits) {   // never taken for the sizes the launcher computed
            if (threadIdx.x == 0) record_error(a.err, WV_ERR_DEVICE);
            return;
        }
        // 1. gather + horizontal synthesis into A
        gather_rows<WAV, NB, FOV, QM, CHK>(a, pg, plane, G, P, A);
        __syncthreads();
        // 2. vertical synthesis of the columns the outputs need
        const int nv = G.ox.hi - G.ox.lo + 1;
        const int r0 = G.oy.lo - 2 * G.ky.lo, r1 = G.oy.hi - 2 * G.ky.lo + 1;
        const int jc0 = G.ox.lo - 2 * G.kx0 - G.ja4;   // A column of output ox.lo (unswizzled)
        if ((jc0 & 1) == 0 && (nv & 1) == 0) {
            // column pairs: both columns of a pair sit in one 8-byte slot of
            // the swizzled row (swz keeps j and j + 1 together for even j)
            const int np = nv / 2;
            const int nseg = max(1, min((int)blockDim.x / np, (r1 - r0) / 16));
            const int items = np * nseg;
            for (int it = threadIdx.x; it < items; it += blockDim.x) {
                const int jp = it % np, sg = it / np;
                const int ra = r0 + (r1 - r0) * sg / nseg, rb = r0 + (r1 - r0) * (sg + 1) / nseg;
                const int x = G.ox.lo + 2 * jp;
                const int col = swz(jc0 + 2 * jp);
                if (l > a.l_bot) {
                    float *dst = P + (x - pn.col0);
                    column_pair<WAV>(A, G.sa, col, G.rows, ra, rb, [&](int i, float v0, float v1) {
                        float *d = dst + (2 * G.ky.lo + i - G.oy.lo) * pn.stride;
                        d[0] = v0;
                        d[1] = v1;
                    });
                } else if (a.l_bot > 1) {
                    float *dst = a.ll_out[plane] + x;
                    const int pitch = a.ll_out_pitch[plane];
                    column_pair<WAV>(A, G.sa, col, G.rows, ra, rb, [&](int i, float v0, float v1) {
                        float *d = dst + (size_t)(2 * G.ky.lo + i) * pitch;
                        d[0] = v0;
                        d[1] = v1;
                    });
                } else if (a.out_f32 && plane == a.f32_plane) {
                    float *o = a.out_f32 + x;
                    column_pair<WAV>(A, G.sa, col, G.rows, ra, rb, [&](int i, float v0, float v1) {
                        float *d = o + (size_t)(2 * G.ky.lo + i) * pg.w;
                        d[0] = ((WAV == 1) ? v0 : (float)__float_as_int(v0)) + 128.0f;
                        d[1] = ((WAV == 1) ? v1 : (float)__float_as_int(v1)) + 128.0f;
                    });
                } else {
                    uint8_t *o = a.out_u8[plane] + x;
                    column_pair<WAV>(A, G.sa, col, G.rows, ra, rb, [&](int i, float v0, float v1) {
                        int p0, p1;
                        if constexpr (WAV == 1) {
                            p0 = __float2int_rd(v0 + 128.5f);
                            p1 = __float2int_rd(v1 + 128.5f);
                        } else {
                            p0 = __float_as_int(v0) + 128;
                            p1 = __float_as_int(v1) + 128;
                        }
                        const unsigned short w = (unsigned short)(min(max(p0, 0), 255) |
                                                                  (min(max(p1, 0), 255) << 8));
                        *reinterpret_cast<unsigned short *>(o + (size_t)(2 * G.ky.lo + i) * pg.w) = w;
                    });
                }
            }
        } else {
        const int nseg = max(1, min((int)blockDim.x / nv, (r1 - r0) / 16));
        const int items = nv * nseg;
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int jj = it % nv, sg = it / nv;
            const int ra = r0 + (r1 - r0) * sg / nseg, rb = r0 + (r1 - r0) * (sg + 1) / nseg;
            const int x = G.ox.lo + jj;
            if (l > a.l_bot) {
                float *dst = P + (x - pn.col0);
                column_segment<WAV>(A, G.sa, swz(jc0 + jj), G.rows, ra, rb, [&](int i, float v) {
                    dst[(2 * G.ky.lo + i - G.oy.lo) * pn.stride] = v;
                });
            } else if (a.l_bot > 1) {
                float *dst = a.ll_out[plane] + x;
                const int pitch = a.ll_out_pitch[plane];
                column_segment<WAV>(A, G.sa, swz(jc0 + jj), G.rows, ra, rb, [&](int i, float v) {
                    dst[(size_t)(2 * G.ky.lo + i) * pitch] = v;
                });
            } else if (a.out_f32 && plane == a.f32_plane) {
                float *o = a.out_f32 + x;
                column_segment<WAV>(A, G.sa, swz(jc0 + jj), G.rows, ra, rb, [&](int i, float v) {
                    const float f = (WAV == 1) ? v : (float)__float_as_int(v);
                    o[(size_t)(2 * G.ky.lo + i) * pg.w] = f + 128.0f;
                });
            } else {
                uint8_t *o = a.out_u8[plane] + x;
                column_segment<WAV>(A, G.sa, swz(jc0 + jj), G.rows, ra, rb, [&](int i, float v) {
                    int p;
                    if constexpr (WAV == 1) p = __float2int_rd(v + 128.5f);
                    else p = __float_as_int(v) + 128;
                    o[(size_t)(2 * G.ky.lo + i) * pg.w] = (uint8_t)min(max(p, 0), 255);
                });
            }
        }
        }
        __syncthreads();
    }
}

template <int WAV, int NB, int QM, bool CHK = false>
__global__ void __launch_bounds__(kThreads, 2) k_tiles(TileArgs a) {
    extern __shared__ __align__(16) float smem[];
    float *A = smem;
    float *P = smem + a.a_floats;
    const int count = *(volatile const int *)a.count;
    for (int ti = blockIdx.x; ti < count; ti += gridDim.x) decode_one<WAV, NB, false, QM, CHK>(a, a.tiles[ti], A, P);
}

// ---- batched decode: one persistent launch over all surfaces ---------------
//
// Work items are dispensed in order by one atomic counter: first every coarse
// tile of every surface, then every fine tile.  A fine tile waits (thread 0,
// bounded) until all coarse tiles of its surface are finished.  No wait can
// block forever: when a fine item is dispensed, every coarse item has already
// been dispensed to a running CTA, and coarse items never wait.  After
// a number of polls (the batch's wait limit, at most kBatchWaitPolls) the
// wait gives up, records WV_ERR_TIMEOUT and decodes anyway (all reads stay
// in bounds).

__device__ __forceinline__ int load_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool wait_at_least(const int *flag, int target, int polls) {
    for (int it = 0; it < polls; ++it) {
        if (load_acquire(flag) >= target) return true;
        __nanosleep(256);
    }
    return false;
}

template <int WAV, int NB, bool FOV, int QM>
__global__ void __launch_bounds__(kThreads, 2)
    k_tiles_batch(const SurfaceJob *__restrict__ surfs, const uint2 *__restrict__ coarse,
                  const uint2 *__restrict__ fine, int *cls, int *surf, int *err, const int *wait_polls) {
    extern __shared__ __align__(16) float smem[];
    __shared__ TileArgs sa;
    __shared__ uint2 s_item;
    __shared__ int s_kind;   // 0 coarse, 1 fine, 2 no work left
    float *A = smem;
    const int nc = cls[1], nf = cls[2];
    for (;;) {
        if (threadIdx.x == 0) {
            const int item = atomicAdd(&cls[0], 1);
            if (item < nc) {
                s_item = coarse[item];
                s_kind = 0;
            } else if (item < nc + nf) {
                const uint2 w = fine[item - nc];
                s_item = w;
                s_kind = 1;
                const int *c = surf + 2 * (int)w.x;
                const int polls = min(max(__ldg(wait_polls), 0), kBatchWaitPolls);
                if (!wait_at_least(c + 1, c[0], polls)) record_error(err, WV_ERR_TIMEOUT);
            } else {
                s_kind = 2;
            }
        }
        __syncthreads();
        const int kind = s_kind;
        if (kind == 2) break;
        const uint2 w = s_item;
        const int *src = reinterpret_cast<const int *>(kind == 0 ? &surfs[w.x].coarse : &surfs[w.x].fine);
        for (int k = threadIdx.x; k < (int)(sizeof(TileArgs) / 4); k += blockDim.x)
            reinterpret_cast<int *>(&sa)[k] = __ldg(src + k);
        __syncthreads();
        float *P = smem + sa.a_floats;   // a_floats and p_floats fit the launch's shared memory
        decode_one<WAV, NB, FOV, QM, kChecked>(sa, w.y, A, P);
        if (kind == 0) __threadfence();   // LL_2 stores visible GPU-wide before the count
        __syncthreads();
        if (kind == 0 && threadIdx.x == 0) atomicAdd(&surf[2 * (int)w.x + 1], 1);
    }
}

// Shared-memory needs (floats) of A and P for tiles of tw x th outputs at
// level l_bot - 1 synthesised from l_top: the largest row count over tile
// origins in y times the largest row stride over origins in x (A), and the
// largest output row count times the largest P stride (P).  Window sizes
// depend on the tile origin only modulo 2^(l_top - l_bot + 4) * tile, which
// the scan covers.
void smem_needs(int wavelet, int l_top, int l_bot, int tw, int th, int *a_floats, int *p_floats) {
    const int H = wavelet == WV_WAVELET_97 ? 2 : 1;
    int rows_max[kMaxLevels + 2] = {}, sa_max[kMaxLevels + 2] = {}, oy_max[kMaxLevels + 2] = {},
        ps_max[kMaxLevels + 2] = {};
    for (int axis = 0; axis < 2; ++axis) {
        const int tile = axis == 0 ? tw : th;
        for (int origin = 0; origin < 64 * tile; origin += tile) {
            Range outs[kMaxLevels + 2];
            outs[l_bot] = {origin, origin + tile - 1};
            for (int l = l_bot + 1; l <= l_top; ++l)
                outs[l] = {(outs[l - 1].lo >> 1) - H, (outs[l - 1].hi >> 1) + H};
            for (int l = l_bot; l <= l_top; ++l) {
                const Range ox = outs[l];
                const Range kx = {(ox.lo >> 1) - H, (ox.hi >> 1) + H};
                if (axis == 0) {
                    const int kx0 = floor8(kx.lo);
                    const int ja4 = (ox.lo - 2 * kx0) & ~15;
                    const int sa = ((ox.hi - 2 * kx0 + 1) - ja4 + 15) & ~15;
                    sa_max[l] = std::max(sa_max[l], sa);
                    ps_max[l] = std::max(ps_max[l], p_layout(ox).stride);
                } else {
                    rows_max[l] = std::max(rows_max[l], 2 * (kx.hi - kx.lo + 1));
                    oy_max[l] = std::max(oy_max[l], ox.hi - ox.lo + 1);
                }
            }
        }
    }
    int amax = 0, pmax = 0;
    for (int l = l_bot; l <= l_top; ++l) {
        amax = std::max(amax, rows_max[l] * sa_max[l]);
        if (l > l_bot) pmax = std::max(pmax, oy_max[l] * ps_max[l]);
    }
    *a_floats = amax;
    *p_floats = pmax;
}

std::mutex g_cache_mutex;

}  // namespace

void smem_needs_cached(int wavelet, int l_top, int l_bot, int tw, int th, int *a_floats, int *p_floats) {
    static std::map<std::tuple<int, int, int, int, int>, std::pair<int, int>> cache;
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    const auto key = std::make_tuple(wavelet, l_top, l_bot, tw, th);
    auto it = cache.find(key);
    if (it == cache.end()) {
        int af, pf;
        smem_needs(wavelet, l_top, l_bot, tw, th, &af, &pf);
        it = cache.emplace(key, std::make_pair(af, pf)).first;
    }
    *a_floats = it->second.first;
    *p_floats = it->second.second;
}

// Shared-memory sizes and the folded 9/7 scales of a pass.
void fill_tile_scales(TileArgs &a) {
    smem_needs_cached(a.g.wavelet, a.l_top, a.l_bot, a.tw, a.th, &a.a_floats, &a.p_floats);
    const double k2 = kK * kK;
    for (int l = 0; l <= kMaxLevels; ++l) {
        if (a.g.wavelet == WV_WAVELET_97) {
            // dead zone: (2q + sign q) step / 2; byte quantiser: coefficients
            // of samples / 255, back to 8-bit units
            const double unit = a.g.quant == 1 ? 255.0 : 0.5 * a.g.step;
            a.scale[l][0] = (float)(unit * pow(k2, a.g.levels));
            a.scale[l][1] = a.scale[l][2] = (float)(unit * pow(k2, l - 1));
            a.scale[l][3] = (float)(unit * pow(k2, l - 2));
        } else {
            a.scale[l][0] = a.scale[l][1] = a.scale[l][2] = a.scale[l][3] = 1.f;
        }
    }
}

namespace {

template <int WAV, int NB, int QM = 0, bool CHK = kChecked>
cudaError_t launch_t(const TileArgs &a, int grid, int threads, cudaStream_t cs) {
    const int smem = (a.a_floats + a.p_floats) * 4;
    cudaError_t e = opt_in_smem(reinterpret_cast<const void *>(k_tiles<WAV, NB, QM, CHK>), smem);
    if (e != cudaSuccess) return e;
    k_tiles<WAV, NB, QM, CHK><<<grid, threads, smem, cs>>>(a);
    return cudaGetLastError();
}

template <int WAV, int NB, bool FOV, int QM>
cudaError_t launch_batch_t(const SurfaceJob *surfs, const uint2 *coarse, const uint2 *fine,
                           int *cls, int *surf, int *err, const int *wait_polls, int smem_bytes, cudaStream_t cs) {
    int dev = 0, sms = 148, per_sm = 0;
    cudaError_t e = opt_in_smem(reinterpret_cast<const void *>(k_tiles_batch<WAV, NB, FOV, QM>), smem_bytes);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tiles_batch<WAV, NB, FOV, QM>, kThreads,
                                                                  smem_bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    k_tiles_batch<WAV, NB, FOV, QM><<<sms * per_sm, kThreads, smem_bytes, cs>>>(surfs, coarse, fine, cls, surf, err, wait_polls);
    return cudaGetLastError();
}

cudaError_t launch_args(TileArgs &a, cudaStream_t cs) {
    fill_tile_scales(a);
    // the coarse pass has few, small tiles: 4-warp CTAs, four per SM (its
    // latency, not its work, sets its duration); tile passes: 8 warps, two
    const bool coarse = a.l_bot > 1;
    const int threads = coarse ? kThreads / 2 : kThreads;
    const int grid = decode_tiles_grid(a.g) * (coarse ? 2 : 1);
    const int nb = a.bands.n;
    const bool table_check = a.n_slots > 0;
    if (kChecked && !table_check) a.n_slots = a.g.n_blocks;   // every variant checks in WV_CHECKED builds
    if (table_check) {   // table entries checked against the payload's block count (q codes only)
        if (a.g.quant != 0 || a.g.dz_t) return cudaErrorInvalidValue;
        if (a.g.wavelet == WV_WAVELET_97) {
            switch (nb) {
            case 1: return launch_t<1, 1, 0, true>(a, grid, threads, cs);
            case 2: return launch_t<1, 2, 0, true>(a, grid, threads, cs);
            case 3: return launch_t<1, 3, 0, true>(a, grid, threads, cs);
            default: return launch_t<1, 4, 0, true>(a, grid, threads, cs);
            }
        }
        switch (nb) {
        case 1: return launch_t<0, 1, 0, true>(a, grid, threads, cs);
        case 2: return launch_t<0, 2, 0, true>(a, grid, threads, cs);
        case 3: return launch_t<0, 3, 0, true>(a, grid, threads, cs);
        default: return launch_t<0, 4, 0, true>(a, grid, threads, cs);
        }
    }
    if (a.g.quant == 1) {   // paper-faithful byte quantiser (9/7 only)
        switch (nb) {
        case 1: return launch_t<1, 1, 1>(a, grid, threads, cs);
        case 2: return launch_t<1, 2, 1>(a, grid, threads, cs);
        case 3: return launch_t<1, 3, 1>(a, grid, threads, cs);
        default: return launch_t<1, 4, 1>(a, grid, threads, cs);
        }
    }
    if (a.g.wavelet == WV_WAVELET_97 && a.g.dz_t) {   // codes stored as 2q + sign(q)
        switch (nb) {
        case 1: return launch_t<1, 1, 2>(a, grid, threads, cs);
        case 2: return launch_t<1, 2, 2>(a, grid, threads, cs);
        case 3: return launch_t<1, 3, 2>(a, grid, threads, cs);
        default: return launch_t<1, 4, 2>(a, grid, threads, cs);
        }
    }
    if (a.g.wavelet == WV_WAVELET_97) {
        switch (nb) {
        case 1: return launch_t<1, 1>(a, grid, threads, cs);
        case 2: return launch_t<1, 2>(a, grid, threads, cs);
        case 3: return launch_t<1, 3>(a, grid, threads, cs);
        default: return launch_t<1, 4>(a, grid, threads, cs);
        }
    }
    switch (nb) {
    case 1: return launch_t<0, 1>(a, grid, threads, cs);
    case 2: return launch_t<0, 2>(a, grid, threads, cs);
    case 3: return launch_t<0, 3>(a, grid, threads, cs);
    default: return launch_t<0, 4>(a, grid, threads, cs);
    }
}

TileArgs base_args(const Geom &g, const int16_t *payload, const int32_t *table, const Bands &bands,
                   int *err) {
    TileArgs a;
    memset(&a, 0, sizeof(a));
    a.g = g;
    a.payload = payload;
    a.table = table;
    a.bands = bands;
    a.err = err;
    a.f32_plane = -1;
    return a;
}

}  // namespace

int decode_tiles_smem_bytes(const Geom &g) {
    int af, pf;
    smem_needs(g.wavelet, g.levels, 1, g.tw, g.th, &af, &pf);
    return (af + pf) * 4;
}

int decode_tiles_grid(const Geom &g) {
    (void)g;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms * 2;
}

// All levels of every listed tile in one kernel (no intermediate planes).
cudaError_t launch_decode_tiles(const Geom &g, const int16_t *payload, const int32_t *table,
                                const Bands &bands, uint8_t *const *out_u8, float *out_f32,
                                int f32_plane, const uint32_t *tiles, const int *counters,
                                int *err, cudaStream_t cs, int n_slots) {
    TileArgs a = base_args(g, payload, table, bands, err);
    a.n_slots = n_slots;
    a.l_top = g.levels;
    a.l_bot = 1;
    a.tw = g.tw;
    a.th = g.th;
    for (int p = 0; p < 3; ++p) a.out_u8[p] = out_u8[p];
    a.out_f32 = out_f32;
    a.f32_plane = f32_plane;
    a.tiles = tiles;
    a.count = counters;
    return launch_args(a, cs);
}

// Coarse levels L..3 of the listed coarse tiles (kCoarseTile x kCoarseTile at
// level 2) into float LL_2 planes (float bits of int values for 5/3).
cudaError_t launch_decode_coarse(const Geom &g, const int16_t *payload, const int32_t *table,
                                 const Bands &bands, float *const *ll2, const int *ll2_pitch,
                                 const uint32_t *tiles, const int *count, int *err, cudaStream_t cs) {
    TileArgs a = base_args(g, payload, table, bands, err);
    a.l_top = g.levels;
    a.l_bot = 3;
    a.tw = a.th = g.ctile;
    for (int p = 0; p < 3; ++p) {
        a.ll_out[p] = ll2[p];
        a.ll_out_pitch[p] = ll2_pitch[p];
    }
    a.tiles = tiles;
    a.count = count;
    return launch_args(a, cs);
}

// Levels 2 and 1 of the listed tiles, reading LL_2 from the planes written by
// launch_decode_coarse.
cudaError_t launch_decode_fine(const Geom &g, const int16_t *payload, const int32_t *table,
                               const Bands &bands, const float *const *ll2, const int *ll2_pitch,
                               uint8_t *const *out_u8, float *out_f32, int f32_plane,
                               const uint32_t *tiles, const int *count, int *err, cudaStream_t cs) {
    TileArgs a = base_args(g, payload, table, bands, err);
    a.l_top = 2;
    a.l_bot = 1;
    a.tw = g.tw;
    a.th = g.th;
    for (int p = 0; p < 3; ++p) {
        a.ll_in[p] = ll2[p];
        a.ll_in_pitch[p] = ll2_pitch[p];
        a.out_u8[p] = out_u8[p];
    }
    a.out_f32 = out_f32;
    a.f32_plane = f32_plane;
    a.tiles = tiles;
    a.count = count;
    return launch_args(a, cs);
}

// One persistent launch decoding every listed coarse and fine tile of a batch
// (surfaces whose coefficient frames number nb).
template <int WAV, bool FOV, int QM>
cudaError_t launch_batch_nb(int nb, const SurfaceJob *surfs, const uint2 *coarse, const uint2 *fine,
                            int *cls_ctr, int *surf_ctr, int *err, const int *wait_polls, int smem_bytes, cudaStream_t cs) {
    switch (nb) {
    case 1: return launch_batch_t<WAV, 1, FOV, QM>(surfs, coarse, fine, cls_ctr, surf_ctr, err, wait_polls, smem_bytes, cs);
    case 2: return launch_batch_t<WAV, 2, FOV, QM>(surfs, coarse, fine, cls_ctr, surf_ctr, err, wait_polls, smem_bytes, cs);
    case 3: return launch_batch_t<WAV, 3, FOV, QM>(surfs, coarse, fine, cls_ctr, surf_ctr, err, wait_polls, smem_bytes, cs);
    default: return launch_batch_t<WAV, 4, FOV, QM>(surfs, coarse, fine, cls_ctr, surf_ctr, err, wait_polls, smem_bytes, cs);
    }
}

cudaError_t launch_decode_batch(int wavelet, int nb, bool fovea, bool dz_t, const SurfaceJob *surfs,
                                const uint2 *coarse, const uint2 *fine, int *cls_ctr, int *surf_ctr,
                                int *err, const int *wait_polls, int smem_bytes, cudaStream_t cs) {
    if (wavelet == WV_WAVELET_97 && dz_t)
        return fovea ? launch_batch_nb<1, true, 2>(nb, surfs, coarse, fine, cls_ctr, surf_ctr, err, wait_polls, smem_bytes, cs)
                     : launch_batch_nb<1, false, 2>(nb, surfs, coarse, fine, cls_ctr, surf_ctr, err, wait_polls, smem_bytes, cs);
    if (wavelet == WV_WAVELET_97)
        return fovea ? launch_batch_nb<1, true, 0>(nb, surfs, coarse, fine, cls_ctr, surf_ctr, err, wait_polls, smem_bytes, cs)
                     : launch_batch_nb<1, false, 0>(nb, surfs, coarse, fine, cls_ctr, surf_ctr, err, wait_polls, smem_bytes, cs);
    return fovea ? launch_batch_nb<0, true, 0>(nb, surfs, coarse, fine, cls_ctr, surf_ctr, err, wait_polls, smem_bytes, cs)
                 : launch_batch_nb<0, false, 0>(nb, surfs, coarse, fine, cls_ctr, surf_ctr, err, wait_polls, smem_bytes, cs);
}

// ---- dead-zone codes as 2q + sign(q) -----------------------------------------

namespace {

__global__ void k_payload_max_abs(const int4 *__restrict__ p, size_t n, int *out) {
    int m = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int4 v = __ldcs(p + i);
        const uint32_t w[4] = {(uint32_t)v.x, (uint32_t)v.y, (uint32_t)v.z, (uint32_t)v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) m = max(m, max(abs(lo16(w[k])), abs(hi16(w[k]))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__device__ __forceinline__ uint32_t to_t(uint32_t w) {
    const int lo = lo16(w), hi = hi16(w);
    const int tl = 2 * lo + min(max(lo, -1), 1), th = 2 * hi + min(max(hi, -1), 1);
    return ((uint32_t)tl & 0xffffu) | ((uint32_t)th << 16);
}

__global__ void k_payload_to_t(int4 *__restrict__ p, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        int4 v = p[i];
        v.x = (int)to_t((uint32_t)v.x);
        v.y = (int)to_t((uint32_t)v.y);
        v.z = (int)to_t((uint32_t)v.z);
        v.w = (int)to_t((uint32_t)v.w);
        p[i] = v;
    }
}

int grid_for(size_t n) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (int)std::min<size_t>((n + 255) / 256, (size_t)sms * 8);
}

}  // namespace

cudaError_t payload_max_abs(const int16_t *payload, size_t count, int *dev_word, cudaStream_t cs) {
    const size_t n = count / 8;   // block payloads are multiples of 256 codes
    if (n == 0) return cudaSuccess;
    k_payload_max_abs<<<grid_for(n), 256, 0, cs>>>(reinterpret_cast<const int4 *>(payload), n, dev_word);
    return cudaGetLastError();
}

cudaError_t payload_to_deadzone_t(int16_t *payload, size_t count, cudaStream_t cs) {
    const size_t n = count / 8;
    if (n == 0) return cudaSuccess;
    k_payload_to_t<<<grid_for(n), 256, 0, cs>>>(reinterpret_cast<int4 *>(payload), n);
    return cudaGetLastError();
}

}  // namespace wv
