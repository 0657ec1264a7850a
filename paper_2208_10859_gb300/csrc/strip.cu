// strip.cu -- the fine pass of the viewport decode as column strips: levels 2
// and 1 of the masked inverse FWT (Sec. 3.1) with the coefficient gather,
// dequantisation and inverse inter-frame transform (Sec. 3.2, 3.5) of both
// levels, streamed down one strip tile by one warp.
//
// A strip tile is kStripW = 224 output columns (X0 = 224 tx) by th rows
// (Y0 = th ty) of one plane.  Its warp holds
//   level 2: lane i = level-2 interleaved columns C2 + 4i .. C2 + 4i + 3
//            (C2 = X0/2 - 8): two coefficients of each level-2 subband and
//            two LL_2 samples;
//   level 1: lane j = level-1 interleaved columns C1 + 8j .. C1 + 8j + 7
//            (C1 = X0 - 8): four coefficients of each level-1 subband.
// One iteration loads and synthesises one pair of level-2 interleaved rows
// (even row: LL_2 | HL_2, odd row: LH_2 | HH_2).  Horizontal lifting runs in
// registers with one warp shuffle per step for the neighbouring lane's edge
// value; vertical lifting is a running state per column in registers, so a
// pair of input rows completes a pair of output rows a fixed number of rows
// above it.  The two LL_1 rows completed this way pass through an eight-row
// ring in shared memory to the level-1 lanes, which synthesise two pairs of
// level-1 rows (LL_1 | HL_1, LH_1 | HH_1) in the same way and store four
// output rows.  No tile-sized array is kept anywhere.
//
// Lanes at the warp's edges compute with a missing neighbour; after the four
// lifting steps the first and last four columns of the warp are invalid, so
// level-2 lanes 1..30 deliver LL_1 columns X0/2 - 4 .. X0/2 + 115 and level-1
// lanes 1..28 write the strip's 224 columns.  Vertically the first pairs
// of a tile only warm the running state up (four pairs per level for 9/7).
//
// A strip touching the plane's left or right side (an edge strip) may be
// listed as two half strips of th / 2 rows each: its reflected columns make
// it the slowest tile, and the launch lasts as long as its slowest tile.
// The same strips of many decode targets run in one batched launch
// (k_strip_batch), with foveation (Sec. 3.7) dropping the detail rows of
// the cells outside its radii in the gather.
//
// Symmetric extension (whole-sample, in the interleaved line of every level,
// as the transform defines it): a source row or column outside the subband
// is read at its reflected index.  LL_1 outside the plane: above the top
// row and left of the first column, the level-2 synthesis itself yields the
// reflected values (its own extension is about the same sample); below the
// last row and right of the last column the level-1 line reflects about
// its last odd position, so the LL_1 value is read back from the ring at the
// reflected row or column.
//
// No tensor cores: lifting is not a contraction.
#include <string.h>

#include <algorithm>
#include <mutex>

#include "codes.cuh"

namespace wv {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStripWarps = 4;          // warps (strip tiles in flight) per CTA
constexpr int kRing = 8;                // LL_1 rows held per warp (two iterations + reflection)
constexpr int kRingW = 136;             // floats per ring row (128 used + a lane 31 overrun)
constexpr uint32_t kNone = 0xffffffffu; // absent block

template <int WAV>
struct SV;
template <>
struct SV<0> {   // LeGall 5/3, integers
    using T = int;
    static constexpr int D = 2;    // a pair of input rows at i, i + 1 completes rows i - D, i - D + 1
    static constexpr int P0 = 3;   // level-2 pairs before the first LL_1 row a tile needs
};
template <>
struct SV<1> {   // CDF 9/7, float32
    using T = float;
    static constexpr int D = 4;
    static constexpr int P0 = 4;
};

template <class T>
__device__ __forceinline__ T from_f(float f) {
    return reinterpret_cast<const T &>(f);
}
template <class T>
__device__ __forceinline__ float to_f(T v) {
    return reinterpret_cast<const float &>(v);
}

// ---- dequantisation + inter-frame rebuild of one word (two coefficients) ----
//
// w[b]: the two int16 codes of coefficient frame b (0 when the block is
// absent), sign of frame b >= 1 from bands.bit[b].  QM = 2: 9/7 dead-zone
// codes held as t = 2q + sign(q) (c = t step / 2, scale s carries step / 2);
// QM = 0: codes q (9/7: c = (2q + sign q) step / 2; 5/3: integer
// reconstruction sign(q)(|q| step + floor(step / 2))).  5/3 frames combine by
// the inverse S-transform.
template <int WAV, int NB, int QM>
__device__ __forceinline__ void dq_word(const uint32_t (&w)[NB], const Bands &bd, float s, int st,
                                        typename SV<WAV>::T &lo, typename SV<WAV>::T &hi) {
    if constexpr (WAV == 1 && QM == 2 && NB == 1) {
        float a, b;
        halves_to_float(w[0], a, b);
        lo = a * s;
        hi = b * s;
    } else if constexpr (WAV == 1 && QM == 2 && NB == 2) {
        float a, b;
        halves_to_float(bd.bit[1] ? __vadd2(w[0], w[1]) : __vsub2(w[0], w[1]), a, b);
        lo = a * s;
        hi = b * s;
    } else if constexpr (WAV == 1) {
        float al = 0.f, ah = 0.f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            float x, y;
            if constexpr (QM == 2) {
                halves_to_float(w[b], x, y);
            } else {
                const int ql = lo16(w[b]), qh = hi16(w[b]);
                x = (float)(2 * ql + min(max(ql, -1), 1));
                y = (float)(2 * qh + min(max(qh, -1), 1));
            }
            const float sg = (b == 0 || bd.bit[b]) ? 1.f : -1.f;
            al = fmaf(sg, x, al);
            ah = fmaf(sg, y, ah);
        }
        lo = al * s;
        hi = ah * s;
    } else {
        int v[2] = {0, 0};
#pragma unroll
        for (int b = 0; b < NB; ++b) {
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int q = m ? hi16(w[b]) : lo16(w[b]);
                const int c = q == 0 ? 0 : (q > 0 ? q * st + (st >> 1) : q * st - (st >> 1));
                if (b == 0) {
                    v[m] = c;
                } else {   // S-transform inverse: a = L - floor(H / 2), b = a + H
                    const int l = v[m] - (c >> 1);
                    v[m] = bd.bit[b] ? l + c : l;
                }
            }
        }
        lo = v[0];
        hi = v[1];
    }
}

// ---- coefficient rows of one subband for one lane --------------------------

// Per lane and subband: the element offset of the lane's first coefficient in
// row 0 of the current block row, per coefficient frame (kNone: block
// absent), refreshed when the source row enters another block row.
template <int NB>
struct SubRow {
    int by;
    uint32_t off[NB];
};

struct LaneCols {
    int kx;        // first coefficient column (fast lanes)
    int c0;        // first interleaved column
    bool fast;     // all columns inside the plane: vector loads
    bool zero;     // no column can reach a written output: zeros, no loads
    bool mirror;   // columns outside the plane: values from the mirror lane (mirror_row)
    bool scalar;   // columns outside a narrow plane: codes loaded one at a time
};

template <int NB>
__device__ __forceinline__ void sub_refresh(const TileArgs &a, const PlaneGeom &pg, int level, int sub, int by,
                                            const LaneCols &lc, SubRow<NB> &r) {
    const Geom &g = a.g;
    r.by = by;
    const int bid = pg.base[level][sub] + by * pg.nbx[level] + (lc.kx >> g.log2b);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
#if WV_CHECKED
        int slot = lc.fast ? __ldg(&a.table[(size_t)a.bands.t[b] * g.nbpf + bid]) : -1;
        if (slot >= 0 && !checked_in(slot, g.n_blocks, a.err)) slot = -1;
#else
        const int slot = lc.fast ? __ldg(&a.table[(size_t)a.bands.t[b] * g.nbpf + bid]) : -1;
#endif
        r.off[b] = slot >= 0 ? ((uint32_t)slot << (2 * g.log2b)) + (uint32_t)(lc.kx & (g.block - 1)) : kNone;
    }
}

// One int16 code of subband `sub` at level `level`, (kx, ky) inside the
// subband, packed into bits 0-15 of the result (0 for an absent block).
template <int NB>
__device__ __noinline__ void code1(const TileArgs &a, const PlaneGeom &pg, int level, int sub, int kx, int ky,
                                   uint32_t (&v)[NB]) {
    const Geom &g = a.g;
    const int lb = g.log2b, bm = g.block - 1;
    const int bid = pg.base[level][sub] + (ky >> lb) * pg.nbx[level] + (kx >> lb);
    const size_t off = (size_t)((ky & bm) << lb) + (kx & bm);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
#if WV_CHECKED
        int slot = __ldg(&a.table[(size_t)a.bands.t[b] * g.nbpf + bid]);
        if (slot >= 0 && !checked_in(slot, g.n_blocks, a.err)) slot = -1;
#else
        const int slot = __ldg(&a.table[(size_t)a.bands.t[b] * g.nbpf + bid]);
#endif
        v[b] = slot >= 0 ? (uint32_t)(uint16_t)__ldg(&a.payload[((size_t)slot << (2 * lb)) + off]) : 0u;
    }
}

// Foveated decoding (Sec. 3.7): whether the level-l (l = 1, 2) detail
// coefficient (kx, ky) of a plane is kept, from the foveation bits of the
// mask cell holding its nominal luma position (kx 2^l sub, ky 2^l sub).  A
// lane's coefficients of one subband row (four at level 1, two at level 2)
// share one cell: strips start on a cell boundary and a lane's columns are
// 8-aligned.
__device__ __forceinline__ bool fov_keep(const TileArgs &a, const PlaneGeom &pg, int l, int kx, int ky) {
    const int X = (kx << l) * pg.sub, Y = (ky << l) * pg.sub;
    return (__ldg(&a.fmask[(Y >> kLogCell) * a.g.cells_x + (X >> kLogCell)]) >> (l - 1)) & 1;
}

// ---- asynchronous staging of each lane's coefficient words -----------------
//
// Iteration q of a tile reads, per lane, NW words of each level-2 subband
// (NW = 1) and of each level-1 subband of its two row pairs (NW = 2) per
// coefficient frame, plus two LL_2 samples.  They are copied global ->
// shared with cp.async by the lane that will read them, kStages - 1
// iterations ahead, into a per-warp ring of stages (zero fill for absent
// blocks), so no iteration waits on DRAM.  Lanes whose columns need
// symmetric extension load their codes one at a time when they compute.

constexpr int kStages = 3;

__device__ __forceinline__ void cp_async(uint32_t *dst, const void *src, int bytes, bool fill) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(fill ? 8 : 0)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(fill ? 4 : 0)
                     : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Stage layout (32-bit words, lane-major items): level-1 items (pair h,
// subband 1..3, frame b) of NW = 2 words, level-2 items (subband 0..3, frame
// b) of one word, one LL_2 item of two words.
template <int NB>
struct Stage {
    static constexpr int kL1 = 6 * NB;                     // items of 2 words
    static constexpr int kL2 = 4 * NB;                     // items of 1 word
    static constexpr int kWords = 32 * (2 * kL1 + kL2 + 2);
    __device__ static uint32_t *l1(uint32_t *st, int h, int sub, int b, int lane) {
        return st + 2 * (((h * 3 + sub - 1) * NB + b) * 32 + lane);
    }
    __device__ static uint32_t *l2(uint32_t *st, int sub, int b, int lane) {
        return st + 64 * kL1 + (sub * NB + b) * 32 + lane;
    }
    __device__ static uint32_t *ll(uint32_t *st, int lane) { return st + 64 * kL1 + 32 * kL2 + 2 * lane; }
};

// Issue the copies of one subband row (source row kr) for this lane; dst(b)
// is the lane's item of frame b.  Lanes without a vector path copy nothing
// (zero lanes: zero fill).
template <int NB, int NW, class Dst>
__device__ __forceinline__ void sub_issue(const TileArgs &a, const PlaneGeom &pg, int level, int sub, int kr,
                                          const LaneCols &lc, SubRow<NB> &r, Dst dst, bool keep = true) {
    const Geom &g = a.g;
    // one path for every lane: lanes without a vector load copy zero bytes
    // (zero fill); the block row is the warp's, so the refresh is uniform
    const int by = kr >> g.log2b;
    if (by != r.by) sub_refresh<NB>(a, pg, level, sub, by, lc, r);
    const uint32_t roff = (uint32_t)(kr & (g.block - 1)) << g.log2b;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const bool have = r.off[b] != kNone && keep;   // kNone for all but vector lanes
        cp_async(dst(b), a.payload + (have ? r.off[b] + roff : 0u), 4 * NW, have);
    }
}

// Codes of a lane whose columns leave the plane, one at a time at the
// reflected column (out of line: edge strips only).
template <int NB, int NW, bool FOV>
__device__ __noinline__ void sub_fetch_slow(const TileArgs &a, const PlaneGeom &pg, int level, int sub, int par,
                                            int n2, int kr, int c0, uint32_t (&w)[NB][NW]) {
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int k = 0; k < NW; ++k) w[b][k] = 0u;
#pragma unroll
    for (int m = 0; m < 2 * NW; ++m) {
        const int kc = refl(c0 + 2 * m + par, n2) >> 1;
        uint32_t v[NB];
        code1<NB>(a, pg, level, sub, kc, kr, v);
        if (FOV && !fov_keep(a, pg, level, kc, kr))
#pragma unroll
            for (int b = 0; b < NB; ++b) v[b] = 0u;
#pragma unroll
        for (int b = 0; b < NB; ++b) w[b][m >> 1] |= v[b] << (16 * (m & 1));
    }
}

// The lane's NW words of a subband row: from the stage (vector lanes), or
// one code at a time at the reflected column (interleaved parity `par`, line
// length `n2` = twice the subband width).
template <int NB, int NW, bool FOV = false, class Src>
__device__ __forceinline__ void sub_fetch(const TileArgs &a, const PlaneGeom &pg, int level, int sub, int par,
                                          int n2, int kr, const LaneCols &lc, Src src, uint32_t (&w)[NB][NW]) {
    if (!lc.scalar) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const uint32_t *p = src(b);
            if constexpr (NW == 2) {
                const uint2 x = *reinterpret_cast<const uint2 *>(p);
                w[b][0] = x.x;
                w[b][NW - 1] = x.y;
            } else {
                w[b][0] = *p;
            }
        }
    } else {
        sub_fetch_slow<NB, NW, FOV>(a, pg, level, sub, par, n2, kr, lc.c0, w);
    }
}

// Dequantised values of NW words into out[2 NW].
template <int WAV, int NB, int QM, int NW>
__device__ __forceinline__ void dq_row(const TileArgs &a, const uint32_t (&w)[NB][NW], float s,
                                       typename SV<WAV>::T (&out)[2 * NW]) {
    const int st = (int)a.g.step;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        uint32_t x[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) x[b] = w[b][k];
        dq_word<WAV, NB, QM>(x, a.bands, s, st, out[2 * k], out[2 * k + 1]);
    }
}

// ---- lifting -------------------------------------------------------------------

// Horizontal synthesis of one interleaved row held as N values per lane
// (v[even] low band, v[odd] high band, lanes in column order).
template <int WAV, int N>
__device__ __forceinline__ void hsynth(typename SV<WAV>::T (&v)[N]) {
    using T = typename SV<WAV>::T;
    if constexpr (WAV == 1) {
        float L = __shfl_up_sync(kFull, v[N - 1], 1);
        v[0] = fmaf(-kDelta, L + v[1], v[0]);
#pragma unroll
        for (int m = 2; m < N; m += 2) v[m] = fmaf(-kDelta, v[m - 1] + v[m + 1], v[m]);
        float R = __shfl_down_sync(kFull, v[0], 1);
#pragma unroll
        for (int m = 1; m < N - 1; m += 2) v[m] = fmaf(-kGamma, v[m - 1] + v[m + 1], v[m]);
        v[N - 1] = fmaf(-kGamma, v[N - 2] + R, v[N - 1]);
        L = __shfl_up_sync(kFull, v[N - 1], 1);
        v[0] = fmaf(-kBeta, L + v[1], v[0]);
#pragma unroll
        for (int m = 2; m < N; m += 2) v[m] = fmaf(-kBeta, v[m - 1] + v[m + 1], v[m]);
        R = __shfl_down_sync(kFull, v[0], 1);
#pragma unroll
        for (int m = 1; m < N - 1; m += 2) v[m] = fmaf(-kAlpha, v[m - 1] + v[m + 1], v[m]);
        v[N - 1] = fmaf(-kAlpha, v[N - 2] + R, v[N - 1]);
    } else {
        const T L = __shfl_up_sync(kFull, v[N - 1], 1);
        v[0] -= (L + v[1] + 2) >> 2;
#pragma unroll
        for (int m = 2; m < N; m += 2) v[m] -= (v[m - 1] + v[m + 1] + 2) >> 2;
        const T R = __shfl_down_sync(kFull, v[0], 1);
#pragma unroll
        for (int m = 1; m < N - 1; m += 2) v[m] += (v[m - 1] + v[m + 1]) >> 1;
        v[N - 1] += (v[N - 2] + R) >> 1;
    }
}

// Running vertical synthesis of one column: a pair of interleaved rows
// (e = row i, o = row i + 1) completes rows i - D (returned in oe) and
// i - D + 1 (oo).
template <int WAV>
struct VState;
template <>
struct VState<1> {
    float po, y1, y2, y3;
    __device__ __forceinline__ void clear() { po = y1 = y2 = y3 = 0.f; }
    __device__ __forceinline__ void step(float e, float o, float &oe, float &oo) {
        const float y1k = fmaf(-kDelta, po + o, e);     // even row i:     undo delta
        const float y2m = fmaf(-kGamma, y1 + y1k, po);   // odd row i - 1:  undo gamma
        const float y3m = fmaf(-kBeta, y2 + y2m, y1);    // even row i - 2: undo beta
        oo = fmaf(-kAlpha, y3 + y3m, y2);                // odd row i - 3:  undo alpha
        oe = y3;                                         // even row i - 4 is final
        y3 = y3m;
        y2 = y2m;
        y1 = y1k;
        po = o;
    }
};
template <>
struct VState<0> {
    int po, y1;
    __device__ __forceinline__ void clear() { po = y1 = 0; }
    __device__ __forceinline__ void step(int e, int o, int &oe, int &oo) {
        const int y1k = e - ((po + o + 2) >> 2);   // even row i
        oo = po + ((y1 + y1k) >> 1);               // odd row i - 1
        oe = y1;                                   // even row i - 2
        y1 = y1k;
        po = o;
    }
};

// Running vertical synthesis of N columns.  9/7: adjacent columns run as
// pairs in packed fp32x2 arithmetic (each element rounds exactly as fmaf).
template <int WAV, int N>
struct VCols {
    VState<WAV> s[N];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int c = 0; c < N; ++c) s[c].clear();
    }
    __device__ __forceinline__ void step(const int (&e)[N], const int (&o)[N], int (&oe)[N], int (&oo)[N]) {
#pragma unroll
        for (int c = 0; c < N; ++c) s[c].step(e[c], o[c], oe[c], oo[c]);
    }
};
template <int N>
struct VCols<1, N> {
    float2 po[N / 2], y1[N / 2], y2[N / 2], y3[N / 2];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int c = 0; c < N / 2; ++c) po[c] = y1[c] = y2[c] = y3[c] = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void step(const float (&e)[N], const float (&o)[N], float (&oe)[N],
                                         float (&oo)[N]) {
        const float2 nd = make_float2(-kDelta, -kDelta), ng = make_float2(-kGamma, -kGamma);
        const float2 nb = make_float2(-kBeta, -kBeta), na = make_float2(-kAlpha, -kAlpha);
#pragma unroll
        for (int c = 0; c < N / 2; ++c) {
            const float2 ee = make_float2(e[2 * c], e[2 * c + 1]);
            const float2 o2 = make_float2(o[2 * c], o[2 * c + 1]);
            const float2 y1k = __ffma2_rn(nd, __fadd2_rn(po[c], o2), ee);       // even row i
            const float2 y2m = __ffma2_rn(ng, __fadd2_rn(y1[c], y1k), po[c]);   // odd row i - 1
            const float2 y3m = __ffma2_rn(nb, __fadd2_rn(y2[c], y2m), y1[c]);   // even row i - 2
            const float2 o4 = __ffma2_rn(na, __fadd2_rn(y3[c], y3m), y2[c]);    // odd row i - 3
            oe[2 * c] = y3[c].x;                                                 // even row i - 4
            oe[2 * c + 1] = y3[c].y;
            oo[2 * c] = o4.x;
            oo[2 * c + 1] = o4.y;
            y3[c] = y3m;
            y2[c] = y2m;
            y1[c] = y1k;
            po[c] = o2;
        }
    }
};


// Symmetric extension across the warp: a lane whose N interleaved columns
// c0 .. c0 + N - 1 lie outside the line (active) takes each value from the
// lane holding its mirror image -c (left side) or 2 Wl - 2 - c (right side);
// lane j holds columns Cx + N j .. (Cx, c0 and Wl - Cx multiples of N, so
// the image of position m sits at the same position (-m or -2 - m, mod N)
// in every source lane).  Other lanes keep their values.
template <int N, class T>
__device__ __forceinline__ void mirror_row(T (&v)[N], bool right, int c0, int Cx, int Wl, bool active) {
    constexpr int LG = N == 8 ? 3 : 2;
    const int lane = threadIdx.x & 31;
    T t[N];
    if (right) {
#pragma unroll
        for (int m = 0; m < N; ++m) {
            const int sl = active ? (2 * Wl - 2 - (c0 + m) - Cx) >> LG : lane;
            t[m] = __shfl_sync(kFull, v[(2 * N - 2 - m) % N], sl);
        }
    } else {
#pragma unroll
        for (int m = 0; m < N; ++m) {
            const int sl = active ? (-(c0 + m) - Cx) >> LG : lane;
            t[m] = __shfl_sync(kFull, v[(N - m) % N], sl);
        }
    }
    if (active) {
#pragma unroll
        for (int m = 0; m < N; ++m) v[m] = t[m];
    }
}

// Level 1: a mirror lane's columns that reach a written output are the four
// next to the plane (c0 + 4 .. c0 + 7 left of it, c0 .. c0 + 3 right of
// it); their images are the lane's neighbour's columns 4, 3, 2, 1 (left:
// lane 1 for lane 0) or 6, 5, 4, 3 (right: the lane below).
template <class T>
__device__ __forceinline__ void mirror_l1(T (&v)[8], bool right, bool active) {
    T t[4];
    if (right) {
#pragma unroll
        for (int m = 0; m < 4; ++m) t[m] = __shfl_up_sync(kFull, v[6 - m], 1);
        if (active) {
#pragma unroll
            for (int m = 0; m < 4; ++m) v[m] = t[m];
        }
    } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) t[m] = __shfl_down_sync(kFull, v[4 - m], 1);
        if (active) {
#pragma unroll
            for (int m = 0; m < 4; ++m) v[4 + m] = t[m];
        }
    }
}

// Four integers clamped to [0, 255] and packed into bytes (p0 lowest).
__device__ __forceinline__ uint32_t pack4_sat(int p0, int p1, int p2, int p3) {
    uint32_t hi, d;
    asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, 0;" : "=r"(hi) : "r"(p3), "r"(p2));
    asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(p1), "r"(p0), "r"(hi));
    return d;
}

// ---- one strip tile ---------------------------------------------------------------
//
// Schedule (iteration t = 0 .. P2): the level-2 row pair t (while t < P2)
// and the level-1 row pairs of the two LL_1 rows the level-2 pair t - 1
// completed (t - 1 >= P0).  The two halves of an iteration are independent
// (they meet only through ring rows written one iteration earlier), so
// their dependency chains interleave.  EDGE = false: every lane's columns
// lie inside the plane; EDGE = true: strips touching the plane's left or
// right side (mirror_row, and codes loaded one at a time for the edge lanes
// of planes narrower than 256).

template <int WAV, int NB, int QM, bool EDGE, bool FOV = false>
__device__ __forceinline__ void strip_tile(const TileArgs &a, uint32_t e, float *ring, uint32_t *stage,
                                           int lane) {
    using T = typename SV<WAV>::T;
    using St = Stage<NB>;
    constexpr int D = SV<WAV>::D, P0 = SV<WAV>::P0;
    const Geom &g = a.g;
    const int plane = (int)((e >> 28) & 3);
    const int ty = (int)((e >> 14) & 0x3fff), tx = (int)(e & 0x3fff);
    const PlaneGeom &pg = g.p[plane];
    const int W = pg.w, H = pg.h;            // level-1 interleaved line lengths
    const int W2 = W >> 1, H2 = H >> 1;      // level-2 interleaved line lengths (LL_1 size)
    const int th = (e & kHalfStrip) ? a.th >> 1 : a.th;
    const int X0 = tx * kStripW, Y0 = ty * a.th + ((e & kLowerHalf) ? th : 0);
    const int TH = min(th, H - Y0);
    if (TH <= 0) return;
    // edge strips of planes at least 256 wide touch one side only and find
    // every mirror image in an interior lane of the warp
    const bool wide = W >= 256;
    LaneCols l1, l2;
    l1.c0 = X0 - 8 + 8 * lane;
    l1.kx = l1.c0 >> 1;
    l1.fast = !EDGE || (l1.c0 >= 0 && l1.c0 + 8 <= W);
    l1.zero = EDGE && l1.c0 >= W + 8;
    l1.mirror = EDGE && wide && !l1.fast && !l1.zero;
    l1.scalar = EDGE && !wide && !l1.fast && !l1.zero;
    l2.c0 = (X0 >> 1) - 8 + 4 * lane;
    l2.kx = l2.c0 >> 1;
    l2.fast = !EDGE || (l2.c0 >= 0 && l2.c0 + 4 <= W2);
    l2.zero = EDGE && l2.c0 >= W2 + 8;
    l2.mirror = EDGE && wide && !l2.fast && !l2.zero;
    l2.scalar = EDGE && !wide && !l2.fast && !l2.zero;
    const bool right = X0 > 0;   // an edge strip of a wide plane: its right side, else its left
    const int C2 = (X0 >> 1) - 8;            // LL_1 column of ring column 0
    const float *llp = a.ll_in[plane];
    const int llpitch = a.ll_in_pitch[plane];
    const bool writer = lane >= 1 && lane <= 28 && (!EDGE || l1.c0 + 8 <= W);
    uint8_t *out8 = a.out_u8[plane];
    const int pair_sh = a.out_pair && plane > 0 ? 1 : 0;

    SubRow<NB> r2[4], r1[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        r2[k].by = -1;
        r1[k].by = -1;
    }
    VCols<WAV, 4> v2;
    VCols<WAV, 8> v1;
    v2.clear();
    v1.clear();

    const int n_l1 = TH / 2 + 4;                 // level-1 row pairs (TH a multiple of 4)
    const int P2 = P0 + n_l1 / 2;                // level-2 row pairs
    const int NT = P2 + 1;                       // iterations
    // copies of iteration t: level-2 pair t (sig = Y0/2 - 6 + 2t) and the
    // level-1 pairs k = Y0/2 - 2 + 2(t - 1 - P0) + h
    auto issue = [&](int t) {
        uint32_t *sb = stage + (t % kStages) * St::kWords;
        if (t < P2) {
            const int sig = (Y0 >> 1) - 6 + 2 * t;
            const int ke = refl(sig, H2) >> 1, ko = refl(sig + 1, H2) >> 1;
#if WV_CHECKED
            const bool ll_ok =
                !l2.fast || checked_in((long long)ke * llpitch + l2.kx + 1, (long long)llpitch * (H >> 2), a.err);
            cp_async(St::ll(sb, lane), l2.fast && ll_ok ? llp + (size_t)ke * llpitch + l2.kx : llp, 8,
                     l2.fast && ll_ok);
#else
            cp_async(St::ll(sb, lane), l2.fast ? llp + (size_t)ke * llpitch + l2.kx : llp, 8, l2.fast);
#endif
            const bool ke2 = !FOV || !l2.fast || fov_keep(a, pg, 2, l2.kx, ke);
            const bool ko2 = !FOV || !l2.fast || fov_keep(a, pg, 2, l2.kx, ko);
            sub_issue<NB, 1>(a, pg, 2, 1, ke, l2, r2[1], [&](int b) { return St::l2(sb, 1, b, lane); }, ke2);
            sub_issue<NB, 1>(a, pg, 2, 2, ko, l2, r2[2], [&](int b) { return St::l2(sb, 2, b, lane); }, ko2);
            sub_issue<NB, 1>(a, pg, 2, 3, ko, l2, r2[3], [&](int b) { return St::l2(sb, 3, b, lane); }, ko2);
        }
        if (t - 1 >= P0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = (Y0 >> 1) - 2 + 2 * (t - 1 - P0) + h;
                const int ke1 = refl(2 * k, H) >> 1, ko1 = refl(2 * k + 1, H) >> 1;
                const bool kee = !FOV || !l1.fast || fov_keep(a, pg, 1, l1.kx, ke1);
                const bool koo = !FOV || !l1.fast || fov_keep(a, pg, 1, l1.kx, ko1);
                sub_issue<NB, 2>(a, pg, 1, 1, ke1, l1, r1[1], [&](int b) { return St::l1(sb, h, 1, b, lane); }, kee);
                sub_issue<NB, 2>(a, pg, 1, 2, ko1, l1, r1[2], [&](int b) { return St::l1(sb, h, 2, b, lane); }, koo);
                sub_issue<NB, 2>(a, pg, 1, 3, ko1, l1, r1[3], [&](int b) { return St::l1(sb, h, 3, b, lane); }, koo);
            }
        }
        cp_commit();
    };
#pragma unroll 1
    for (int t = 0; t < kStages - 1; ++t) {
        if (t < NT) issue(t);
        else cp_commit();
    }
#pragma unroll 1
    for (int t = 0; t < NT; ++t) {
        if (t + kStages - 1 < NT) issue(t + kStages - 1);
        else cp_commit();   // an empty group keeps the wait count below uniform
        cp_wait<kStages - 1>();   // this thread's copies of iteration t have landed
        uint32_t *sb = stage + (t % kStages) * St::kWords;
        // ---- level 2: interleaved rows sig (LL_2 | HL_2), sig + 1 (LH_2 | HH_2)
        if (t < P2) {
            const int sig = (Y0 >> 1) - 6 + 2 * t;
            const int ke = refl(sig, H2) >> 1, ko = refl(sig + 1, H2) >> 1;
            T ev[4], od[4];
            {
                T ll[2], hl[2], lh[2], hh[2];
                uint32_t w[NB][1];
                if (!l2.scalar) {
                    const float2 x = *reinterpret_cast<const float2 *>(St::ll(sb, lane));
                    ll[0] = from_f<T>(x.x);
                    ll[1] = from_f<T>(x.y);
                } else {
#pragma unroll
                    for (int m = 0; m < 2; ++m)
#if WV_CHECKED
                    {
                        const long long li = (long long)ke * llpitch + (refl(l2.c0 + 2 * m, W2) >> 1);
                        ll[m] = checked_in(li, (long long)llpitch * (H >> 2), a.err) ? from_f<T>(__ldcg(llp + li))
                                                                                      : T(0);
                    }
#else
                        ll[m] = from_f<T>(__ldcg(llp + (size_t)ke * llpitch + (refl(l2.c0 + 2 * m, W2) >> 1)));
#endif
                }
                sub_fetch<NB, 1, FOV>(a, pg, 2, 1, 1, W2, ke, l2, [&](int b) { return St::l2(sb, 1, b, lane); }, w);
                dq_row<WAV, NB, QM, 1>(a, w, a.scale[2][1], hl);
                sub_fetch<NB, 1, FOV>(a, pg, 2, 2, 0, W2, ko, l2, [&](int b) { return St::l2(sb, 2, b, lane); }, w);
                dq_row<WAV, NB, QM, 1>(a, w, a.scale[2][2], lh);
                sub_fetch<NB, 1, FOV>(a, pg, 2, 3, 1, W2, ko, l2, [&](int b) { return St::l2(sb, 3, b, lane); }, w);
                dq_row<WAV, NB, QM, 1>(a, w, a.scale[2][3], hh);
                ev[0] = ll[0];
                ev[1] = hl[0];
                ev[2] = ll[1];
                ev[3] = hl[1];
                od[0] = lh[0];
                od[1] = hh[0];
                od[2] = lh[1];
                od[3] = hh[1];
            }
            if (EDGE && wide) {
                mirror_row<4>(ev, right, l2.c0, C2, W2, l2.mirror);
                mirror_row<4>(od, right, l2.c0, C2, W2, l2.mirror);
            }
            hsynth<WAV, 4>(ev);
            hsynth<WAV, 4>(od);
            // LL_1 rows sig - D (even) and sig - D + 1 (odd) into the ring
            T oe[4], oo[4];
            v2.step(ev, od, oe, oo);
            float re[4], ro[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                re[c] = to_f<T>(oe[c]);
                ro[c] = to_f<T>(oo[c]);
            }
            const int k0 = sig - D;
            *reinterpret_cast<float4 *>(ring + (k0 & (kRing - 1)) * kRingW + 4 * lane) =
                make_float4(re[0], re[1], re[2], re[3]);
            *reinterpret_cast<float4 *>(ring + ((k0 + 1) & (kRing - 1)) * kRingW + 4 * lane) =
                make_float4(ro[0], ro[1], ro[2], ro[3]);
        }
        // ---- level 1: the LL_1 rows completed in the previous iteration
        if (t - 1 >= P0) {
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                // interleaved rows 2k (LL_1 | HL_1), 2k + 1 (LH_1 | HH_1)
                const int p1 = 2 * (t - 1 - P0) + h;
                const int k = (Y0 >> 1) - 2 + p1;
                const int rho = 2 * k;
                const int ke = refl(rho, H) >> 1, ko = refl(rho + 1, H) >> 1;
                const int kl = k >= H2 ? ke : k;     // LL_1 ring row (see the head comment)
                const float *rr = ring + (kl & (kRing - 1)) * kRingW;
                T ev[8], od[8];
                {
                    T ll[4], hl[4], lh[4], hh[4];
                    // virtual columns left of the plane: ring as is; mirror lanes
                    // are overwritten below
                    if (!EDGE || !l1.scalar || l1.c0 + 8 <= W) {
                        const float4 x = *reinterpret_cast<const float4 *>(rr + (l1.c0 >> 1) - C2);
                        ll[0] = from_f<T>(x.x);
                        ll[1] = from_f<T>(x.y);
                        ll[2] = from_f<T>(x.z);
                        ll[3] = from_f<T>(x.w);
                    } else if (!l1.zero) {
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            const int c = l1.c0 + 2 * m;
                            const int kc = (c < W ? c : refl(c, W)) >> 1;
                            ll[m] = from_f<T>(rr[kc - C2]);
                        }
                    } else {
#pragma unroll
                        for (int m = 0; m < 4; ++m) ll[m] = T(0);
                    }
                    uint32_t w[NB][2];
                    sub_fetch<NB, 2, FOV>(a, pg, 1, 1, 1, W, ke, l1, [&](int b) { return St::l1(sb, h, 1, b, lane); }, w);
                    dq_row<WAV, NB, QM, 2>(a, w, a.scale[1][1], hl);
                    sub_fetch<NB, 2, FOV>(a, pg, 1, 2, 0, W, ko, l1, [&](int b) { return St::l1(sb, h, 2, b, lane); }, w);
                    dq_row<WAV, NB, QM, 2>(a, w, a.scale[1][2], lh);
                    sub_fetch<NB, 2, FOV>(a, pg, 1, 3, 1, W, ko, l1, [&](int b) { return St::l1(sb, h, 3, b, lane); }, w);
                    dq_row<WAV, NB, QM, 2>(a, w, a.scale[1][3], hh);
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        ev[2 * m] = ll[m];
                        ev[2 * m + 1] = hl[m];
                        od[2 * m] = lh[m];
                        od[2 * m + 1] = hh[m];
                    }
                }
                if (EDGE && wide) {
                    mirror_l1(ev, right, l1.mirror);
                    mirror_l1(od, right, l1.mirror);
                }
                hsynth<WAV, 8>(ev);
                hsynth<WAV, 8>(od);
                T oe[8], oo[8];
                v1.step(ev, od, oe, oo);
                const int r0 = rho - D;   // output rows r0 (even) and r0 + 1
                if (writer && r0 >= Y0 && r0 < Y0 + TH) {
#pragma unroll
                    for (int rr2 = 0; rr2 < 2; ++rr2) {
                        const T *v = rr2 ? oo : oe;
                        const size_t o = (size_t)(r0 + rr2) * W + l1.c0;
                        int p[8];
#pragma unroll
                        for (int m = 0; m < 8; ++m) {
                            if constexpr (WAV == 1) p[m] = __float2int_rd(v[m] + 128.5f);
                            else p[m] = v[m] + 128;
                        }
                        // two groups of 4 samples: adjacent, or (chroma groups)
                        // with the other chroma plane's group between them
#if WV_CHECKED
                        if (!checked_in((long long)o + 7, (long long)W * H, a.err)) continue;
#endif
                        uint32_t *d = reinterpret_cast<uint32_t *>(out8 + (o << pair_sh));
                        d[0] = pack4_sat(p[0], p[1], p[2], p[3]);
                        d[1 << pair_sh] = pack4_sat(p[4], p[5], p[6], p[7]);
                    }
                }
            }
        }
        __syncwarp();   // this iteration's ring rows are read by the next one
    }
}

template <int WAV, int NB, int QM>
__global__ void __launch_bounds__(32 * kStripWarps, 3) k_strip(TileArgs a) {
    __shared__ __align__(16) float rings[kStripWarps][kRing * kRingW];
    extern __shared__ __align__(16) uint32_t stages[];   // kStripWarps x kStages x Stage<NB>::kWords
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    float *ring = rings[wi];
    uint32_t *stage = stages + (size_t)wi * kStages * Stage<NB>::kWords;
    for (int i = lane; i < kRing * kRingW; i += 32) ring[i] = 0.f;
    __syncwarp();
    const int count = *(volatile const int *)a.count;
    // tiles are dealt to the CTAs first and to their warps second, so every
    // SM gets the same share of busy warps
    for (int t = blockIdx.x + wi * gridDim.x; t < count; t += kStripWarps * gridDim.x) {
        const uint32_t e = a.tiles[t];
        if (strip_interior((int)(e & 0x3fff), a.g.p[(e >> 28) & 3].w))
            strip_tile<WAV, NB, QM, false>(a, e, ring, stage, lane);
        else
            strip_tile<WAV, NB, QM, true>(a, e, ring, stage, lane);
    }
}

template <int WAV, int NB, int QM>
cudaError_t launch_s(const TileArgs &a, cudaStream_t cs) {
    // stage memory is fixed per instantiation: opt in once per device
    static std::once_flag once[64];
    static cudaError_t set_err[64];
    const int smem = kStripWarps * kStages * Stage<NB>::kWords * 4;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::call_once(once[dev], [&] {
        set_err[dev] = cudaFuncSetAttribute(k_strip<WAV, NB, QM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
    if (set_err[dev] != cudaSuccess) return set_err[dev];
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_strip<WAV, NB, QM>, 32 * kStripWarps, smem);
    if (e != cudaSuccess) return e;
    k_strip<WAV, NB, QM><<<sms * std::max(per_sm, 1), 32 * kStripWarps, smem, cs>>>(a);
    return cudaGetLastError();
}

template <int WAV, int QM>
cudaError_t launch_nb(const TileArgs &a, cudaStream_t cs) {
    switch (a.bands.n) {
    case 1: return launch_s<WAV, 1, QM>(a, cs);
    case 2: return launch_s<WAV, 2, QM>(a, cs);
    case 3: return launch_s<WAV, 3, QM>(a, cs);
    default: return launch_s<WAV, 4, QM>(a, cs);
    }
}

// Batched decoding: the strip tiles of the decode targets ("surfaces") of
// one decode class in one launch, after their coarse tiles (another launch).
// List entries are (surface, strip entry); a tile reads its surface's
// arguments from the job table (read-only, through the cache).
template <int WAV, int NB, int QM, bool FOV>
__global__ void __launch_bounds__(32 * kStripWarps, 3)
    k_strip_batch(const SurfaceJob *__restrict__ surfs, const uint2 *__restrict__ list, const int *count_p) {
    __shared__ __align__(16) float rings[kStripWarps][kRing * kRingW];
    extern __shared__ __align__(16) uint32_t stages[];   // kStripWarps x kStages x Stage<NB>::kWords
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    float *ring = rings[wi];
    uint32_t *stage = stages + (size_t)wi * kStages * Stage<NB>::kWords;
    for (int i = lane; i < kRing * kRingW; i += 32) ring[i] = 0.f;
    __syncwarp();
    const int count = *(volatile const int *)count_p;
    for (int t = blockIdx.x + wi * gridDim.x; t < count; t += kStripWarps * gridDim.x) {
        const uint2 it = list[t];
        const TileArgs &a = surfs[it.x].fine;
        const uint32_t e = it.y;
        if (strip_interior((int)(e & 0x3fff), a.g.p[(e >> 28) & 3].w))
            strip_tile<WAV, NB, QM, false, FOV>(a, e, ring, stage, lane);
        else
            strip_tile<WAV, NB, QM, true, FOV>(a, e, ring, stage, lane);
    }
}

template <int WAV, int NB, int QM, bool FOV>
cudaError_t launch_b(const SurfaceJob *surfs, const uint2 *list, const int *count, cudaStream_t cs) {
    static std::once_flag once[64];
    static cudaError_t set_err[64];
    const int smem = kStripWarps * kStages * Stage<NB>::kWords * 4;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::call_once(once[dev], [&] {
        set_err[dev] =
            cudaFuncSetAttribute(k_strip_batch<WAV, NB, QM, FOV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
    if (set_err[dev] != cudaSuccess) return set_err[dev];
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_strip_batch<WAV, NB, QM, FOV>,
                                                                  32 * kStripWarps, smem);
    if (e != cudaSuccess) return e;
    k_strip_batch<WAV, NB, QM, FOV><<<sms * std::max(per_sm, 1), 32 * kStripWarps, smem, cs>>>(surfs, list, count);
    return cudaGetLastError();
}

}  // namespace

bool strip_batch_supported(int wavelet, int nb, bool dz_t) {
    return nb >= 1 && nb <= 2 && (wavelet == WV_WAVELET_53 || dz_t);
}

cudaError_t launch_decode_strips_batch(int wavelet, int nb, bool fovea, bool dz_t, const SurfaceJob *surfs,
                                       const uint2 *list, const int *count, cudaStream_t cs) {
    if (!strip_batch_supported(wavelet, nb, dz_t)) return cudaErrorInvalidValue;
    if (wavelet == WV_WAVELET_97) {
        if (nb == 1) return fovea ? launch_b<1, 1, 2, true>(surfs, list, count, cs)
                                  : launch_b<1, 1, 2, false>(surfs, list, count, cs);
        return fovea ? launch_b<1, 2, 2, true>(surfs, list, count, cs) : launch_b<1, 2, 2, false>(surfs, list, count, cs);
    }
    if (nb == 1) return fovea ? launch_b<0, 1, 0, true>(surfs, list, count, cs)
                              : launch_b<0, 1, 0, false>(surfs, list, count, cs);
    return fovea ? launch_b<0, 2, 0, true>(surfs, list, count, cs) : launch_b<0, 2, 0, false>(surfs, list, count, cs);
}

// Levels 2 and 1 of the listed strip tiles, LL_2 from the planes written by
// the coarse pass (streams of three or more levels).
cudaError_t launch_decode_strips(const Geom &g, const int16_t *payload, const int32_t *table,
                                 const Bands &bands, const float *const *ll2, const int *ll2_pitch,
                                 uint8_t *const *out_u8, float *out_f32, int f32_plane,
                                 const uint32_t *tiles, int *counters, int *err, cudaStream_t cs,
                                 bool chroma_pairs) {
    if (chroma_pairs && (g.planes != 3 || out_u8[2] != out_u8[1] + 4 || ((uintptr_t)out_u8[1] & 15)))
        return cudaErrorInvalidValue;
    TileArgs a;
    memset(&a, 0, sizeof(a));
    a.g = g;
    a.payload = payload;
    a.table = table;
    a.bands = bands;
    a.err = err;
    a.l_top = 2;
    a.l_bot = 1;
    a.tw = g.tw;
    a.th = g.th;
    for (int p = 0; p < 3; ++p) {
        a.ll_in[p] = ll2 ? ll2[p] : nullptr;
        a.ll_in_pitch[p] = ll2 ? ll2_pitch[p] : 0;
        a.out_u8[p] = out_u8[p];
    }
    // 8-bit samples only (float output takes the square-tile pass): the
    // float store path cost the kernel 16 spilled bytes and 9 % of its time
    if (out_f32) return cudaErrorInvalidValue;
    (void)f32_plane;
    a.out_pair = chroma_pairs ? 1 : 0;
    a.tiles = tiles;
    a.count = counters;
    a.work = counters + 2;
    fill_tile_scales(a);
    if (!g.strip || g.levels < 3 || g.quant != 0 || !ll2) return cudaErrorInvalidValue;
    if (g.wavelet == WV_WAVELET_97) return g.dz_t ? launch_nb<1, 2>(a, cs) : launch_nb<1, 0>(a, cs);
    return launch_nb<0, 0>(a, cs);
}

}  // namespace wv
