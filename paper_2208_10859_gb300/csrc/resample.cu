// resample.cu -- reprojection of the decoded equirectangular region into the
// viewport (Sec. 3.6: a mapping pass after the inverse wavelet transform) and
// YCbCr -> RGBA conversion.
//
// Per viewport pixel: the same projection as the footprint kernel gives the
// luma position (u, v); u wraps around the longitude seam, v clamps at the
// poles.  Bilinear filtering in fixed point: the fraction is rounded to 1/256
// (half up, with carry), the four integer weights sum to 65536 and the result
// is (sum + 32768) >> 16.  Chroma (4:2:0, centre-sited) is sampled at
// ((u + 1/2) / 2 - 1/2, (v + 1/2) / 2 - 1/2).  Colour: BT.709 full range,
// coefficients rounded to 1/65536, result rounded half up and clamped.
// The paper itself stores no colour transform (Sec. 5); the YCbCr 4:2:0
// stream and this conversion belong to this decoder's format.
#include <string.h>

#include "wv_impl.h"

namespace wv {

namespace {

// The 2 x 2 taps of a bilinear sample of a w x h plane at (u, v): x wraps
// (projected positions lie in [-1/2, w - 1/2), so one conditional add
// suffices; other positions take a modulo), y clamps.  Offsets into the
// row-major plane (planes are < 2^31 bytes) and 1/256 weights.
struct Taps {
    int a0, a1, b0, b1;   // (ya, xa), (ya, xb), (yb, xa), (yb, xb)
    int fx, fy;
};

// fixed_split for |t| < 2^15 (every projected position): there t * 256 +
// 1/2 is exact in float32, so floor(t * 256 + 1/2) = 256 i + f, the carry
// included, and one rounding conversion gives both parts.
__device__ __forceinline__ void fixed_split_near(float t, int &i, int &f) {
    const int T = __float2int_rd(fmaf(t, 256.0f, 0.5f));
    i = T >> 8;
    f = T & 255;
}

__device__ __forceinline__ Taps bilinear_taps(int w, int r_lo, int r_n, float u, float v) {
    int x0, fx, y0, fy;
    if (fabsf(u) < 32768.0f && fabsf(v) < 32768.0f) {
        fixed_split_near(u, x0, fx);
        fixed_split_near(v, y0, fy);
    } else {
        fixed_split(u, x0, fx);
        fixed_split(v, y0, fy);
    }
    Taps t;
    t.fx = fx;
    t.fy = fy;
    if ((unsigned)x0 < (unsigned)(w - 1) && y0 >= r_lo && y0 < r_lo + r_n - 1) {   // no wrap, no clamp
        t.a0 = y0 * w + x0;
        t.a1 = t.a0 + 1;
        t.b0 = t.a0 + w;
        t.b1 = t.b0 + 1;
        return t;
    }
    int xa = x0;
    if (xa < 0) xa += w;
    else if (xa >= w) xa -= w;
    if ((unsigned)xa >= (unsigned)w) {   // positions far outside (caller-given)
        xa %= w;
        if (xa < 0) xa += w;
    }
    const int xb = (xa + 1 == w) ? 0 : xa + 1;
    const int ya = min(max(y0, r_lo), r_lo + r_n - 1) * w;
    const int yb = min(max(y0 + 1, r_lo), r_lo + r_n - 1) * w;
    t.a0 = ya + xa;
    t.a1 = ya + xb;
    t.b0 = yb + xa;
    t.b1 = yb + xb;
    return t;
}

__device__ __forceinline__ int blend(const uint8_t *__restrict__ img, const Taps &t) {
    const int p00 = __ldg(img + t.a0), p01 = __ldg(img + t.a1);
    const int p10 = __ldg(img + t.b0), p11 = __ldg(img + t.b1);
    const int wx1 = t.fx, wx0 = 256 - t.fx;
    const int top = wx0 * p00 + wx1 * p01, bot = wx0 * p10 + wx1 * p11;
    return ((256 - t.fy) * top + t.fy * bot + 32768) >> 16;
}

// Cb and Cr of chroma sample e (row-major index) from a plane of
// alternating 4-sample groups (Cb of positions 4k..4k+3, then Cr of the
// same positions): one 8-byte load.
__device__ __forceinline__ uint2 tap_pair(const uint8_t *__restrict__ img, int e) {
    const uint2 q = __ldg(reinterpret_cast<const uint2 *>(img + 2 * (e & ~3)));
    const int sh = 8 * (e & 3);
    return make_uint2((q.x >> sh) & 255u, (q.y >> sh) & 255u);
}

// Cb and Cr of one tap set: four 8-byte loads instead of eight byte loads.
__device__ __forceinline__ void blend_pair(const uint8_t *__restrict__ img, const Taps &t, int &cb, int &cr) {
    const uint2 p00 = tap_pair(img, t.a0), p01 = tap_pair(img, t.a1);
    const uint2 p10 = tap_pair(img, t.b0), p11 = tap_pair(img, t.b1);
    const int wx1 = t.fx, wx0 = 256 - t.fx;
    const int tb = wx0 * (int)p00.x + wx1 * (int)p01.x, bb = wx0 * (int)p10.x + wx1 * (int)p11.x;
    const int tr = wx0 * (int)p00.y + wx1 * (int)p01.y, br = wx0 * (int)p10.y + wx1 * (int)p11.y;
    cb = ((256 - t.fy) * tb + t.fy * bb + 32768) >> 16;
    cr = ((256 - t.fy) * tr + t.fy * br + 32768) >> 16;
}

// Y, Cb, Cr of luma position (u, v); Cb and Cr share their taps.  Rows
// clamp to the eye's part of the frame (all of it for mono streams).
// WV_CHECKED builds: every tap offset inside the w x h plane.
__device__ __forceinline__ bool taps_in(const Taps &t, int w, int h, int *err) {
    const long long n = (long long)w * h;
    return checked_in(t.a0, n, err) && checked_in(t.a1, n, err) && checked_in(t.b0, n, err) &&
           checked_in(t.b1, n, err);
}

__device__ __forceinline__ void sample_ycbcr(const ResampleArgs &a, float u, float v, int &y, int &cb,
                                             int &cr) {
    const Taps ty = bilinear_taps(a.w[0], a.v.row0, a.v.rows, u, v);
    y = !kChecked || taps_in(ty, a.w[0], a.h[0], a.err) ? blend(a.plane[0], ty) : 0;
    cb = cr = 128;
    if (a.planes == 3) {
        float uc = u, vc = v;
        if (a.c420) {
            uc = fmaf(u + 0.5f, 0.5f, -0.5f);
            vc = fmaf(v + 0.5f, 0.5f, -0.5f);
        }
        const int sh = a.c420 ? 1 : 0;
        const Taps t = bilinear_taps(a.w[1], a.v.row0 >> sh, a.v.rows >> sh, uc, vc);
        if (kChecked && !taps_in(t, a.w[1], a.h[1], a.err)) return;
        if (a.c_pair) {
            blend_pair(a.plane[1], t, cb, cr);
        } else {
            cb = blend(a.plane[1], t);
            cr = blend(a.plane[2], t);
        }
    }
}

__device__ __forceinline__ uchar4 sample_px(const ResampleArgs &a, float u, float v) {
    int y, cb, cr;
    sample_ycbcr(a, u, v, y, cb, cr);
    return to_rgba(y, cb, cr);
}

// Luma / 255, Cb and Cr of viewport pixel (i, j) into the planes.
__device__ __forceinline__ void sample_ycc(const ResampleArgs &a, int i, int j) {
    float u, v;
    project_px(a.v, i, j, u, v);
    int y, cb, cr;
    sample_ycbcr(a, u, v, y, cb, cr);
    const size_t o = (size_t)j * a.v.out_w + i;
    a.y_plane[o] = (float)y * (1.0f / 255.0f);
    a.cb_plane[o] = (uint8_t)cb;
    a.cr_plane[o] = (uint8_t)cr;
}

__device__ __forceinline__ uint32_t rgba_word(uchar4 c) {
    return (uint32_t)c.x | ((uint32_t)c.y << 8) | ((uint32_t)c.z << 16) | ((uint32_t)c.w << 24);
}

__device__ __forceinline__ void position(const ResampleArgs &a, int i, int j, float &u, float &v) {
    if (a.uv) {
        const float2 p = reinterpret_cast<const float2 *>(a.uv)[(size_t)j * a.v.out_w + i];
        u = p.x;
        v = p.y;
    } else {
        project_px(a.v, i, j, u, v);
    }
}

// kPx horizontally adjacent pixels (i .. i + kPx - 1, j) per thread
// (independent work for the scheduler to overlap), written with one
// 4 kPx-byte store when the row holds all of them and the address is
// aligned.
constexpr int kPx = 2;

__device__ __forceinline__ void resample_run(const ResampleArgs &a, int i, int j) {
    if (i >= a.v.out_w || j >= a.v.out_h) return;
    if (a.y_plane) {
        for (int k = 0; k < kPx && i + k < a.v.out_w; ++k) sample_ycc(a, i + k, j);
        return;
    }
    uchar4 *dst = reinterpret_cast<uchar4 *>(a.out + (size_t)j * a.pitch) + i;
    if (i + kPx <= a.v.out_w && (reinterpret_cast<uintptr_t>(dst) & (4 * kPx - 1)) == 0) {
        uint32_t w[kPx];
#pragma unroll
        for (int k = 0; k < kPx; ++k) {
            float u, v;
            position(a, i + k, j, u, v);
            w[k] = rgba_word(sample_px(a, u, v));
        }
        if constexpr (kPx == 4) *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
        else if constexpr (kPx == 2) *reinterpret_cast<uint2 *>(dst) = make_uint2(w[0], w[1]);
        else *reinterpret_cast<uint32_t *>(dst) = w[0];
        return;
    }
    for (int k = 0; k < kPx && i + k < a.v.out_w; ++k) {
        float u, v;
        position(a, i + k, j, u, v);
        dst[k] = sample_px(a, u, v);
    }
}

__global__ void k_resample(ResampleArgs a) {
    resample_run(a, kPx * (blockIdx.x * blockDim.x + threadIdx.x), blockIdx.y * blockDim.y + threadIdx.y);
}

// Batch: one z-slice of the grid per request.
__global__ void k_resample_batch(const RequestJob *__restrict__ reqs) {
    const ResampleArgs &a = reqs[blockIdx.z].rs;
    resample_run(a, kPx * (blockIdx.x * blockDim.x + threadIdx.x), blockIdx.y * blockDim.y + threadIdx.y);
}

}  // namespace

void launch_resample(const Geom &g, const View &v, uint8_t *const *recon, const float *uv,
                     uint8_t *out, size_t pitch, cudaStream_t cs, float *y_plane,
                     uint8_t *cb_plane, uint8_t *cr_plane, bool c_pair, int *err) {
    ResampleArgs a;
    memset(&a, 0, sizeof(a));
    a.err = err;
    a.y_plane = y_plane;
    a.cb_plane = cb_plane;
    a.cr_plane = cr_plane;
    a.v = v;
    for (int p = 0; p < 3; ++p) {
        a.plane[p] = recon[p];
        a.w[p] = p < g.planes ? g.p[p].w : 0;
        a.h[p] = p < g.planes ? g.p[p].h : 0;
    }
    a.planes = g.planes;
    a.c420 = g.c420;
    a.c_pair = c_pair && g.planes == 3 ? 1 : 0;
    a.uv = uv;
    a.out = out;
    a.pitch = pitch;
    dim3 block(32, 8);
    dim3 grid((v.out_w + 32 * kPx - 1) / (32 * kPx), (v.out_h + 7) / 8);
    k_resample<<<grid, block, 0, cs>>>(a);
}

void launch_resample_batch(const RequestJob *reqs, int n, int max_w, int max_h, cudaStream_t cs) {
    dim3 block(32, 8);
    dim3 grid((max_w + 32 * kPx - 1) / (32 * kPx), (max_h + 7) / 8, n);
    k_resample_batch<<<grid, block, 0, cs>>>(reqs);
}

}  // namespace wv
