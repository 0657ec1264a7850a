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

__device__ __forceinline__ Taps bilinear_taps(int w, int r_lo, int r_n, float u, float v) {
    int x0, fx, y0, fy;
    fixed_split(u, x0, fx);
    fixed_split(v, y0, fy);
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

// Y, Cb, Cr of luma position (u, v); Cb and Cr share their taps.  Rows
// clamp to the eye's part of the frame (all of it for mono streams).
__device__ __forceinline__ void sample_ycbcr(const ResampleArgs &a, float u, float v, int &y, int &cb,
                                             int &cr) {
    y = blend(a.plane[0], bilinear_taps(a.w[0], a.v.row0, a.v.rows, u, v));
    cb = cr = 128;
    if (a.planes == 3) {
        float uc = u, vc = v;
        if (a.c420) {
            uc = fmaf(u + 0.5f, 0.5f, -0.5f);
            vc = fmaf(v + 0.5f, 0.5f, -0.5f);
        }
        const int sh = a.c420 ? 1 : 0;
        const Taps t = bilinear_taps(a.w[1], a.v.row0 >> sh, a.v.rows >> sh, uc, vc);
        cb = blend(a.plane[1], t);
        cr = blend(a.plane[2], t);
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

// Two horizontally adjacent pixels (i, j), (i + 1, j) per thread
// (independent work for the scheduler to overlap), written with one 8-byte
// store when aligned.
__device__ __forceinline__ void resample_pair(const ResampleArgs &a, int i, int j) {
    if (i >= a.v.out_w || j >= a.v.out_h) return;
    if (a.y_plane) {
        sample_ycc(a, i, j);
        if (i + 1 < a.v.out_w) sample_ycc(a, i + 1, j);
        return;
    }
    const bool two = i + 1 < a.v.out_w;
    float u0, v0, u1 = 0.f, v1 = 0.f;
    if (a.uv) {
        const float2 *row = reinterpret_cast<const float2 *>(a.uv) + (size_t)j * a.v.out_w;
        const float2 p0 = row[i];
        u0 = p0.x;
        v0 = p0.y;
        if (two) {
            const float2 p1 = row[i + 1];
            u1 = p1.x;
            v1 = p1.y;
        }
    } else {
        project_px(a.v, i, j, u0, v0);
        if (two) project_px(a.v, i + 1, j, u1, v1);
    }
    const uchar4 c0 = sample_px(a, u0, v0);
    uchar4 *dst = reinterpret_cast<uchar4 *>(a.out + (size_t)j * a.pitch) + i;
    if (two) {
        const uchar4 c1 = sample_px(a, u1, v1);
        if ((reinterpret_cast<uintptr_t>(dst) & 7) == 0) {
            uint2 w;
            w.x = (uint32_t)c0.x | ((uint32_t)c0.y << 8) | ((uint32_t)c0.z << 16) | ((uint32_t)c0.w << 24);
            w.y = (uint32_t)c1.x | ((uint32_t)c1.y << 8) | ((uint32_t)c1.z << 16) | ((uint32_t)c1.w << 24);
            *reinterpret_cast<uint2 *>(dst) = w;
        } else {
            dst[0] = c0;
            dst[1] = c1;
        }
    } else {
        dst[0] = c0;
    }
}

__global__ void k_resample(ResampleArgs a) {
    resample_pair(a, 2 * (blockIdx.x * blockDim.x + threadIdx.x), blockIdx.y * blockDim.y + threadIdx.y);
}

// Batch: one z-slice of the grid per request.
__global__ void k_resample_batch(const RequestJob *__restrict__ reqs) {
    const ResampleArgs &a = reqs[blockIdx.z].rs;
    resample_pair(a, 2 * (blockIdx.x * blockDim.x + threadIdx.x), blockIdx.y * blockDim.y + threadIdx.y);
}

}  // namespace

void launch_resample(const Geom &g, const View &v, uint8_t *const *recon, const float *uv,
                     uint8_t *out, size_t pitch, cudaStream_t cs, float *y_plane,
                     uint8_t *cb_plane, uint8_t *cr_plane) {
    ResampleArgs a;
    memset(&a, 0, sizeof(a));
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
    a.uv = uv;
    a.out = out;
    a.pitch = pitch;
    dim3 block(32, 8);
    dim3 grid((v.out_w + 63) / 64, (v.out_h + 7) / 8);
    k_resample<<<grid, block, 0, cs>>>(a);
}

void launch_resample_batch(const RequestJob *reqs, int n, int max_w, int max_h, cudaStream_t cs) {
    dim3 block(32, 8);
    dim3 grid((max_w + 63) / 64, (max_h + 7) / 8, n);
    k_resample_batch<<<grid, block, 0, cs>>>(reqs);
}

}  // namespace wv
