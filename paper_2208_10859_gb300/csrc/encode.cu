// encode.cu -- GPU encoder of the wavelet video stream (offline; not on the
// decode path).
//
// Per frame and plane: DC shift by 128 and the 2D forward FWT, level by level
// (columns, then rows, in place, Mallat layout; Sec. 3.1), in float32 for
// CDF 9/7 (the paper transforms 32-bit floats, Sec. 3.3) and int32 for the
// reversible LeGall 5/3.  Per inter-frame set of 2^k frames: the Haar
// transform along time, run to the last level (Sec. 3.2), followed by the
// dead-zone quantiser q = sign(c) floor(|c| / step).  Blocks whose quantised
// coefficients are all zero are omitted (Sec. 3.4 loads only stored blocks).
// Simple line-per-thread kernels: the encoder is not timed.
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "wv_impl.h"

namespace wv {

namespace {

constexpr float kAlpha = -1.586134342059924f;
constexpr float kBeta = -0.052980118572961f;
constexpr float kGamma = 0.882911075530934f;
constexpr float kDelta = 0.443506852043971f;
constexpr float kKf = 1.230174104914001f;

__device__ __forceinline__ int refl(int i, int n) { return i < 0 ? -i : (i >= n ? 2 * (n - 1) - i : i); }

// Forward 1D transform of `lines` lines of n samples: element m of line q is
// a[q * lstride + m * estride].  Results go to tmp in the same addressing as
// [s | d] and are then copied back.
template <typename T>
__global__ void k_fwd_lines(T *a, T *tmp, int lines, int n, size_t lstride, size_t estride,
                            int wavelet) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= lines) return;
    T *y = a + (size_t)q * lstride;
    auto at = [&](int m) -> T & { return y[(size_t)m * estride]; };
    if (wavelet == WV_WAVELET_97) {
        const float c[4] = {kAlpha, kBeta, kGamma, kDelta};
        for (int step = 0; step < 4; ++step) {
            const int par = (step & 1) ? 0 : 1;   // alpha/gamma update odd samples
            for (int m = par; m < n; m += 2)
                at(m) = (T)((float)at(m) + c[step] * ((float)at(refl(m - 1, n)) + (float)at(refl(m + 1, n))));
        }
    } else {
        for (int m = 1; m < n; m += 2) {
            const int s = (int)at(refl(m - 1, n)) + (int)at(refl(m + 1, n));
            at(m) = (T)((int)at(m) - (s >> 1));
        }
        for (int m = 0; m < n; m += 2) {
            const int s = (int)at(refl(m - 1, n)) + (int)at(refl(m + 1, n)) + 2;
            at(m) = (T)((int)at(m) + (s >> 2));
        }
    }
    T *t = tmp + (size_t)q * lstride;
    for (int m = 0; m < n / 2; ++m) {
        T s = at(2 * m), d = at(2 * m + 1);
        if (wavelet == WV_WAVELET_97) {
            s = (T)((float)s / kKf);
            d = (T)((float)d * kKf);
        }
        t[(size_t)m * estride] = s;
        t[(size_t)(n / 2 + m) * estride] = d;
    }
    for (int m = 0; m < n; ++m) at(m) = t[(size_t)m * estride];
}

template <typename T>
__global__ void k_load_plane(const uint8_t *src, T *dst, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (T)((int)src[i] - 128);
}

// Inter-frame Haar over the n = 2^k planes work[j], then quantisation into
// the coefficient frames out[slot] (slot order L_k, H_k, H_{k-1}[..], ...).
template <typename T>
__global__ void k_haar_quant(const T *work, size_t plane_elems, int k, float step,
                             int16_t *const *out, size_t n_elems, int *err) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_elems) return;
    const int n = 1 << k;
    T low[8];
    T bands[8];
    for (int j = 0; j < n; ++j) low[j] = work[(size_t)j * plane_elems + i];
    int cnt = n;
    int slot_end = n;
    for (int j = 1; j <= k; ++j) {
        const int half = cnt / 2;
        slot_end -= half;   // details of level j occupy slots [slot_end, slot_end + half)
        for (int m = 0; m < half; ++m) {
            const T a = low[2 * m], b = low[2 * m + 1];
            T l, h;
            if constexpr (std::is_floating_point<T>::value) {
                l = (a + b) * (T)0.5f;
                h = (b - a) * (T)0.5f;
            } else {
                h = b - a;
                l = a + (h >> 1);
            }
            bands[slot_end + m] = h;
            low[m] = l;
        }
        cnt = half;
    }
    bands[0] = low[0];
    for (int s = 0; s < n; ++s) {
        int q;
        if constexpr (std::is_floating_point<T>::value) {
            const float c = (float)bands[s];
            const float m = floorf(fabsf(c) / step);
            if (m > 32767.f) { atomicCAS(err, 0, WV_ERR_RANGE); q = 0; }
            else q = c < 0.f ? -(int)m : (int)m;
        } else {
            const int c = (int)bands[s];
            const int st = (int)step;
            const int m = (c < 0 ? -c : c) / st;
            if (m > 32767) { atomicCAS(err, 0, WV_ERR_RANGE); q = 0; }
            else q = c < 0 ? -m : m;
        }
        out[s][i] = (int16_t)q;
    }
}

struct BlockDesc {
    int plane, x0, y0, bw, bh;
};

__global__ void k_block_flags(int16_t *const *coef, const BlockDesc *desc, const int *plane_w,
                              const size_t *plane_off, int nbpf, int *flags) {
    const int t = blockIdx.y, b = blockIdx.x;
    const BlockDesc d = desc[b];
    const int16_t *c = coef[t] + plane_off[d.plane];
    const int w = plane_w[d.plane];
    int any = 0;
    for (int idx = threadIdx.x; idx < d.bw * d.bh && !any; idx += blockDim.x) {
        const int y = idx / d.bw, x = idx % d.bw;
        any = c[(size_t)(d.y0 + y) * w + d.x0 + x] != 0;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) flags[t * nbpf + b] = any;
}

__global__ void k_pack(int16_t *const *coef, const BlockDesc *desc, const int *plane_w,
                       const size_t *plane_off, int nbpf, const int *slots, int B,
                       int16_t *payload) {
    const int t = blockIdx.y, b = blockIdx.x;
    const int slot = slots[t * nbpf + b];
    if (slot < 0) return;
    const BlockDesc d = desc[b];
    const int16_t *c = coef[t] + plane_off[d.plane];
    const int w = plane_w[d.plane];
    int16_t *o = payload + (size_t)slot * B * B;
    for (int idx = threadIdx.x; idx < B * B; idx += blockDim.x) {
        const int y = idx / B, x = idx % B;
        o[idx] = (x < d.bw && y < d.bh) ? c[(size_t)(d.y0 + y) * w + d.x0 + x] : (int16_t)0;
    }
}

struct ScratchLayout {
    size_t work, tmp, coef, flags, desc, misc, payload, total;
    size_t plane_elems_max, coef_frame_elems;
};

ScratchLayout scratch_layout(const Geom &g) {
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    ScratchLayout s;
    const int n = 1 << g.tlevels;
    s.plane_elems_max = (size_t)g.p[0].w * g.p[0].h;
    s.coef_frame_elems = 0;
    for (int p = 0; p < g.planes; ++p) s.coef_frame_elems += (size_t)g.p[p].w * g.p[p].h;
    size_t o = 0;
    s.work = o;
    o = al(o + (size_t)n * s.plane_elems_max * 4);
    s.tmp = o;
    o = al(o + s.plane_elems_max * 4);
    s.coef = o;
    o = al(o + (size_t)g.num_frames * s.coef_frame_elems * 2);
    s.flags = o;
    o = al(o + (size_t)g.num_frames * g.nbpf * 4);
    s.desc = o;
    o = al(o + (size_t)g.nbpf * sizeof(BlockDesc));
    s.misc = o;   // err, plane widths, plane offsets, coef frame pointers
    o = al(o + 4096 + (size_t)g.num_frames * sizeof(void *));
    s.payload = o;
    if (g.quant == 1)   // paper format: record start per block, then at most one record per coefficient
        o = al(o + (size_t)g.num_frames * g.nbpf * 8 + (size_t)g.num_frames * s.coef_frame_elems * 4);
    else
        o = al(o + (size_t)g.num_frames * g.nbpf * g.block * g.block * 2);
    s.total = o;
    return s;
}

std::vector<BlockDesc> block_descs(const Geom &g) {
    std::vector<BlockDesc> v;
    const int B = g.block;
    for (int p = 0; p < g.planes; ++p) {
        const PlaneGeom &pg = g.p[p];
        const int L = g.levels;
        auto add = [&](int x0, int y0, int sw, int sh) {
            for (int by = 0; by < sh; by += B)
                for (int bx = 0; bx < sw; bx += B)
                    v.push_back({p, x0 + bx, y0 + by, std::min(B, sw - bx), std::min(B, sh - by)});
        };
        add(0, 0, pg.w >> L, pg.h >> L);
        for (int l = L; l >= 1; --l) {
            const int sw = pg.w >> l, sh = pg.h >> l;
            add(sw, 0, sw, sh);
            add(0, sh, sw, sh);
            add(sw, sh, sw, sh);
        }
    }
    return v;
}

template <typename T>
cudaError_t transform_plane(T *a, T *tmp, int w, int h, int levels, int wavelet, cudaStream_t cs) {
    for (int l = 0; l < levels; ++l) {
        const int cw = w >> l, ch = h >> l;
        // columns: line q = column q, elements strided by the row pitch w
        k_fwd_lines<T><<<(cw + 127) / 128, 128, 0, cs>>>(a, tmp, cw, ch, 1, (size_t)w, wavelet);
        // rows: line q = row q, contiguous elements
        k_fwd_lines<T><<<(ch + 127) / 128, 128, 0, cs>>>(a, tmp, ch, cw, (size_t)w, 1, wavelet);
    }
    return cudaGetLastError();
}

template <typename T>
int run(const Geom &g, const void *const *planes, char *base, const ScratchLayout &S, void *out,
        size_t cap, size_t *out_len, cudaStream_t cs) {
    const int n = 1 << g.tlevels;
    T *work = (T *)(base + S.work);
    T *tmp = (T *)(base + S.tmp);
    int16_t *coef = (int16_t *)(base + S.coef);
    int *flags = (int *)(base + S.flags);
    BlockDesc *desc = (BlockDesc *)(base + S.desc);
    int *err = (int *)(base + S.misc);
    int *plane_w = (int *)(base + S.misc + 64);
    size_t *plane_off = (size_t *)(base + S.misc + 128);
    int16_t **coef_ptrs = (int16_t **)(base + S.misc + 4096);
    int16_t *payload = (int16_t *)(base + S.payload);

    const std::vector<BlockDesc> bd = block_descs(g);
    if ((int)bd.size() != g.nbpf) return WV_ERR_ARG;
    std::vector<int16_t *> cptr(g.num_frames);
    for (int t = 0; t < g.num_frames; ++t) cptr[t] = coef + (size_t)t * S.coef_frame_elems;
    int pw[3] = {0, 0, 0};
    size_t poff[3] = {0, 0, 0};
    size_t acc = 0;
    for (int p = 0; p < g.planes; ++p) {
        pw[p] = g.p[p].w;
        poff[p] = acc;
        acc += (size_t)g.p[p].w * g.p[p].h;
    }
    cudaError_t e = cudaMemsetAsync(err, 0, 4, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(desc, bd.data(), bd.size() * sizeof(BlockDesc), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(plane_w, pw, sizeof(pw), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(plane_off, poff, sizeof(poff), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(coef_ptrs, cptr.data(), cptr.size() * sizeof(void *), cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return WV_ERR_CUDA;

    std::vector<int16_t *> outp(8);
    for (int set = 0; set < g.num_frames / n && e == cudaSuccess; ++set) {
        for (int p = 0; p < g.planes && e == cudaSuccess; ++p) {
            const size_t ne = (size_t)g.p[p].w * g.p[p].h;
            for (int j = 0; j < n; ++j) {
                const uint8_t *src = (const uint8_t *)planes[(size_t)(set * n + j) * g.planes + p];
                if (!src) return WV_ERR_ARG;
                k_load_plane<T><<<(unsigned)((ne + 255) / 256), 256, 0, cs>>>(src, work + (size_t)j * S.plane_elems_max, ne);
                e = transform_plane<T>(work + (size_t)j * S.plane_elems_max, tmp, g.p[p].w, g.p[p].h,
                                       g.levels, g.wavelet, cs);
                if (e != cudaSuccess) break;
            }
            // pointer table of this set's coefficient planes (slot order)
            for (int sl = 0; sl < n; ++sl) outp[sl] = cptr[set * n + sl] + poff[p];
            int16_t **ptab = (int16_t **)(base + S.misc + 2048);
            e = cudaMemcpyAsync(ptab, outp.data(), n * sizeof(void *), cudaMemcpyHostToDevice, cs);
            if (e != cudaSuccess) break;
            k_haar_quant<T><<<(unsigned)((ne + 255) / 256), 256, 0, cs>>>(work, S.plane_elems_max, g.tlevels,
                                                                          g.step, ptab, ne, err);
            e = cudaStreamSynchronize(cs);   // ptab is reused by the next plane
        }
    }
    if (e != cudaSuccess) return WV_ERR_CUDA;
    k_block_flags<<<dim3(g.nbpf, g.num_frames), 256, 0, cs>>>(coef_ptrs, desc, plane_w, plane_off, g.nbpf, flags);
    std::vector<int> fl((size_t)g.num_frames * g.nbpf);
    int herr = 0;
    e = cudaMemcpyAsync(fl.data(), flags, fl.size() * 4, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return WV_ERR_CUDA;
    if (herr) return herr;
    std::vector<int> slots(fl.size());
    int nslots = 0;
    for (size_t i = 0; i < fl.size(); ++i) slots[i] = fl[i] ? nslots++ : -1;
    const size_t table_off = kHeaderBytes;
    const size_t table_bytes = slots.size() * 4;
    const size_t payload_off = (table_off + table_bytes + 255) & ~size_t(255);
    const size_t bbytes = (size_t)g.block * g.block * 2;
    const size_t total = payload_off + (size_t)nslots * bbytes;
    *out_len = total;
    if (cap < total) return WV_ERR_OOM;
    e = cudaMemcpyAsync(flags, slots.data(), table_bytes, cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return WV_ERR_CUDA;
    k_pack<<<dim3(g.nbpf, g.num_frames), 256, 0, cs>>>(coef_ptrs, desc, plane_w, plane_off, g.nbpf, flags,
                                                       g.block, payload);
    char *o = (char *)out;
    memset(o, 0, payload_off);
    StreamHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "WVS1", 4);
    h.version = 1;
    h.width = g.p[0].w;
    h.height = g.p[0].h;
    h.planes = g.planes;
    h.c420 = g.c420;
    h.levels = g.levels;
    h.wavelet = g.wavelet;
    h.num_frames = g.num_frames;
    h.tlevels = g.tlevels;
    h.block = g.block;
    h.quant = 0;
    h.reserved0 = (uint32_t)g.stereo;
    h.step = g.step;
    h.nbpf = g.nbpf;
    h.n_payload = nslots;
    h.table_off = table_off;
    h.payload_off = payload_off;
    memcpy(o, &h, sizeof(h));
    memcpy(o + table_off, slots.data(), table_bytes);
    if (nslots) e = cudaMemcpyAsync(o + payload_off, payload, (size_t)nslots * bbytes, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    return e == cudaSuccess ? WV_OK : WV_ERR_CUDA;
}

// ---- paper-faithful format (Sec. 3.3, 3.4) ---------------------------------

// Subband level (LL_L: levels) and the row inside the subband, with its
// height, of Mallat position (x, y) of a w x h plane.
__device__ __forceinline__ void subband_of(int x, int y, int w, int h, int levels, int &lev, int &ysub,
                                           int &sh) {
    for (int l = 1; l <= levels; ++l) {
        if (x >= (w >> l) || y >= (h >> l)) {
            lev = l;
            sh = h >> l;
            ysub = y >= sh ? y - sh : y;
            return;
        }
    }
    lev = levels;
    sh = h >> levels;
    ysub = y;
}

// Eq. 3 with the mapping factor H(y) = 1 - sin(pi y / S_y) (Sec. 3.6): the
// detail bands of level l take alpha ((L - l) / L)^2 + H; the approximation
// band (l = l_max) takes the level term alone, which is 0 -- H thins the
// detail the equirectangular mapping oversamples toward the poles, it does
// not remove the image itself.
__device__ __forceinline__ float paper_threshold(float alpha, int l, int L, int ysub, int sh, bool approx) {
    const float r = (float)(L - l) / (float)L;
    return alpha * r * r + (approx ? 0.0f : 1.0f - sinpif((float)ysub / (float)sh));
}

__global__ void k_load_unit(const uint8_t *src, float *dst, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = ((float)src[i] - 128.0f) * (1.0f / 255.0f);
}

__global__ void k_threshold(float *c, int w, int h, int levels, float alpha) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)w * h) return;
    const int x = (int)(i % w), y = (int)(i / w);
    int lev, ysub, sh;
    subband_of(x, y, w, h, levels, lev, ysub, sh);
    const bool ll = x < (w >> levels) && y < (h >> levels);
    if (!(fabsf(c[i]) > paper_threshold(alpha, ll ? levels : lev, levels, ysub, sh, ll))) c[i] = 0.f;
}

// Ordered-integer image of a float (monotonic), for atomic min / max.
__device__ __forceinline__ int ord(float f) {
    const int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float unord(int o) { return __int_as_float(o >= 0 ? o : o ^ 0x7FFFFFFF); }

// Float inter-frame Haar over the set's n planes (slot order), the
// inter-frame threshold per slot (temporal level j; the low band as level k),
// and the extremes of the survivors per slot and class: ext[slot][class][0 min, 1 max].
__global__ void k_haar_paper(float *work, size_t plane_elems, int k, int w, int h, int levels, float alpha_t,
                             int *ext) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < (size_t)w * h;
    const int n = 1 << k;
    float low[8], bands[8];
    int lev = 0, ysub = 0, sh = 1;
    bool ll = false;
    if (valid) {
        for (int j = 0; j < n; ++j) low[j] = work[(size_t)j * plane_elems + i];
        const int x = (int)(i % w), y = (int)(i / w);
        subband_of(x, y, w, h, levels, lev, ysub, sh);
        ll = x < (w >> levels) && y < (h >> levels);
    }
    int cnt = n, slot_end = n;
    int slot_level[8];
    slot_level[0] = k;
    for (int j = 1; j <= k; ++j) {
        const int half = cnt / 2;
        slot_end -= half;
        for (int m = 0; m < half; ++m) {
            if (valid) {
                const float a = low[2 * m], b = low[2 * m + 1];
                bands[slot_end + m] = (b - a) * 0.5f;
                low[m] = (a + b) * 0.5f;
            }
            slot_level[slot_end + m] = j;
        }
        cnt = half;
    }
    if (valid) bands[0] = low[0];
    for (int s = 0; s < n; ++s) {
        float c = 0.f;
        if (valid) {
            c = bands[s];
            const float r = k > 0 ? (float)(k - slot_level[s]) / (float)k : 0.f;
            // H on the temporal detail bands' spatial detail only (the low
            // band and the approximation area keep the level term, 0 / small)
            const bool approx = ll || s == 0;
            const float T = alpha_t * r * r + (approx ? 0.0f : 1.0f - sinpif((float)ysub / (float)sh));
            if (!(fabsf(c) > T)) c = 0.f;
            work[(size_t)s * plane_elems + i] = c;
        }
        // extremes of the survivors: warp-level min / max per class, then atomics
        for (int cls = 0; cls < 2; ++cls) {
            const bool mine = valid && c != 0.f && (cls == 0) == ll;
            int mn = mine ? ord(c) : 0x7FFFFFFF, mx = mine ? ord(c) : (int)0x80000000;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            if ((threadIdx.x & 31) == 0 && mn <= mx) {
                atomicMin(ext + (s * 2 + cls) * 2, mn);
                atomicMax(ext + (s * 2 + cls) * 2 + 1, mx);
            }
        }
    }
}

// Byte codes (stored as code + 1; 0 = dropped) of one slot's plane.
__global__ void k_codes(const float *c, int w, int h, int levels, const int *ext, int16_t *out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)w * h) return;
    const float v = c[i];
    if (v == 0.f) {
        out[i] = 0;
        return;
    }
    const int x = (int)(i % w), y = (int)(i / w);
    const int cls = (x < (w >> levels) && y < (h >> levels)) ? 0 : 1;
    const float lo = unord(ext[cls * 2]), hi = unord(ext[cls * 2 + 1]);
    int code = 0;
    if (hi > lo) code = min(max(__float2int_rd((v - lo) / (hi - lo) * 255.0f + 0.5f), 0), 255);
    out[i] = (int16_t)(code + 1);
}

__global__ void k_block_counts(int16_t *const *coef, const BlockDesc *desc, const int *plane_w,
                               const size_t *plane_off, int nbpf, int *counts) {
    const int t = blockIdx.y, b = blockIdx.x;
    const BlockDesc d = desc[b];
    const int16_t *c = coef[t] + plane_off[d.plane];
    const int w = plane_w[d.plane];
    int n = 0;
    for (int idx = threadIdx.x; idx < d.bw * d.bh; idx += blockDim.x) {
        const int y = idx / d.bw, x = idx % d.bw;
        n += c[(size_t)(d.y0 + y) * w + d.x0 + x] != 0;
    }
    __shared__ int sum;
    if (threadIdx.x == 0) sum = 0;
    __syncthreads();
    atomicAdd(&sum, n);
    __syncthreads();
    if (threadIdx.x == 0) counts[t * nbpf + b] = sum;
}

// Records of one block (1024 threads, thread = row-major element): order-
// preserving compaction with ballots and a scan of the 32 warp counts.
__global__ void __launch_bounds__(1024) k_records(int16_t *const *coef, const BlockDesc *desc, const int *plane_w,
                                                  const size_t *plane_off, int nbpf, const long long *start,
                                                  uint32_t *recs) {
    const int t = blockIdx.y, b = blockIdx.x;
    const BlockDesc d = desc[b];
    const int16_t *c = coef[t] + plane_off[d.plane];
    const int w = plane_w[d.plane];
    const int idx = threadIdx.x, y = idx >> 5, x = idx & 31;
    const int v = (x < d.bw && y < d.bh) ? c[(size_t)(d.y0 + y) * w + d.x0 + x] : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, v != 0);
    __shared__ int wc[32], wo[32];
    if ((idx & 31) == 0) wc[idx >> 5] = __popc(bal);
    __syncthreads();
    if (idx == 0) {
        int o = 0;
        for (int k = 0; k < 32; ++k) {
            wo[k] = o;
            o += wc[k];
        }
    }
    __syncthreads();
    if (v != 0) {
        const long long pos = start[t * nbpf + b] + wo[idx >> 5] + __popc(bal & ((1u << (idx & 31)) - 1u));
        recs[pos] = (uint32_t)(y * 32 + x) | ((uint32_t)(v - 1) << 16);
    }
}

int run_paper(const Geom &g, const void *const *planes, char *base, const ScratchLayout &S, float alpha,
              float alpha_t, void *out, size_t cap, size_t *out_len, cudaStream_t cs) {
    const int n = 1 << g.tlevels;
    float *work = (float *)(base + S.work);
    float *tmp = (float *)(base + S.tmp);
    int16_t *coef = (int16_t *)(base + S.coef);
    int *counts = (int *)(base + S.flags);
    BlockDesc *desc = (BlockDesc *)(base + S.desc);
    int *ext = (int *)(base + S.misc);           // [8 slots][2][2] per (set, plane) pass
    int *plane_w = (int *)(base + S.misc + 512);
    size_t *plane_off = (size_t *)(base + S.misc + 576);
    int16_t **coef_ptrs = (int16_t **)(base + S.misc + 4096);
    long long *start = (long long *)(base + S.payload);
    uint32_t *recs = (uint32_t *)(base + S.payload + (size_t)g.num_frames * g.nbpf * 8);

    const std::vector<BlockDesc> bd = block_descs(g);
    if ((int)bd.size() != g.nbpf) return WV_ERR_ARG;
    std::vector<int16_t *> cptr(g.num_frames);
    for (int t = 0; t < g.num_frames; ++t) cptr[t] = coef + (size_t)t * S.coef_frame_elems;
    int pw[3] = {0, 0, 0};
    size_t poff[3] = {0, 0, 0};
    size_t acc = 0;
    for (int p = 0; p < g.planes; ++p) {
        pw[p] = g.p[p].w;
        poff[p] = acc;
        acc += (size_t)g.p[p].w * g.p[p].h;
    }
    cudaError_t e = cudaMemcpyAsync(desc, bd.data(), bd.size() * sizeof(BlockDesc), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(plane_w, pw, sizeof(pw), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(plane_off, poff, sizeof(poff), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(coef_ptrs, cptr.data(), cptr.size() * sizeof(void *), cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return WV_ERR_CUDA;
    // extremes (c_min, c_max) per coefficient frame, plane, class
    std::vector<float> ext_host((size_t)g.num_frames * g.planes * 4, 0.f);
    for (int set = 0; set < g.num_frames / n && e == cudaSuccess; ++set) {
        for (int p = 0; p < g.planes && e == cudaSuccess; ++p) {
            const int w = g.p[p].w, h = g.p[p].h;
            const size_t ne = (size_t)w * h;
            const unsigned blocks = (unsigned)((ne + 255) / 256);
            for (int j = 0; j < n; ++j) {
                const uint8_t *src = (const uint8_t *)planes[(size_t)(set * n + j) * g.planes + p];
                if (!src) return WV_ERR_ARG;
                float *wj = work + (size_t)j * S.plane_elems_max;
                k_load_unit<<<blocks, 256, 0, cs>>>(src, wj, ne);
                e = transform_plane<float>(wj, tmp, w, h, g.levels, WV_WAVELET_97, cs);
                if (e != cudaSuccess) break;
                k_threshold<<<blocks, 256, 0, cs>>>(wj, w, h, g.levels, alpha);
            }
            std::vector<int> init(8 * 4);
            for (int q = 0; q < 8 * 2; ++q) {
                init[2 * q] = 0x7FFFFFFF;
                init[2 * q + 1] = (int)0x80000000;
            }
            e = cudaMemcpyAsync(ext, init.data(), init.size() * 4, cudaMemcpyHostToDevice, cs);
            if (e != cudaSuccess) break;
            k_haar_paper<<<blocks, 256, 0, cs>>>(work, S.plane_elems_max, g.tlevels, w, h, g.levels, alpha_t, ext);
            for (int sl = 0; sl < n; ++sl)
                k_codes<<<blocks, 256, 0, cs>>>(work + (size_t)sl * S.plane_elems_max, w, h, g.levels, ext + sl * 4,
                                                cptr[set * n + sl] + poff[p]);
            std::vector<int> eh(8 * 4);
            e = cudaMemcpyAsync(eh.data(), ext, eh.size() * 4, cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
            if (e != cudaSuccess) break;
            auto unord_h = [](int o) {
                const int b = o >= 0 ? o : o ^ 0x7FFFFFFF;
                float f;
                memcpy(&f, &b, 4);
                return f;
            };
            for (int sl = 0; sl < n; ++sl)
                for (int cls = 0; cls < 2; ++cls) {
                    const int mn = eh[(sl * 2 + cls) * 2], mx = eh[(sl * 2 + cls) * 2 + 1];
                    float *dst = &ext_host[(((size_t)(set * n + sl)) * g.planes + p) * 4 + cls * 2];
                    if (mn <= mx) {
                        dst[0] = unord_h(mn);
                        dst[1] = unord_h(mx);
                    }
                }
        }
    }
    if (e != cudaSuccess) return WV_ERR_CUDA;
    k_block_counts<<<dim3(g.nbpf, g.num_frames), 256, 0, cs>>>(coef_ptrs, desc, plane_w, plane_off, g.nbpf, counts);
    std::vector<int> cnt((size_t)g.num_frames * g.nbpf);
    e = cudaMemcpyAsync(cnt.data(), counts, cnt.size() * 4, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return WV_ERR_CUDA;
    // layout: header, frame offsets, per frame: count, 0, extremes, BlockEnd, records (16-byte padded)
    std::vector<long long> st(cnt.size());
    std::vector<size_t> foff(g.num_frames);
    std::vector<uint32_t> fcount(g.num_frames);
    long long total_recs = 0;
    size_t o = kHeaderBytes + 8 * (size_t)g.num_frames;
    o = (o + 15) & ~size_t(15);
    for (int t = 0; t < g.num_frames; ++t) {
        foff[t] = o;
        long long c = 0;
        for (int b = 0; b < g.nbpf; ++b) {
            st[(size_t)t * g.nbpf + b] = total_recs + c;
            c += cnt[(size_t)t * g.nbpf + b];
        }
        fcount[t] = (uint32_t)c;
        total_recs += c;
        o += 8 + 16 * (size_t)g.planes + 4 * (size_t)g.nbpf + 4 * (size_t)c;
        o = (o + 15) & ~size_t(15);
    }
    *out_len = o;
    if (cap < o) return WV_ERR_OOM;
    if ((size_t)total_recs * 4 + (size_t)g.num_frames * g.nbpf * 8 > S.total - S.payload) return WV_ERR_OOM;
    e = cudaMemcpyAsync(start, st.data(), st.size() * 8, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) {
        k_records<<<dim3(g.nbpf, g.num_frames), 1024, 0, cs>>>(coef_ptrs, desc, plane_w, plane_off, g.nbpf, start, recs);
        e = cudaGetLastError();
    }
    std::vector<uint32_t> rh((size_t)total_recs);
    if (e == cudaSuccess && total_recs)
        e = cudaMemcpyAsync(rh.data(), recs, rh.size() * 4, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return WV_ERR_CUDA;
    char *ob = (char *)out;
    memset(ob, 0, o);
    uint32_t hdr[11] = {1, (uint32_t)g.p[0].w, (uint32_t)g.p[0].h, (uint32_t)g.planes, (uint32_t)g.c420,
                        (uint32_t)g.levels, (uint32_t)g.num_frames, (uint32_t)g.tlevels, 32u, (uint32_t)g.nbpf, 0};
    memcpy(ob, "WVP1", 4);
    memcpy(ob + 4, hdr, 10 * 4);
    memcpy(ob + 44, &alpha, 4);
    memcpy(ob + 48, &alpha_t, 4);
    for (int t = 0; t < g.num_frames; ++t) {
        const uint64_t off = foff[t];
        memcpy(ob + kHeaderBytes + 8 * t, &off, 8);
        char *f = ob + off;
        memcpy(f, &fcount[t], 4);
        memcpy(f + 8, &ext_host[(size_t)t * g.planes * 4], 16 * (size_t)g.planes);
        uint32_t *ends = (uint32_t *)(f + 8 + 16 * g.planes);
        uint32_t c = 0;
        for (int b = 0; b < g.nbpf; ++b) {
            c += (uint32_t)cnt[(size_t)t * g.nbpf + b];
            ends[b] = c;
        }
        if (fcount[t])
            memcpy(f + 8 + 16 * g.planes + 4 * (size_t)g.nbpf, &rh[(size_t)st[(size_t)t * g.nbpf]], 4 * (size_t)fcount[t]);
    }
    return WV_OK;
}

}  // namespace

int encode_paper(const Geom &g, const void *const *planes, void *scratch, size_t scratch_bytes, float alpha,
                 float alpha_t, void *out, size_t cap, size_t *out_len, cudaStream_t cs) {
    const ScratchLayout S = scratch_layout(g);
    if (scratch_bytes < S.total || ((uintptr_t)scratch % 256)) return WV_ERR_OOM;
    if (g.tlevels > 3 || g.wavelet != WV_WAVELET_97 || g.block != 32) return WV_ERR_ARG;
    return run_paper(g, planes, (char *)scratch, S, alpha, alpha_t, out, cap, out_len, cs);
}

int encode_sizes(const Geom &g, size_t *scratch, size_t *max_stream) {
    const ScratchLayout S = scratch_layout(g);
    if (scratch) *scratch = S.total;
    if (max_stream) {
        const size_t tb = (size_t)g.num_frames * g.nbpf * 4;
        if (g.quant == 1)
            *max_stream = kHeaderBytes + 8 * (size_t)g.num_frames +
                          (size_t)g.num_frames * (32 + 16 * (size_t)g.planes + tb / g.num_frames) +
                          (size_t)g.num_frames * S.coef_frame_elems * 4;
        else
            *max_stream = ((kHeaderBytes + tb + 255) & ~size_t(255)) +
                          (size_t)g.num_frames * g.nbpf * g.block * g.block * 2;
    }
    return WV_OK;
}

int encode_run(const Geom &g, const void *const *planes, void *scratch, size_t scratch_bytes,
               void *out, size_t cap, size_t *out_len, cudaStream_t cs) {
    const ScratchLayout S = scratch_layout(g);
    if (scratch_bytes < S.total || ((uintptr_t)scratch % 256)) return WV_ERR_OOM;
    if (g.tlevels > 3) return WV_ERR_ARG;
    if (g.wavelet == WV_WAVELET_97)
        return run<float>(g, planes, (char *)scratch, S, out, cap, out_len, cs);
    return run<int>(g, planes, (char *)scratch, S, out, cap, out_len, cs);
}

}  // namespace wv
