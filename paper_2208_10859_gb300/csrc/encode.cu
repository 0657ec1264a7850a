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

}  // namespace

int encode_sizes(const Geom &g, size_t *scratch, size_t *max_stream) {
    const ScratchLayout S = scratch_layout(g);
    if (scratch) *scratch = S.total;
    if (max_stream) {
        const size_t tb = (size_t)g.num_frames * g.nbpf * 4;
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
