// postfilter.cu -- residual CNN post-filter on the decoded viewport's luma.
//
// The paper has no learned component; this network extends the decoder: it
// removes quantisation artefacts from the viewport's luma.  Five 3x3
// convolutions with zero padding: 1 -> 32 channels (ReLU), three 32 -> 32
// (ReLU), 32 -> 1; the output is the input luma plus that residual.  Weights
// are bf16 (fp32 master copies for training), activations bf16 between
// layers, every product accumulated in fp32 on the tensor cores.
//
// Convolutions are implicit GEMMs on tcgen05 (one elected thread issues the
// MMAs, operands in shared memory, accumulator in TMEM):
//   forward / input gradient, 32 input channels: M = 128 pixels of one image
//     row, N = 32 (or 16 for the 1-channel output), K = 9 taps x 32 channels
//     = 18 K-steps.  The three input rows live in shared memory as 8-channel
//     columns of 130 pixels (16 bytes per pixel), so the A operand of tap
//     (dy, dx) is the row slot of dy shifted by dx pixels: only the
//     descriptor's start address changes (SBO = 128 bytes, LBO = one column).
//   forward / input gradient, 1 input channel: K = the 9 taps (padded to 16).
//   weight gradient, 32 -> 32: D[tap, ci][co] = sum over pixels of
//     input[p + tap][ci] * dZ[p][co]: M = 288 rows (+ one row of ones that
//     yields the bias gradient), N = 32, K = pixels in chunks of 64.
//   The input gradient of a layer is a forward convolution of the output
//   gradient with the spatially flipped, channel-transposed weights; the
//   ReLU of the layer below gates it in the epilogue.
// The weight gradients of the first and last layers (1 channel on one side,
// 1/32 of the work) run on CUDA cores.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "umma.h"
#include "wv_impl.h"

namespace wv {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kC = 32;                  // channels of the hidden layers
constexpr int kLayers = 5;
constexpr int kTilePx = 128;            // pixels per MMA tile (M)
constexpr int kRowPx = kTilePx + 2;     // input pixels of one row slot (1-pixel halo)
constexpr int kLbo = kRowPx * 16;       // bytes between the 8-channel columns of a slot
constexpr int kSlot = 4 * kLbo;         // one input row: 4 columns of 8 channels
constexpr int kStrip = 16;              // output rows per work item
constexpr int kStep32 = 32 * 32;        // bytes of one K-step of a 32-row operand
constexpr int kBMid = 18 * kStep32;     // 32 x 288
constexpr int kBLast = 18 * 16 * 32;    // 16 x 288 (row 0 real)
constexpr int kBIn1 = kStep32;          // 32 x 16 (taps 0..8)

__host__ __device__ constexpr int layer_co(int l) { return l == kLayers - 1 ? 1 : kC; }
__host__ __device__ constexpr int layer_ci(int l) { return l == 0 ? 1 : kC; }
__host__ __device__ constexpr int off_w(int l) {
    int o = 0;
    for (int k = 0; k < l; ++k) o += layer_co(k) * layer_ci(k) * 9 + layer_co(k);
    return o;
}
__host__ __device__ constexpr int off_b(int l) { return off_w(l) + layer_co(l) * layer_ci(l) * 9; }
constexpr int kParams = off_w(kLayers);

// packed bf16 B operands: forward of layers 0..4, input gradient of 4..1
enum Pack { kPF0 = 0, kPF1 = kPF0 + kBIn1, kPF2 = kPF1 + kBMid, kPF3 = kPF2 + kBMid, kPF4 = kPF3 + kBMid,
            kPB4 = kPF4 + kBLast, kPB3 = kPB4 + kBIn1, kPB2 = kPB3 + kBMid, kPB1 = kPB2 + kBMid,
            kPackBytes = kPB1 + kBMid };

enum Mode { kRelu = 0, kGate = 1, kLastTrain = 2, kLastOut = 3, kLastRgba = 4 };

struct ConvArgs {
    const bf16 *in;          // NHWC, 32 channels (k_conv_mid)
    const float *in_plane;   // one channel (k_conv_in1)
    const uint8_t *wpack;    // packed B operand
    const float *bias;       // per output channel, or null
    int n, h, w;
    int mode;
    bf16 *out;               // NHWC, 32 channels
    const bf16 *gate;        // kGate: ReLU outputs of the layer below (NHWC)
    const float *x;          // last layer: input luma
    const float *t;          // kLastTrain: target
    float *y;                // last layer: output plane (optional)
    float *dz;               // kLastTrain: dL/dr plane
    float *loss;             // kLastTrain: sum of squared errors
    float grad_scale;        // kLastTrain: 2 / pixel count
    const uint8_t *cb, *cr;  // kLastRgba: chroma planes of the viewport
    uint8_t *rgba;
    size_t pitch;
    int *err;
};

__device__ __forceinline__ size_t pix(const ConvArgs &a, int img, int y, int x) {
    return ((size_t)img * a.h + y) * a.w + x;
}

// Epilogue of the 32-channel modes for one pixel: bias + ReLU, or the ReLU
// gate of the layer below; bf16 NHWC store.
__device__ __forceinline__ void load_gate(const ConvArgs &a, size_t p, uint4 (&g)[4]) {
    const uint4 *src = reinterpret_cast<const uint4 *>(a.gate + p * kC);
#pragma unroll
    for (int q = 0; q < 4; ++q) g[q] = __ldg(src + q);
}

__device__ __forceinline__ void store32(const ConvArgs &a, size_t p, const float (&v)[32], const uint4 (&gate)[4]) {
    float o[32];
    if (a.mode == kRelu) {
#pragma unroll
        for (int c = 0; c < 32; ++c) o[c] = fmaxf(v[c] + (a.bias ? __ldg(a.bias + c) : 0.f), 0.f);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 gv = gate[q];
            const bf16 *gb = reinterpret_cast<const bf16 *>(&gv);
#pragma unroll
            for (int e = 0; e < 8; ++e) o[8 * q + e] = __bfloat162float(gb[e]) > 0.f ? v[8 * q + e] : 0.f;
        }
    }
    uint4 *dst = reinterpret_cast<uint4 *>(a.out + p * kC);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint4 w;
        uint32_t *wp = reinterpret_cast<uint32_t *>(&w);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(o[8 * q + 2 * e], o[8 * q + 2 * e + 1]);
            wp[e] = *reinterpret_cast<const uint32_t *>(&b2);
        }
        dst[q] = w;
    }
}

// Epilogue of the last layer (residual in column 0).
__device__ __forceinline__ void store_last(const ConvArgs &a, size_t p, float r, bool valid) {
    float e2 = 0.f;
    if (valid) {
        const float yv = __ldg(a.x + p) + r + __ldg(a.bias);
        if (a.y) a.y[p] = yv;
        if (a.mode == kLastTrain) {
            const float e = yv - __ldg(a.t + p);
            a.dz[p] = a.grad_scale * e;
            e2 = e * e;
        } else if (a.mode == kLastRgba) {
            const int yy = min(max(__float2int_rd(fmaf(yv, 255.f, 0.5f)), 0), 255);
            const uchar4 c = to_rgba(yy, a.cb[p], a.cr[p]);
            const int xw = (int)(p % a.w), yh = (int)(p / a.w);
            *reinterpret_cast<uchar4 *>(a.rgba + (size_t)yh * a.pitch + 4 * (size_t)xw) = c;
        }
    }
    if (a.mode == kLastTrain) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
        if ((threadIdx.x & 31) == 0 && e2 != 0.f) atomicAdd(a.loss, e2);
    }
}

// Convolution with 32 input channels (forward of layers 1-4, input gradient
// of layers 1-3).  CTA: 128 threads, a strip of kStrip rows x 128 pixels.
__global__ void __launch_bounds__(128) k_conv_mid(ConvArgs a, int nb) {
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *slots = sm;              // 3 row slots
    uint8_t *sB = sm + 3 * kSlot;     // packed B
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int bbytes = nb == 32 ? kBMid : kBLast;
    for (int i = tid * 16; i < bbytes; i += 128 * 16)
        *reinterpret_cast<uint4 *>(sB + i) = __ldg(reinterpret_cast<const uint4 *>(a.wpack + i));
    if (tid == 0) umma::mbar_init(&mbar, 1);
    if (warp == 0) umma::tmem_alloc<32>(&tmem_base);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = nb == 32 ? umma::idesc_bf16(128, 32) : umma::idesc_bf16(128, 16);
    const int bstep = nb * 32;
    uint32_t phase = 0;
    // input row r: 130 pixels x 4 columns of 8 channels, 16 bytes each,
    // staged through registers so that the next row's loads overlap the
    // MMAs and the epilogue of the current one
    constexpr int kPer = (kRowPx * 4 + 127) / 128;
    uint4 pre[kPer];
    auto load_row = [&](int img, int x0, int r) {
        const bool rin = r >= 0 && r < a.h;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int idx = tid + 128 * j;
            const int px = idx >> 2, c = idx & 3, gx = x0 - 1 + px;
            pre[j] = make_uint4(0u, 0u, 0u, 0u);
            if (idx < kRowPx * 4 && rin && gx >= 0 && gx < a.w)
                pre[j] = __ldg(reinterpret_cast<const uint4 *>(a.in + pix(a, img, r, gx) * kC + c * 8));
        }
    };
    auto store_row = [&](int r) {
        uint8_t *slot = slots + ((r + 3) % 3) * kSlot;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int idx = tid + 128 * j;
            if (idx < kRowPx * 4) *reinterpret_cast<uint4 *>(slot + (idx & 3) * kLbo + (idx >> 2) * 16) = pre[j];
        }
    };
    // work items: strips of kStrip rows x 128 pixels, CTA b takes b, b + grid, ...
    const int tiles_x = (a.w + kTilePx - 1) / kTilePx, strips = (a.h + kStrip - 1) / kStrip;
    const int items = tiles_x * strips * a.n;
    bool ok = true;
    for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
        const int img = it / (tiles_x * strips), sy = (it / tiles_x) % strips;
        const int x0 = (it % tiles_x) * kTilePx, y0 = sy * kStrip, y1 = min(y0 + kStrip, a.h);
        // the slots are free: the previous item's MMAs have completed
        for (int r = y0 - 1; r <= y0 + 1; ++r) {
            load_row(img, x0, r);
            store_row(r);
        }
        const int xg = x0 + tid;
        const bool valid = xg < a.w;
        for (int y = y0; y < y1; ++y) {
            umma::fence_smem_to_async();
            umma::fence_before_sync();
            __syncthreads();
            umma::fence_after_sync();
            if (tid == 0) {
                const uint32_t sb = umma::smem_addr(sB);
#pragma unroll 1
                for (int tap = 0; tap < 9; ++tap) {
                    const int dy = tap / 3, dx = tap % 3;
                    const uint32_t abase = umma::smem_addr(slots + ((y + dy - 1 + 3) % 3) * kSlot) + dx * 16;
#pragma unroll
                    for (int s = 0; s < 2; ++s)
                        umma::mma(tmem, umma::desc(abase + 2 * s * kLbo, kLbo, 128),
                                  umma::desc(sb + (tap * 2 + s) * bstep, 128, 256), idesc, tap > 0 || s > 0);
                }
                umma::commit(&mbar);
            }
            const bool more = y + 1 < y1;
            if (more) load_row(img, x0, y + 2);
            uint4 gate[4] = {};
            if (nb == 32 && a.mode == kGate && valid) load_gate(a, pix(a, img, y, xg), gate);
            const bool got = __syncthreads_and(umma::mbar_wait(&mbar, phase));
            phase ^= 1;
            if (!got) {
                if (tid == 0) record_error(a.err, WV_ERR_TIMEOUT);
                ok = false;
                break;
            }
            umma::fence_after_sync();
            float v[32];
            umma::ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
            if (nb == 32) {
                if (valid) store32(a, pix(a, img, y, xg), v, gate);
            } else {
                store_last(a, valid ? pix(a, img, y, xg) : 0, v[0], valid);
            }
            // the slot of row y - 1 is free: this row's MMAs have completed
            if (more) store_row(y + 2);
            umma::fence_before_sync();
        }
    }
    __syncthreads();
    if (warp == 0) umma::tmem_free<32>(tmem);
}

// Convolution with one input channel (forward of layer 0, input gradient of
// layer 4): A row of a pixel = its 9 taps, padded to K = 16.
__global__ void __launch_bounds__(128) k_conv_in1(ConvArgs a) {
    __shared__ __align__(128) uint8_t sA[128 * 32];
    __shared__ __align__(128) uint8_t sB[kBIn1];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int x0 = blockIdx.x * kTilePx, y0 = blockIdx.y * kStrip, img = blockIdx.z;
    for (int i = tid * 16; i < kBIn1; i += 128 * 16)
        *reinterpret_cast<uint4 *>(sB + i) = __ldg(reinterpret_cast<const uint4 *>(a.wpack + i));
    if (tid == 0) umma::mbar_init(&mbar, 1);
    if (warp == 0) umma::tmem_alloc<32>(&tmem_base);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = umma::idesc_bf16(128, 32);
    uint32_t phase = 0;
    const int xg = x0 + tid;
    const int y1 = min(y0 + kStrip, a.h);
    for (int y = y0; y < y1; ++y) {
        float t[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            t[k] = 0.f;
            if (k < 9) {
                const int yy = y + k / 3 - 1, xx = xg + k % 3 - 1;
                if (yy >= 0 && yy < a.h && xx >= 0 && xx < a.w) t[k] = __ldg(a.in_plane + pix(a, img, yy, xx));
            }
        }
#pragma unroll
        for (int k = 0; k < 16; k += 2) {
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(t[k], t[k + 1]);
            *reinterpret_cast<__nv_bfloat162 *>(sA + umma::kstep_offset(tid, k)) = b2;
        }
        umma::fence_smem_to_async();
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();
        if (tid == 0) {
            umma::mma(tmem, umma::desc(umma::smem_addr(sA), 128, 256), umma::desc(umma::smem_addr(sB), 128, 256),
                      idesc, false);
            umma::commit(&mbar);
        }
        const bool got = __syncthreads_and(umma::mbar_wait(&mbar, phase));
        phase ^= 1;
        if (!got) {
            if (tid == 0) record_error(a.err, WV_ERR_TIMEOUT);
            break;
        }
        umma::fence_after_sync();
        float v[32];
        umma::ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
        uint4 gate[4] = {};
        if (a.mode == kGate && xg < a.w) load_gate(a, pix(a, img, y, xg), gate);
        if (xg < a.w) store32(a, pix(a, img, y, xg), v, gate);
        umma::fence_before_sync();
        __syncthreads();
    }
    __syncthreads();
    if (warp == 0) umma::tmem_free<32>(tmem);
}

// Weight gradient of a 32 -> 32 layer on the tensor cores.  Per chunk of 64
// pixels of one image row: A[(tap, ci)][p] = act[p + tap][ci] (288 rows, row
// 288 = 1 for the bias gradient, rows up to 383 zero), B[co][p] = dz[p][co],
// both transposed into K-major tiles in shared memory; three M-tiles of 128
// rows accumulate in TMEM over all chunks of the CTA, then are added to the
// global gradient.
constexpr int kWChunk = 64;
constexpr int kWRows = 384;
constexpr int kWAStep = kWRows * 32;
constexpr int kWA = 4 * kWAStep;
constexpr int kWB = 4 * kStep32;
constexpr int kWAct = 3 * (kWChunk + 2) * 64;
constexpr int kWDz = kWChunk * 64;
constexpr int kWSmem = kWA + kWB + kWAct + kWDz;

__global__ void __launch_bounds__(128) k_wgrad_mid(const bf16 *__restrict__ act, const bf16 *__restrict__ dz,
                                                   int n, int h, int w, float *dW, float *db, int *err) {
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *sA = sm, *sB = sm + kWA, *sAct = sB + kWB, *sDz = sAct + kWAct;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    // rows 288..383 of every K-step: ones (row 288), zeros
    for (int i = tid; i < 4 * 96 * 8; i += 128) {
        const int s = i / (96 * 8), r = 288 + (i / 8) % 96, kp = i % 8;
        const float one = r == 288 ? 1.f : 0.f;
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(one, one);
        *reinterpret_cast<__nv_bfloat162 *>(sA + s * kWAStep + umma::kstep_offset(r, 2 * kp)) = b2;
    }
    if (tid == 0) umma::mbar_init(&mbar, 1);
    if (warp == 0) umma::tmem_alloc<128>(&tmem_base);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = umma::idesc_bf16(128, 32);
    const int xchunks = (w + kWChunk - 1) / kWChunk;
    const int total = n * h * xchunks;
    uint32_t phase = 0;
    bool first = true, ok = true;
    for (int ch = blockIdx.x; ch < total; ch += gridDim.x) {
        const int xc = ch % xchunks, y = (ch / xchunks) % h, img = ch / (xchunks * h);
        const int x0 = xc * kWChunk;
        for (int i = tid; i < 3 * (kWChunk + 2) * 4; i += 128) {
            const int q = i & 3, px = (i >> 2) % (kWChunk + 2), dy = (i >> 2) / (kWChunk + 2);
            const int yy = y + dy - 1, xx = x0 - 1 + px;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (yy >= 0 && yy < h && xx >= 0 && xx < w)
                v = __ldg(reinterpret_cast<const uint4 *>(act + (((size_t)img * h + yy) * w + xx) * kC + q * 8));
            *reinterpret_cast<uint4 *>(sAct + (dy * (kWChunk + 2) + px) * 64 + q * 16) = v;
        }
        for (int i = tid; i < kWChunk * 4; i += 128) {
            const int q = i & 3, px = i >> 2, xx = x0 + px;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (xx < w) v = __ldg(reinterpret_cast<const uint4 *>(dz + (((size_t)img * h + y) * w + xx) * kC + q * 8));
            *reinterpret_cast<uint4 *>(sDz + px * 64 + q * 16) = v;
        }
        __syncthreads();
        // transpose into the K-major operands: pairs of pixels per store
        for (int i = tid; i < 288 * (kWChunk / 2); i += 128) {
            const int m = i % 288, kp = i / 288, k = 2 * kp;
            const int tap = m >> 5, ci = m & 31, dy = tap / 3, dx = tap % 3;
            const bf16 *row = reinterpret_cast<const bf16 *>(sAct + (dy * (kWChunk + 2) + k + dx) * 64) + ci;
            __nv_bfloat162 b2;
            b2.x = row[0];
            b2.y = row[32];
            *reinterpret_cast<__nv_bfloat162 *>(sA + (k >> 4) * kWAStep + umma::kstep_offset(m, k & 15)) = b2;
        }
        for (int i = tid; i < 32 * (kWChunk / 2); i += 128) {
            const int co = i & 31, kp = i >> 5, k = 2 * kp;
            const bf16 *col = reinterpret_cast<const bf16 *>(sDz + k * 64) + co;
            __nv_bfloat162 b2;
            b2.x = col[0];
            b2.y = col[32];
            *reinterpret_cast<__nv_bfloat162 *>(sB + (k >> 4) * kStep32 + umma::kstep_offset(co, k & 15)) = b2;
        }
        umma::fence_smem_to_async();
        umma::fence_before_sync();
        __syncthreads();
        umma::fence_after_sync();
        if (tid == 0) {
            const uint32_t a0 = umma::smem_addr(sA), b0 = umma::smem_addr(sB);
#pragma unroll 1
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int mt = 0; mt < 3; ++mt)
                    umma::mma(tmem + 32 * mt, umma::desc(a0 + s * kWAStep + mt * 4096, 128, 256),
                              umma::desc(b0 + s * kStep32, 128, 256), idesc, !(first && s == 0));
            umma::commit(&mbar);
        }
        const bool got = __syncthreads_and(umma::mbar_wait(&mbar, phase));
        phase ^= 1;
        if (!got) {
            ok = false;
            if (tid == 0) record_error(err, WV_ERR_TIMEOUT);
            break;
        }
        first = false;
    }
    if (!first && ok) {
        umma::fence_after_sync();
        for (int mt = 0; mt < 3; ++mt) {
            float v[32];
            umma::ld32(tmem + 32 * mt + ((uint32_t)(warp * 32) << 16), v);
            const int m = mt * 128 + warp * 32 + (tid & 31);
            if (m < 288) {
                const int tap = m >> 5, ci = m & 31;
                for (int co = 0; co < 32; ++co) atomicAdd(dW + (co * kC + ci) * 9 + tap, v[co]);
            } else if (m == 288) {
                for (int co = 0; co < 32; ++co) atomicAdd(db + co, v[co]);
            }
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_free<128>(tmem);
}

// Weight gradients of the first (1 -> 32) and last (32 -> 1) layers on CUDA
// cores: thread j of 320 accumulates one (channel, tap) product over the
// chunks of its CTA (tap 9 = the bias).
__global__ void __launch_bounds__(320) k_wgrad_edge(const float *__restrict__ plane, const bf16 *__restrict__ act,
                                                    int first_layer, int n, int h, int w, float *dW, float *db) {
    __shared__ float sP[3 * (kWChunk + 2)];       // first layer: input luma rows
    __shared__ float sG[kWChunk];                 // last layer: dz plane
    __shared__ __align__(16) bf16 sT[3 * (kWChunk + 2) * kC];   // 32-channel tensor rows
    const int tid = threadIdx.x;
    const int xchunks = (w + kWChunk - 1) / kWChunk;
    const int total = n * h * xchunks;
    float acc = 0.f;
    // first layer: c = tid % 32 output channel, j = tid / 32 tap (9: bias);
    // last layer: c = tid % 32 input channel, j = tid / 32 tap (9: bias)
    const int c = tid & 31, j = tid >> 5;
    for (int ch = blockIdx.x; ch < total; ch += gridDim.x) {
        const int xc = ch % xchunks, y = (ch / xchunks) % h, img = ch / (xchunks * h);
        const int x0 = xc * kWChunk;
        __syncthreads();
        if (first_layer) {
            // plane = input luma (3 rows with halo); act = dZ of layer 0 (this row)
            for (int i = tid; i < 3 * (kWChunk + 2); i += 320) {
                const int px = i % (kWChunk + 2), dy = i / (kWChunk + 2);
                const int yy = y + dy - 1, xx = x0 - 1 + px;
                sP[i] = (yy >= 0 && yy < h && xx >= 0 && xx < w) ? plane[((size_t)img * h + yy) * w + xx] : 0.f;
            }
            for (int i = tid; i < kWChunk * 4; i += 320) {
                const int q = i & 3, px = i >> 2, xx = x0 + px;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (xx < w) v = __ldg(reinterpret_cast<const uint4 *>(act + (((size_t)img * h + y) * w + xx) * kC + q * 8));
                *reinterpret_cast<uint4 *>(sT + px * kC + q * 8) = v;
            }
        } else {
            // plane = dZ of the last layer (this row); act = its input (3 rows)
            for (int i = tid; i < kWChunk; i += 320) {
                const int xx = x0 + i;
                sG[i] = xx < w ? plane[((size_t)img * h + y) * w + xx] : 0.f;
            }
            for (int i = tid; i < 3 * (kWChunk + 2) * 4; i += 320) {
                const int q = i & 3, px = (i >> 2) % (kWChunk + 2), dy = (i >> 2) / (kWChunk + 2);
                const int yy = y + dy - 1, xx = x0 - 1 + px;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (yy >= 0 && yy < h && xx >= 0 && xx < w)
                    v = __ldg(reinterpret_cast<const uint4 *>(act + (((size_t)img * h + yy) * w + xx) * kC + q * 8));
                *reinterpret_cast<uint4 *>(sT + (dy * (kWChunk + 2) + px) * kC + q * 8) = v;
            }
        }
        __syncthreads();
        if (j <= 9) {
            const int tap = j < 9 ? j : 0, dy = tap / 3, dx = tap % 3;
            if (first_layer) {
                for (int k = 0; k < kWChunk; ++k) {
                    const float g = __bfloat162float(sT[k * kC + c]);
                    acc = fmaf(g, j < 9 ? sP[dy * (kWChunk + 2) + k + dx] : 1.f, acc);
                }
            } else {
                for (int k = 0; k < kWChunk; ++k) {
                    const float a = j < 9 ? __bfloat162float(sT[(dy * (kWChunk + 2) + k + dx) * kC + c]) : 1.f;
                    acc = fmaf(sG[k], a, acc);
                }
            }
        }
    }
    if (j < 9) {
        // first layer: dW0[c][0][j]; last layer: dW4[0][c][j]
        atomicAdd(dW + c * 9 + j, acc);
    } else if (j == 9) {
        if (first_layer) atomicAdd(db + c, acc);
        else if (c == 0) {
            // bias of the last layer: every c accumulated the same sum; use c = 0
            atomicAdd(db, acc);
        }
    }
}

// bf16 B operands from the fp32 master parameters (one thread per element).
__global__ void k_pack(const float *__restrict__ P, uint8_t *pack) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;   // bf16 element index
    const int byte = 2 * e;
    if (byte >= kPackBytes) return;
    float v = 0.f;
    auto mid = [&](int base, int layer, bool bwd) {
        // K index k = tap * 32 + c, K-step t = k / 16; 32 rows
        const int o = byte - base, t = o / kStep32, in = o % kStep32;
        const int rg = in / 256, kc = (in % 256) / 128, r8 = (in % 128) / 16, k8 = (in % 16) / 2;
        const int r = rg * 8 + r8, kk = kc * 8 + k8, k = t * 16 + kk, tap = k >> 5, c = k & 31;
        // forward: row = co, K = (tap, ci); input gradient: row = ci, K = (flipped tap, co)
        const int co = bwd ? c : r, ci = bwd ? r : c, tp = bwd ? 8 - tap : tap;
        return P[off_w(layer) + (co * kC + ci) * 9 + tp];
    };
    auto in1 = [&](int base, int layer, bool bwd) {
        const int in = byte - base;
        const int rg = in / 256, kc = (in % 256) / 128, r8 = (in % 128) / 16, k8 = (in % 16) / 2;
        const int r = rg * 8 + r8, k = kc * 8 + k8;
        if (k >= 9) return 0.f;
        // forward layer 0: row = co, K = tap; input gradient of layer 4: row = ci, K = flipped tap
        return bwd ? P[off_w(layer) + r * 9 + (8 - k)] : P[off_w(layer) + r * 9 + k];
    };
    if (byte < kPF1) v = in1(kPF0, 0, false);
    else if (byte < kPF2) v = mid(kPF1, 1, false);
    else if (byte < kPF3) v = mid(kPF2, 2, false);
    else if (byte < kPF4) v = mid(kPF3, 3, false);
    else if (byte < kPB4) {
        const int o = byte - kPF4, t = o / 512, in = o % 512;
        const int rg = in / 256, kc = (in % 256) / 128, r8 = (in % 128) / 16, k8 = (in % 16) / 2;
        const int r = rg * 8 + r8, k = t * 16 + kc * 8 + k8;
        v = r == 0 ? P[off_w(4) + (k & 31) * 9 + (k >> 5)] : 0.f;
    } else if (byte < kPB3) v = in1(kPB4, 4, true);
    else if (byte < kPB2) v = mid(kPB3, 3, true);
    else if (byte < kPB1) v = mid(kPB2, 2, true);
    else v = mid(kPB1, 1, true);
    reinterpret_cast<bf16 *>(pack)[e] = __float2bfloat16_rn(v);
}

__global__ void k_adam(float *P, const float *G, float *M, float *V, int n, float lr, float b1, float b2,
                       float c1, float c2, float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

int sm_count() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace
}  // namespace wv

using namespace wv;

struct wv_cnn {
    int device = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    uint8_t *pack = nullptr;
    bool packed = false;
    int step = 0;
    size_t cap_px = 0;
    bf16 *act[4] = {};
    bf16 *g[2] = {};
    float *dz5 = nullptr, *loss = nullptr, *xbuf = nullptr;
    uint8_t *cb = nullptr, *cr = nullptr;
    int *err = nullptr;
    std::vector<void *> owned;
};

namespace {

int ensure_workspace(wv_cnn *c, size_t px) {
    if (px <= c->cap_px) return WV_OK;
    for (void *p : c->owned) cudaFree(p);
    c->owned.clear();
    const size_t want = px + px / 8;
    auto get = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
        c->owned.push_back(p);
        return p;
    };
    for (int i = 0; i < 4; ++i) c->act[i] = (bf16 *)get(want * kC * 2);
    for (int i = 0; i < 2; ++i) c->g[i] = (bf16 *)get(want * kC * 2);
    c->dz5 = (float *)get(want * 4);
    c->xbuf = (float *)get(want * 4);
    c->cb = (uint8_t *)get(want);
    c->cr = (uint8_t *)get(want);
    for (void *p : c->owned)
        if (!p) {
            cudaGetLastError();
            c->cap_px = 0;
            return WV_ERR_OOM;
        }
    c->cap_px = want;
    return WV_OK;
}

void pack_params(wv_cnn *c, cudaStream_t cs) {
    const int elems = kPackBytes / 2;
    k_pack<<<(elems + 255) / 256, 256, 0, cs>>>(c->params, c->pack);
    c->packed = true;
}

ConvArgs conv_args(wv_cnn *c, int n, int h, int w) {
    ConvArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.h = h;
    a.w = w;
    a.err = c->err;
    return a;
}

cudaError_t launch_mid(const ConvArgs &a, int nb, cudaStream_t cs) {
    const int smem = 3 * kSlot + kBMid;
    cudaError_t e = opt_in_smem(reinterpret_cast<const void *>(k_conv_mid), smem);
    if (e != cudaSuccess) return e;
    // one work item (strip) per CTA: measured faster than persistent CTAs
    const int items = ((a.w + kTilePx - 1) / kTilePx) * ((a.h + kStrip - 1) / kStrip) * a.n;
    k_conv_mid<<<items, 128, smem, cs>>>(a, nb);
    return cudaGetLastError();
}

cudaError_t launch_in1(const ConvArgs &a, cudaStream_t cs) {
    dim3 grid((a.w + kTilePx - 1) / kTilePx, (a.h + kStrip - 1) / kStrip, a.n);
    k_conv_in1<<<grid, 128, 0, cs>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_wgrad_mid(const bf16 *act, const bf16 *dz, int n, int h, int w, float *dW, float *db, int *err,
                             cudaStream_t cs) {
    cudaError_t e = opt_in_smem(reinterpret_cast<const void *>(k_wgrad_mid), kWSmem);
    if (e != cudaSuccess) return e;
    const int total = n * h * ((w + kWChunk - 1) / kWChunk);
    const int grid = std::max(1, std::min(total, 3 * sm_count()));
    k_wgrad_mid<<<grid, 128, kWSmem, cs>>>(act, dz, n, h, w, dW, db, err);
    return cudaGetLastError();
}

cudaError_t launch_wgrad_edge(const float *plane, const bf16 *act, int first, int n, int h, int w, float *dW,
                              float *db, cudaStream_t cs) {
    const int total = n * h * ((w + kWChunk - 1) / kWChunk);
    const int grid = std::max(1, std::min(total, 2 * sm_count()));
    k_wgrad_edge<<<grid, 320, 0, cs>>>(plane, act, first, n, h, w, dW, db);
    return cudaGetLastError();
}

// Forward pass; last-layer epilogue per `last` (with its outputs in `fin`).
cudaError_t forward(wv_cnn *c, const float *x, int n, int h, int w, const ConvArgs &fin, cudaStream_t cs) {
    if (!c->packed) pack_params(c, cs);
    ConvArgs a = conv_args(c, n, h, w);
    a.in_plane = x;
    a.wpack = c->pack + kPF0;
    a.bias = c->params + off_b(0);
    a.mode = kRelu;
    a.out = c->act[0];
    cudaError_t e = launch_in1(a, cs);
    const int packs[3] = {kPF1, kPF2, kPF3};
    for (int l = 1; l <= 3 && e == cudaSuccess; ++l) {
        a = conv_args(c, n, h, w);
        a.in = c->act[l - 1];
        a.wpack = c->pack + packs[l - 1];
        a.bias = c->params + off_b(l);
        a.mode = kRelu;
        a.out = c->act[l];
        e = launch_mid(a, 32, cs);
    }
    if (e != cudaSuccess) return e;
    a = fin;
    a.n = n;
    a.h = h;
    a.w = w;
    a.err = c->err;
    a.in = c->act[3];
    a.wpack = c->pack + kPF4;
    a.bias = c->params + off_b(4);
    a.x = x;
    return launch_mid(a, 16, cs);
}

// Forward with the training epilogue, then every gradient into c->grads.
cudaError_t forward_backward(wv_cnn *c, const float *x, const float *t, int n, int h, int w, cudaStream_t cs) {
    cudaError_t e = cudaMemsetAsync(c->grads, 0, sizeof(float) * kParams, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->loss, 0, sizeof(float), cs);
    if (e != cudaSuccess) return e;
    ConvArgs fin;
    memset(&fin, 0, sizeof(fin));
    fin.mode = kLastTrain;
    fin.t = t;
    fin.dz = c->dz5;
    fin.loss = c->loss;
    fin.grad_scale = 2.f / (float)((double)n * h * w);
    e = forward(c, x, n, h, w, fin, cs);
    if (e != cudaSuccess) return e;
    float *G = c->grads;
    // layer 4
    e = launch_wgrad_edge(c->dz5, c->act[3], 0, n, h, w, G + off_w(4), G + off_b(4), cs);
    ConvArgs a = conv_args(c, n, h, w);
    a.in_plane = c->dz5;
    a.wpack = c->pack + kPB4;
    a.mode = kGate;
    a.gate = c->act[3];
    a.out = c->g[0];
    if (e == cudaSuccess) e = launch_in1(a, cs);
    // layers 3, 2, 1: weight gradient from (input, dZ), then dZ of the layer below
    const int bw[4] = {0, kPB1, kPB2, kPB3};
    int cur = 0;
    for (int l = 3; l >= 1 && e == cudaSuccess; --l) {
        e = launch_wgrad_mid(c->act[l - 1], c->g[cur], n, h, w, G + off_w(l), G + off_b(l), c->err, cs);
        if (e != cudaSuccess) break;
        a = conv_args(c, n, h, w);
        a.in = c->g[cur];
        a.wpack = c->pack + bw[l];
        a.mode = kGate;
        a.gate = c->act[l - 1];
        a.out = c->g[1 - cur];
        e = launch_mid(a, 32, cs);
        cur = 1 - cur;
    }
    // layer 0
    if (e == cudaSuccess) e = launch_wgrad_edge(x, c->g[cur], 1, n, h, w, G + off_w(0), G + off_b(0), cs);
    return e;
}

int check_dims(int n, int h, int w) {
    return (n >= 1 && h >= 1 && w >= 1 && (double)n * h * w < 2e9 && h <= 65535 * kStrip && n <= 65535)
               ? WV_OK
               : WV_ERR_ARG;
}

}  // namespace

extern "C" {

size_t wv_cnn_param_count(void) { return (size_t)kParams; }

int wv_cnn_create(const float *params_host, wv_cnn **out) {
    if (!params_host || !out) return WV_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return WV_ERR_CUDA;
    }
    wv_cnn *c = new (std::nothrow) wv_cnn();
    if (!c) return WV_ERR_OOM;
    cudaGetDevice(&c->device);
    bool ok = cudaMalloc(&c->params, sizeof(float) * kParams) == cudaSuccess &&
              cudaMalloc(&c->grads, sizeof(float) * kParams) == cudaSuccess &&
              cudaMalloc(&c->m, sizeof(float) * kParams) == cudaSuccess &&
              cudaMalloc(&c->v, sizeof(float) * kParams) == cudaSuccess &&
              cudaMalloc(&c->pack, kPackBytes) == cudaSuccess && cudaMalloc(&c->loss, 64) == cudaSuccess &&
              cudaMalloc(&c->err, 64) == cudaSuccess;
    if (ok)
        ok = cudaMemcpy(c->params, params_host, sizeof(float) * kParams, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemset(c->m, 0, sizeof(float) * kParams) == cudaSuccess &&
             cudaMemset(c->v, 0, sizeof(float) * kParams) == cudaSuccess &&
             cudaMemset(c->err, 0, 64) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        wv_cnn_close(c);
        return WV_ERR_OOM;
    }
    *out = c;
    return WV_OK;
}

void wv_cnn_close(wv_cnn *c) {
    if (!c) return;
    cudaDeviceSynchronize();
    for (void *p : c->owned) cudaFree(p);
    cudaFree(c->params);
    cudaFree(c->grads);
    cudaFree(c->m);
    cudaFree(c->v);
    cudaFree(c->pack);
    cudaFree(c->loss);
    cudaFree(c->err);
    delete c;
}

int wv_cnn_get_params(wv_cnn *c, float *host) {
    if (!c || !host) return WV_ERR_ARG;
    return cudaMemcpy(host, c->params, sizeof(float) * kParams, cudaMemcpyDeviceToHost) == cudaSuccess ? WV_OK
                                                                                                       : WV_ERR_CUDA;
}

int wv_cnn_set_params(wv_cnn *c, const float *host) {
    if (!c || !host) return WV_ERR_ARG;
    c->packed = false;
    c->step = 0;
    if (cudaMemset(c->m, 0, sizeof(float) * kParams) != cudaSuccess ||
        cudaMemset(c->v, 0, sizeof(float) * kParams) != cudaSuccess)
        return WV_ERR_CUDA;
    return cudaMemcpy(c->params, host, sizeof(float) * kParams, cudaMemcpyHostToDevice) == cudaSuccess ? WV_OK
                                                                                                       : WV_ERR_CUDA;
}

int wv_cnn_get_state(wv_cnn *c, float *m_host, float *v_host, int *steps) {
    if (!c || !m_host || !v_host || !steps) return WV_ERR_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(m_host, c->m, sizeof(float) * kParams, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(v_host, c->v, sizeof(float) * kParams, cudaMemcpyDeviceToHost) != cudaSuccess)
        return WV_ERR_CUDA;
    *steps = c->step;
    return WV_OK;
}

int wv_cnn_set_state(wv_cnn *c, const float *m_host, const float *v_host, int steps) {
    if (!c || !m_host || !v_host || steps < 0) return WV_ERR_ARG;
    if (cudaMemcpy(c->m, m_host, sizeof(float) * kParams, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->v, v_host, sizeof(float) * kParams, cudaMemcpyHostToDevice) != cudaSuccess)
        return WV_ERR_CUDA;
    c->step = steps;
    return WV_OK;
}

int wv_cnn_forward(wv_cnn *c, const float *x_dev, float *y_dev, int n, int h, int w, void *cuda_stream) {
    if (!c || !x_dev || !y_dev || check_dims(n, h, w) != WV_OK) return WV_ERR_ARG;
    if (ensure_workspace(c, (size_t)n * h * w) != WV_OK) return WV_ERR_OOM;
    ConvArgs fin;
    memset(&fin, 0, sizeof(fin));
    fin.mode = kLastOut;
    fin.y = y_dev;
    return forward(c, x_dev, n, h, w, fin, (cudaStream_t)cuda_stream) == cudaSuccess ? WV_OK : WV_ERR_CUDA;
}

int wv_cnn_gradients(wv_cnn *c, const float *x_dev, const float *t_dev, int n, int h, int w, float *grads_host,
                     float *loss_host, void *cuda_stream) {
    if (!c || !x_dev || !t_dev || check_dims(n, h, w) != WV_OK) return WV_ERR_ARG;
    if (ensure_workspace(c, (size_t)n * h * w) != WV_OK) return WV_ERR_OOM;
    cudaStream_t cs = (cudaStream_t)cuda_stream;
    if (forward_backward(c, x_dev, t_dev, n, h, w, cs) != cudaSuccess) return WV_ERR_CUDA;
    float loss = 0.f;
    cudaError_t e = cudaMemcpyAsync(&loss, c->loss, 4, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess && grads_host)
        e = cudaMemcpyAsync(grads_host, c->grads, sizeof(float) * kParams, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (loss_host) *loss_host = loss / (float)((double)n * h * w);
    return e == cudaSuccess ? WV_OK : WV_ERR_CUDA;
}

int wv_cnn_train_step(wv_cnn *c, const float *x_dev, const float *t_dev, int n, int h, int w, float lr,
                      float *loss_host, void *cuda_stream) {
    if (!c || !x_dev || !t_dev || check_dims(n, h, w) != WV_OK || !(lr > 0.f)) return WV_ERR_ARG;
    if (ensure_workspace(c, (size_t)n * h * w) != WV_OK) return WV_ERR_OOM;
    cudaStream_t cs = (cudaStream_t)cuda_stream;
    if (forward_backward(c, x_dev, t_dev, n, h, w, cs) != cudaSuccess) return WV_ERR_CUDA;
    c->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)c->step), c2 = 1.f - powf(b2, (float)c->step);
    k_adam<<<(kParams + 255) / 256, 256, 0, cs>>>(c->params, c->grads, c->m, c->v, kParams, lr, b1, b2, c1, c2,
                                                  1e-8f);
    pack_params(c, cs);
    if (cudaGetLastError() != cudaSuccess) return WV_ERR_CUDA;
    if (loss_host) {
        float loss = 0.f;
        if (cudaMemcpyAsync(&loss, c->loss, 4, cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
            cudaStreamSynchronize(cs) != cudaSuccess)
            return WV_ERR_CUDA;
        *loss_host = loss / (float)((double)n * h * w);
    }
    return WV_OK;
}

int wv_cnn_sync_status(wv_cnn *c) {
    if (!c) return WV_ERR_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return WV_ERR_CUDA;
    int err = 0;
    if (cudaMemcpy(&err, c->err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return WV_ERR_CUDA;
    if (err) cudaMemset(c->err, 0, 4);
    return err;
}

// Viewport decode with the post-filter: the steps of wv_decode_viewport up
// to the decoded region, reprojection into luma / chroma planes, the network
// on the luma, colour conversion in the last layer's epilogue.
int wv_decode_viewport_filtered(wv_stream *s, int frame, float yaw, float pitch, float fov, wv_cnn *c,
                                const wv_image *out) {
    if (!s || !c || !out || !out->dptr || out->width <= 0 || out->height <= 0 ||
        out->pitch_bytes < (size_t)out->width * 4 || (out->pitch_bytes % 4) != 0)
        return WV_ERR_ARG;
    if (frame < 0 || frame >= s->g.num_frames || !(fov > 0.f && fov < 3.14159f)) return WV_ERR_ARG;
    const size_t px = (size_t)out->width * out->height;
    if (ensure_workspace(c, px) != WV_OK) return WV_ERR_OOM;
    // the region decode of the plain path, then the planes instead of RGBA
    int rc = wv::decode_region(s, frame, yaw, pitch, fov, out->width, out->height);
    if (rc != WV_OK) return rc;
    int row0, rows;
    eye_view(s->g, 0, &row0, &rows);   // eye 0 (the top half of a stereo frame)
    const View v = make_view(yaw, pitch, fov, out->width, out->height, s->g.p[0].w, rows, row0);
    launch_resample(s->g, v, recon_planes(s), nullptr, nullptr, 0, s->cs, c->xbuf, c->cb, c->cr, recon_pairs(s),
                    s->err);
    release_recon(s);
    ConvArgs fin;
    memset(&fin, 0, sizeof(fin));
    fin.mode = kLastRgba;
    fin.cb = c->cb;
    fin.cr = c->cr;
    fin.rgba = (uint8_t *)out->dptr;
    fin.pitch = out->pitch_bytes;
    return forward(c, c->xbuf, 1, out->height, out->width, fin, s->cs) == cudaSuccess ? WV_OK : WV_ERR_CUDA;
}

}  // extern "C"
