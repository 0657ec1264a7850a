// paper.cu -- the paper-faithful stream format ("WVP1", Sec. 3.3 / 3.4).
//
// Layout (little endian):
//   header (128 bytes)  magic "WVP1", version 1, luma width, height, planes,
//                       chroma_420, levels, num_frames, tlevels (inter-frame
//                       sets of 2^tlevels frames, transformed to the last
//                       level), block (32), blocks per frame, the two
//                       threshold constants (float, informative).
//   frame offsets       uint64 [num_frames]: byte offset of each coefficient
//                       frame's package (the per-frame metadata of Sec. 3.4).
//   per coefficient frame (stream slot order of the inter-frame set):
//     metadata          uint32 record count, uint32 0, float [planes][2][2]:
//                       (c_min, c_max) of the approximation band and of the
//                       detail bands (Sec. 3.3 quantisation);
//     BlockEnd          uint32 [blocks]: end of each block's records
//                       (exclusive, cumulative), blocks level-wise from the
//                       lowest frequency;
//     records           uint32: index inside the 32 x 32 block (y * 32 + x)
//                       | byte << 16.
// Opening a stream transcodes the records on the GPU into the decoder's
// dense block store: every block with records becomes a 32 x 32 int16 block
// holding byte + 1 (0 = absent coefficient), and the byte quantiser's
// (c_min, step) pairs ride along with each decode (tile decoder variant
// QM = 1).  Blocks without records are not stored.
#include <math.h>
#include <string.h>

#include "wv_impl.h"

namespace wv {

namespace {

struct PaperHeader {
    char magic[4];
    uint32_t version, width, height, planes, c420, levels, num_frames, tlevels, block, nbpf;
    float alpha, alpha_t;
};
static_assert(sizeof(PaperHeader) == 52, "paper header layout");

// One CTA per stored block: clear it, then place every record's byte + 1.
__global__ void k_transcode(const uint8_t *__restrict__ blob, const uint2 *__restrict__ src,
                            int16_t *__restrict__ payload) {
    const uint2 sd = src[blockIdx.x];
    int16_t *dst = payload + (size_t)blockIdx.x * 1024;
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) dst[i] = 0;
    __syncthreads();
    const uint32_t *rec = reinterpret_cast<const uint32_t *>(blob + sd.x);
    for (uint32_t i = threadIdx.x; i < sd.y; i += blockDim.x) {
        const uint32_t r = rec[i];
        const uint32_t idx = r & 0xFFFFu;
        if (idx < 1024u) dst[idx] = (int16_t)(((r >> 16) & 0xFFu) + 1u);
    }
}

}  // namespace

bool is_paper_stream(const void *bytes, size_t n) {
    return bytes && n >= 4 && memcmp(bytes, "WVP1", 4) == 0;
}

int paper_parse(const void *bytes, size_t n, wv_stream_desc *d, PaperInfo *info) {
    if (!is_paper_stream(bytes, n) || n < kHeaderBytes) return WV_ERR_FORMAT;
    PaperHeader h;
    memcpy(&h, bytes, sizeof(h));
    if (h.version != 1 || h.block != 32) return WV_ERR_FORMAT;
    d->width = (int)h.width;
    d->height = (int)h.height;
    d->planes = (int)h.planes;
    d->chroma_420 = (int)h.c420;
    d->levels = (int)h.levels;
    d->wavelet = WV_WAVELET_97;
    d->num_frames = (int)h.num_frames;
    d->tlevels = (int)h.tlevels;
    d->block = 32;
    d->quant = 1;
    d->step = 1.f;
    d->stereo = 0;
    Geom g;
    if (build_geom(*d, &g) != WV_OK || (int)h.nbpf != g.nbpf) return WV_ERR_FORMAT;
    const char *base = (const char *)bytes;
    const uint64_t nf = (uint64_t)g.num_frames;
    if (kHeaderBytes + 8 * nf > n) return WV_ERR_FORMAT;
    info->n_slots = 0;
    info->table.assign(nf * g.nbpf, -1);
    info->src.clear();
    info->qp.assign(nf * 3 * 2 * 2, 0.f);
    for (uint64_t t = 0; t < nf; ++t) {
        uint64_t off;
        memcpy(&off, base + kHeaderBytes + 8 * t, 8);
        const uint64_t ext_bytes = 16ull * g.planes, ends_bytes = 4ull * g.nbpf;
        if (off % 4 || off < kHeaderBytes || off + 8 + ext_bytes + ends_bytes > n) return WV_ERR_FORMAT;
        uint32_t count;
        memcpy(&count, base + off, 4);
        const uint64_t recs = off + 8 + ext_bytes + ends_bytes;
        if (recs + 4ull * count > n) return WV_ERR_FORMAT;
        for (int p = 0; p < g.planes; ++p)
            for (int c = 0; c < 2; ++c) {
                float lohi[2];
                memcpy(lohi, base + off + 8 + 16 * p + 8 * c, 8);
                if (!isfinite(lohi[0]) || !isfinite(lohi[1])) return WV_ERR_FORMAT;
                float *q = &info->qp[((t * 3 + p) * 2 + c) * 2];
                q[0] = lohi[0];
                q[1] = (lohi[1] - lohi[0]) / 255.f;
            }
        uint32_t prev = 0;
        for (int b = 0; b < g.nbpf; ++b) {
            uint32_t end;
            memcpy(&end, base + off + 8 + ext_bytes + 4ull * b, 4);
            if (end < prev || end > count) return WV_ERR_FORMAT;
            if (end > prev) {
                info->table[t * g.nbpf + b] = (int32_t)info->n_slots++;
                info->src.push_back(make_uint2((uint32_t)(recs + 4ull * prev), end - prev));
            }
            prev = end;
        }
        if (prev != count) return WV_ERR_FORMAT;
    }
    if (n > 0xFFFFFFFFull) return WV_ERR_FORMAT;   // record offsets are 32-bit
    return WV_OK;
}

cudaError_t paper_transcode(const void *bytes, size_t n, const PaperInfo &info, int16_t *payload,
                            cudaStream_t cs) {
    if (info.n_slots == 0) return cudaSuccess;
    void *blob = nullptr, *src = nullptr;
    cudaError_t e = cudaMalloc(&blob, n);
    if (e == cudaSuccess) e = cudaMalloc(&src, info.src.size() * sizeof(uint2));
    if (e == cudaSuccess) e = cudaMemcpyAsync(blob, bytes, n, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(src, info.src.data(), info.src.size() * sizeof(uint2), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) {
        k_transcode<<<(unsigned)info.n_slots, 256, 0, cs>>>((const uint8_t *)blob, (const uint2 *)src, payload);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (blob) cudaFree(blob);
    if (src) cudaFree(src);
    return e;
}

}  // namespace wv
