// noalloc.cu -- whole-plane decode that allocates no device memory.
//
// Callers such as a host application's plug-in, which must not allocate GPU
// memory of its own (its host owns the allocator, or allocation is forbidden
// in the context it runs in), already hold the coefficient table and blocks
// on the device and only want one plane decoded into a buffer they own.
// wv_decode_plane_static serves them: its only scratch, the tile list and
// counters of the tile-decode kernel, lives in the file-scope array below,
// which every GPU that loads the library holds until the process exits.
#include <stdint.h>

#include <mutex>

#include "wv_impl.h"

namespace {

// One plane of up to 8192 x 8192 samples: (8192 / 128)^2 = 4096 tiles.
constexpr int kStaticMaxTiles = 4096;
constexpr size_t kTilesBytes = kStaticMaxTiles * sizeof(uint32_t);
constexpr size_t kScratchBytes = kTilesBytes + 256;   // + counters and error word

static __device__ __align__(256) unsigned char g_wv_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return WV_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_wv_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return WV_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return WV_OK;
}

}  // namespace

extern "C" int wv_decode_plane_static(const wv_stream_desc *desc, const void *payload_dev,
                                      size_t payload_blocks, const void *table_dev, int frame, int plane,
                                      void *out_dev, int as_float, void *cuda_stream, int *status) {
    if (!desc || !payload_dev || !table_dev || !out_dev) return WV_ERR_ARG;
    if (payload_blocks == 0 || payload_blocks > (size_t)INT32_MAX) return WV_ERR_ARG;
    if (desc->quant != 0) return WV_ERR_ARG;   // the byte quantiser needs per-frame parameters
    wv::Geom g;
    if (wv::build_geom(*desc, &g) != WV_OK) return WV_ERR_ARG;
    if (frame < 0 || frame >= g.num_frames || plane < 0 || plane >= g.planes) return WV_ERR_ARG;
    if (g.p[plane].tiles_x * g.p[plane].tiles_y > kStaticMaxTiles) return WV_ERR_RANGE;
    void *base = nullptr;
    const int rc = scratch_address(&base);
    if (rc != WV_OK) return rc;
    uint32_t *tiles = (uint32_t *)base;
    int *counters = (int *)((char *)base + kTilesBytes);
    int *err = counters + 16;
    cudaStream_t cs = (cudaStream_t)cuda_stream;
    // the array keeps the previous call's contents: the error word must start
    // at zero; the tile list and its count are rewritten below
    if (cudaMemsetAsync(err, 0, sizeof(int), cs) != cudaSuccess) {
        cudaGetLastError();
        return WV_ERR_CUDA;
    }
    uint8_t *outs[3] = {nullptr, nullptr, nullptr};
    float *f32 = nullptr;
    if (as_float) f32 = (float *)out_dev;
    else outs[plane] = (uint8_t *)out_dev;
    wv::launch_all_tiles(g, plane, tiles, counters, cs);
    // table entries at or above payload_blocks read as absent blocks and
    // leave WV_ERR_FORMAT in the error word
    cudaError_t e = wv::launch_decode_tiles(
        g, (const int16_t *)payload_dev, (const int32_t *)table_dev, wv::frame_bands(g, frame), outs,
        f32, as_float ? plane : -1, tiles, counters, err, cs, (int)payload_blocks);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return WV_ERR_CUDA;
    if (status) {
        // wait for this call's work and hand back the device error word
        if (cudaMemcpyAsync(status, err, sizeof(int), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
            cudaStreamSynchronize(cs) != cudaSuccess) {
            cudaGetLastError();
            return WV_ERR_CUDA;
        }
    }
    return WV_OK;
}
