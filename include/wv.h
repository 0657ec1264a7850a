/*
 * wv.h -- C ABI of the GB300 viewport-dependent wavelet video decoder.
 *
 * The method is the wavelet-based 360-degree video codec of Groth, Fricke,
 * Castillo and Magnor, "Wavelet-Based Fast Decoding of 360 deg Videos":
 *   - frame-wise 2D fast wavelet transform, CDF 9/7 (Sec. 3.1) or the
 *     reversible LeGall 5/3 integer wavelet (Sec. 2.2);
 *   - inter-frame Haar transform along time over sets of 2^k frames, run to
 *     the last level, applied to the 2D coefficients (Sec. 3.2);
 *   - quantised coefficients stored in blocks with a per-block table
 *     (the BlockEnd pointers of Sec. 3.4);
 *   - decoding of only the viewport of the current frame for the current head
 *     pose: a low-resolution binary mask marks the region to reconstruct
 *     (Sec. 3.1), the inverse inter-frame transform runs over the needed
 *     coefficients (Sec. 3.2, 3.5), the masked 2D iFWT follows (Sec. 3.5) and
 *     a mapping pass reprojects the equirectangular result into the viewport
 *     (Sec. 3.6).
 *
 * Conventions for every call:
 *   - Return value: WV_OK (0) or a negative WV_ERR_* code; wv_strerror() names
 *     it.  Nothing is printed and nothing aborts.
 *   - Device pointers are CUDA global-memory addresses of the current device;
 *     host pointers are ordinary process memory.  The library never frees
 *     memory it did not allocate.
 *   - Decode calls are asynchronous: they enqueue kernels on the stream's CUDA
 *     stream (set at open, changed by wv_set_cuda_stream) and return before
 *     the GPU finishes; outputs are valid once that CUDA stream is
 *     synchronised.  Device-side errors are reported by wv_stream_sync_status.
 *   - A wv_stream may be used by one host thread at a time.
 *   - There is no CPU fallback: without a usable CUDA device every call that
 *     needs one returns WV_ERR_CUDA.
 *   - Angles are radians.  Yaw turns about +y (from +z toward +x), pitch about
 *     +x (positive looks up), no roll.  `fov` is the full field of view,
 *     horizontal and vertical (square pixels in the viewport).
 */
#ifndef WV_H
#define WV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WV_OK 0
#define WV_ERR_ARG (-1)      /* invalid argument (NULL, range, size)           */
#define WV_ERR_FORMAT (-2)   /* malformed or unsupported stream bytes          */
#define WV_ERR_OOM (-3)      /* caller-provided memory too small / alloc fail  */
#define WV_ERR_CUDA (-4)     /* CUDA runtime error or no device                */
#define WV_ERR_RANGE (-5)    /* value out of representable range (encoder)     */
#define WV_ERR_TIMEOUT (-6)  /* a bounded device-side wait gave up             */
#define WV_ERR_DEVICE (-7)   /* a kernel reported an inconsistency (err word)  */

#define WV_WAVELET_53 0      /* LeGall 5/3, reversible integer lifting         */
#define WV_WAVELET_97 1      /* CDF 9/7, float lifting                          */

/* Geometry and coding parameters of a stream (the header of Sec. 3.4: number
 * of frames, frame size, number of wavelet levels; plus the fields this
 * format adds).  width/height are luma sizes; with chroma_420 the Cb and Cr
 * planes are half width and half height.  Every plane side must be divisible
 * by 2^levels.  The inter-frame set holds 2^tlevels frames (Sec. 3.2);
 * num_frames is a multiple of it.  block is the side of the square
 * coefficient blocks (a power of two, 16..256).  quant 0 = dead-zone uniform
 * quantiser with step `step` (integer >= 1 for 5/3); quant 1 = the byte
 * quantiser of the paper-faithful format (9/7, block 32; streams "WVP1",
 * see wv_encode_paper). */
typedef struct {
    int width, height;
    int planes;        /* 1 (grey) or 3 (Y, Cb, Cr) */
    int chroma_420;    /* 1: Cb/Cr subsampled 2x2, centre-sited */
    int levels;        /* spatial wavelet levels, 1..6 */
    int wavelet;       /* WV_WAVELET_53 or WV_WAVELET_97 */
    int num_frames;
    int tlevels;       /* inter-frame Haar levels k, 0..3 */
    int block;
    int quant;
    float step;
    int stereo;        /* 1: top/bottom stereo frames, each eye an equirect of
                          height / 2 (eye 0 the top half); height % 64 == 0 */
} wv_stream_desc;

/* An RGBA8 output image in device memory, owned by the caller.  Row r starts
 * at dptr + r * pitch_bytes; pitch_bytes >= 4 * width. */
typedef struct {
    void *dptr;
    int width, height;
    size_t pitch_bytes;
} wv_image;

typedef struct wv_stream wv_stream;

/* ---------------------------------------------------------------------------
 * Stream lifetime
 * ------------------------------------------------------------------------- */

/* Parse the stream header and block table in `bytes` (n bytes, host memory)
 * and validate them (Sec. 3.4: header and metadata are preloaded).  Fills
 * *desc if desc != NULL and the number of device bytes wv_open_stream needs
 * in *device_bytes if device_bytes != NULL.  Returns WV_ERR_FORMAT for a
 * truncated or inconsistent stream. */
int wv_stream_query(const void *bytes, size_t n, wv_stream_desc *desc,
                    size_t *device_bytes);

/* Open a stream: validate the bytes, copy the block table and the coefficient
 * payload to the device and set up per-stream decode scratch (reconstruction
 * planes, mask, two sets of tile lists and LL_2 planes).  CDF 9/7 dead-zone
 * codes are rewritten on the device as 2q + sign(q) when every |q| <= 8191
 * (one pass over the payload; decoded results are unchanged).  The call
 * synchronises cuda_stream before it returns.  device_mem is a device
 * buffer of at least device_bytes (from wv_stream_query) that the caller
 * owns and keeps alive until wv_close_stream; pass NULL to let the library
 * allocate (and later free) it.  cuda_stream is a cudaStream_t (NULL = legacy default stream).
 * The host bytes may be freed once this call returns.  On success *out holds
 * the new stream. */
int wv_open_stream(const void *bytes, size_t n, void *device_mem,
                   size_t device_bytes, void *cuda_stream, wv_stream **out);

/* Open flags. */
#define WV_OPEN_HOST_PAYLOAD 1  /* coefficient store in host memory, see below */

/* wv_stream_query / wv_open_stream with flags (0 = the plain calls).
 * WV_OPEN_HOST_PAYLOAD keeps the coefficient payload in host memory instead
 * of copying it to the device: the library copies it into pinned,
 * device-mapped host memory that it allocates (and frees at close), and the
 * tile decoder reads the blocks each viewport needs directly from there.
 * On a Grace-Blackwell node those reads travel over NVLink-C2C, so a video
 * far larger than HBM can be decoded with only the per-stream scratch on
 * the device (Sec. 3.5 streams the viewport's coefficients from storage;
 * here the GPU fetches exactly the coefficients it needs).  Decoded results
 * are identical to the device-resident store.  device_bytes then excludes
 * the payload (query with the same flags).  Returns WV_ERR_ARG for unknown
 * flags and WV_ERR_OOM when pinned host memory cannot be allocated. */
int wv_stream_query_ex(const void *bytes, size_t n, int flags,
                       wv_stream_desc *desc, size_t *device_bytes);
int wv_open_stream_ex(const void *bytes, size_t n, void *device_mem,
                      size_t device_bytes, void *cuda_stream, int flags,
                      wv_stream **out);

/* Use another CUDA stream for the following calls on s. */
int wv_set_cuda_stream(wv_stream *s, void *cuda_stream);

/* Release the stream object (and its device memory if the library allocated
 * it).  Waits for work already enqueued on the stream's CUDA stream. */
void wv_close_stream(wv_stream *s);

/* Describe an error code (static string). */
const char *wv_strerror(int code);

/* ---------------------------------------------------------------------------
 * Decoding
 * ------------------------------------------------------------------------- */

/* Decode the viewport of frame `frame` seen from head pose (yaw, pitch) with
 * field of view fov into out (RGBA8, out->width x out->height, device).
 * Steps (all on the GPU, enqueued on the stream's CUDA stream):
 *   1. footprint: every viewport pixel is projected onto the equirectangular
 *      frame and the 32-pixel cells its bilinear taps touch are marked (the
 *      low-resolution binary mask of Sec. 3.1);
 *   2. the mask becomes a list of output tiles;
 *   3. per tile, the needed coefficients of every level are gathered,
 *      dequantised and rebuilt along time (inverse inter-frame Haar, Sec.
 *      3.2/3.5) and all levels of the 2D iFWT run in one pass (Sec. 3.1);
 *   4. the decoded region is reprojected into the viewport with bilinear
 *      filtering and converted from YCbCr (BT.709, full range) to RGBA
 *      (Sec. 3.6).
 * Grey streams give R = G = B = Y.  Returns WV_ERR_ARG for a frame outside
 * [0, num_frames), fov outside (0, pi) or a bad image. */
/* Steps 1, 2 and the coarse levels of step 3 run on a CUDA stream the
 * library creates for the wv_stream (highest priority), into one of two
 * sets of scratch buffers that alternate between calls; the remaining
 * levels wait for them (CUDA event) and run with step 4 on the stream's
 * CUDA stream.  So consecutive calls overlap, and `out` is complete once the
 * stream's CUDA stream has passed this call's work, as for every decode
 * call.  A call made while the stream's CUDA stream is being captured into
 * a CUDA graph records every step on that stream, and the wv_stream decodes
 * serially from then on (graph replays never race with later calls). */
int wv_decode_viewport(wv_stream *s, int frame, float yaw, float pitch,
                       float fov, const wv_image *out);

/* wv_decode_viewport for one eye of a top/bottom stereo stream (eye 0: the
 * top half of the frame, 1: the bottom half; each half is an equirect of
 * height / 2 rows and the bilinear taps clamp to its rows).  Mono streams
 * accept eye 0 only (WV_ERR_ARG otherwise). */
int wv_decode_viewport_eye(wv_stream *s, int frame, int eye, float yaw, float pitch,
                           float fov, const wv_image *out);

/* One viewport request of a batch.  The fields after `out` select foveated
 * decoding (Sec. 3.7): with fovea = 1 the details of wavelet level 1 (the
 * finest) are decoded only in mask cells whose centre lies within r1 of the
 * gaze and those of level 2 only within r2; elsewhere they are taken as zero
 * and the inverse transform still runs over the whole viewport.  The
 * distance of a cell is the larger of its horizontal and vertical angle from
 * the gaze as the viewer sees it (x right, y up, z forward:
 * max(|atan2(x, z) - gaze_x|, |atan2(y, z) - gaze_y|)), so the regions are
 * rectilinear; cells behind the viewer count as infinitely far.  gaze_x and
 * gaze_y are radians relative to the view centre; r1 and r2 are radians (a
 * negative radius keeps nothing of its level, an infinite one everything).
 * With fovea = 0 the gaze fields are ignored. */
typedef struct {
    wv_stream *s;
    int frame;
    float yaw, pitch, fov;
    wv_image out;
    int fovea;
    float gaze_x, gaze_y;
    float r1, r2;
    int eye;           /* stereo streams: 0 top, 1 bottom; mono: 0 */
} wv_request;

/* Decode n viewport requests, possibly of different streams, sizes, fields
 * of view and foveation settings, as one batch enqueued on cuda_stream
 * (NULL = legacy default stream): one CUDA graph whose tile decode is one
 * persistent launch per decode class (see wv_batch_decode).  Each result
 * equals the result of wv_decode_viewport for the same request (foveated
 * requests: of the foveated decode).  Uses a batch context per device that
 * the library creates on first use and keeps until
 * wv_release_default_batch(); calls from several host threads are
 * serialised.  Returns WV_ERR_ARG for an invalid request (the fields checked
 * by wv_decode_viewport, fovea not 0/1, a non-finite gaze or NaN radius) and
 * WV_ERR_OOM when the batch's device memory cannot be allocated. */
int wv_decode_batch(const wv_request *reqs, int n, void *cuda_stream);

/* Release the per-device contexts of wv_decode_batch (waits for their work). */
void wv_release_default_batch(void);

/* ---------------------------------------------------------------------------
 * Batch contexts (batched decoding with explicit control)
 * ------------------------------------------------------------------------- */

typedef struct wv_batch wv_batch;

/* Statistics of the last wv_batch_decode. */
typedef struct {
    int requests;        /* requests of the batch */
    int surfaces;        /* decode targets: distinct (stream, frame) of the
                            unfoveated requests + one per foveated request */
    int coarse_tiles;    /* coarse tiles decoded (levels L..3) */
    int fine_tiles;      /* output tiles decoded (levels 2..1) */
    size_t bytes;        /* device memory held by the context */
    double ms[4];        /* with wv_batch_set_timing(b, 1): footprint, tile
                            lists, tile decode, reprojection (milliseconds,
                            summed over the waves) */
    int waves;           /* waves of decode targets the batch ran in */
} wv_batch_info;

/* Create a batch context on the current device whose launches go to
 * cuda_stream (NULL = legacy default stream).  The context allocates its
 * device memory (per decode target: reconstruction and LL_2 planes, tile
 * stamps and lists) and a pinned host staging buffer on demand, growing them
 * when a batch needs more; it never shrinks them before wv_batch_close.
 * Decode targets run in waves that share one device region (see
 * wv_batch_set_memory_limit), so the device memory stays bounded by the
 * limit plus the job tables whatever the number of requests. */
int wv_batch_create(void *cuda_stream, wv_batch **out);

/* Wait for the context's work and free it. */
void wv_batch_close(wv_batch *b);

/* Decode n requests as one batch: one CUDA graph of the upload of the job
 * tables from pinned host memory and the clearing of the counters, then per
 * wave of decode targets (1) clearing of the wave's stamps, (2) the
 * footprint of every request of the wave, (3) the tile lists of every decode
 * target of the wave, (4) per decode class (wavelet and 1 + tlevels
 * coefficient frames) one persistent tile-decode launch over every coarse
 * tile (levels L..3), then every output tile (levels 2..1) of its targets,
 * and (5) the reprojection of every request of the wave.  Unfoveated
 * requests of the same stream and frame share one decode target, so a tile
 * several of them need is decoded once; a foveated request (Sec. 3.7) has
 * its own.  Targets are grouped into waves in request order.  The
 * graph is reused while the batch keeps its shape; the call returns before
 * the GPU finishes (outputs valid once the context's CUDA stream is
 * synchronised).  The streams and output images must stay alive until then;
 * the request array may be reused as soon as the call returns. */
int wv_batch_decode(wv_batch *b, const wv_request *reqs, int n);

/* Use another CUDA stream for later launches (ordered after the earlier ones). */
int wv_batch_set_cuda_stream(wv_batch *b, void *cuda_stream);

/* Device bytes a batch of these requests needs in the context (admission
 * control: a server can compare it with the free device memory). */
int wv_batch_device_bytes(wv_batch *b, const wv_request *reqs, int n, size_t *bytes);

/* Wait for the context's last batch and read its device error word: WV_OK,
 * or the first error a kernel recorded (WV_ERR_TIMEOUT: a bounded wait of
 * the tile decode gave up; WV_ERR_DEVICE: an internal size check failed);
 * the word is then cleared. */
int wv_batch_sync_status(wv_batch *b);

/* Wait for the last batch and report its statistics. */
int wv_batch_stats(wv_batch *b, wv_batch_info *info);

/* on = 1 (default): unfoveated requests of the same stream and frame share
 * one decode target; on = 0: every request decodes its own (the work of
 * independent wv_decode_viewport calls, scheduled as one batch). */
int wv_batch_set_sharing(wv_batch *b, int on);

/* on = 1 (default): decode targets whose streams the strip fine pass takes
 * (dead-zone codes, three or more levels, one or two coefficient frames)
 * decode levels 2 and 1 as 224 x 64 strips (k_strip_batch, foveation
 * included), after the class's coarse tiles; on = 0: square tiles for
 * every target.  Outputs are identical either way. */
int wv_batch_set_strips(wv_batch *b, int on);

/* Polls of the tile decode's bounded wait (a fine tile waiting for its
 * target's coarse tiles) before it gives up, records WV_ERR_TIMEOUT in the
 * batch's error word and decodes with what is there (all reads stay in
 * bounds).  Default and maximum 2^21 (about half a second); polls = 0
 * makes every such wait give up at once -- the failure path, exercised
 * without a GPU fault.  Takes effect from the next wv_batch_decode. */
int wv_batch_set_wait_limit(wv_batch *b, int polls);

/* Test hook: the next n device allocations the library makes itself
 * (wv_open_stream without caller memory, batch arenas) fail as if the device
 * were out of memory; the calls then return WV_ERR_OOM.  n = 0 clears it. */
void wv_debug_fail_device_allocs(int n);

/* on = 1: run batches as direct launches with CUDA events between the steps
 * (wv_batch_stats reports per-step times, wv_batch_completion_ms the time
 * each request completed); on = 0: CUDA graph (default). */
int wv_batch_set_timing(wv_batch *b, int on);

/* With timing on: the completion time of each of the last batch's n
 * requests (caller order), in milliseconds from the start of the batch (the
 * end of the reprojection of its wave).  Waits for the batch.  WV_ERR_ARG
 * when timing was off or n differs from the batch's request count. */
int wv_batch_completion_ms(wv_batch *b, double *ms, int n);

/* Device bytes of decode targets one wave may hold (reconstruction and LL_2
 * planes, stamps, list entries and foveation bits of its targets); a target
 * larger than the limit forms a wave of its own.  Default 1 GiB; 0 = a
 * single wave.  Outputs do not depend on it.  Takes effect from the next
 * wv_batch_decode. */
int wv_batch_set_memory_limit(wv_batch *b, size_t bytes);

/* Tile shapes: output tile tile_w x tile_h samples (64 x 64, 128 x 128,
 * 256 x 64 or 256 x 128) and coarse tile side (32 or 64 samples of LL_2) for
 * streams with this wavelet, level count and luma size.  Default 128 x 128 /
 * 64.  wv_batch_autotune times the shapes 128 x 128 / 64, 128 x 128 / 32,
 * 64 x 64 / 64, 64 x 64 / 32, 256 x 64 / 64 and 256 x 128 / 64 on the given
 * requests (reps timed launches after one warm-up per shape, one (wavelet,
 * levels, size) class at a time) and keeps the fastest.  WV_ERR_ARG for
 * other shapes. */
int wv_batch_set_tile_shape(wv_batch *b, int wavelet, int levels, int width, int height,
                            int tile_w, int tile_h, int ctile);
int wv_batch_tile_shape(wv_batch *b, int wavelet, int levels, int width, int height, int *tile_w,
                        int *tile_h, int *ctile);
int wv_batch_autotune(wv_batch *b, const wv_request *reqs, int n, int reps);

/* ---------------------------------------------------------------------------
 * Serving: a request loop with continuous batching
 * ------------------------------------------------------------------------- */

typedef struct wv_server wv_server;

typedef struct {
    int slots;             /* batches in flight at once (one CUDA stream and
                              batch context each), 1..16 */
    int max_batch;         /* requests per batch, >= 1 */
    size_t cache_bytes;    /* device bytes for resident streams; 0 = no limit */
    size_t arena_bytes;    /* device bytes for the batch contexts of all
                              slots; 0 = the free device memory minus
                              reserve_bytes */
    size_t reserve_bytes;  /* device memory left free when arena_bytes = 0 */
} wv_server_config;

/* One request of a client: as wv_request, with a stream registered by
 * wv_server_add_stream instead of a wv_stream. */
typedef struct {
    int stream_id;
    int frame;
    float yaw, pitch, fov;
    wv_image out;
    int fovea;
    float gaze_x, gaze_y;
    float r1, r2;
    int eye;
} wv_server_request;

typedef struct {
    unsigned long long submitted, completed, failed;
    unsigned long long batches, batched_requests;   /* mean batch size = ratio */
    unsigned long long uploads, evictions;          /* stream cache */
    unsigned long long max_batch_bytes;             /* largest admitted batch */
    unsigned long long resident_bytes;              /* streams on the device */
    unsigned long long arena_bytes;                 /* batch contexts of all slots */
} wv_server_stats;

/* Start a server on the current device: `slots` CUDA streams with a batch
 * context each and one worker thread.  Whenever a slot is free and requests
 * are pending, the worker takes the oldest pending requests (at most
 * max_batch), makes their streams resident (uploading from the registered
 * host bytes, evicting the least recently used streams no batch in flight
 * reads when cache_bytes would be exceeded), admits the longest prefix whose
 * batch memory fits (arena_bytes, or the free device memory), and launches
 * it as one batch (wv_batch_decode) on the slot's CUDA stream.  Requests
 * arriving while batches run join the next batch; batches of different slots
 * overlap on the GPU.  Each request's result equals the result of decoding
 * it alone. */
int wv_server_create(const wv_server_config *cfg, wv_server **out);

/* Register a coded stream (bytes copied to pinned host memory; uploaded to
 * the device when a batch first needs it).  *stream_id numbers the streams
 * 0, 1, ... in registration order. */
int wv_server_add_stream(wv_server *sv, const void *bytes, size_t n, int *stream_id);

/* Queue a request (any thread).  The output image must stay valid until the
 * request completes.  *ticket identifies it for wv_server_poll/wait. */
int wv_server_submit(wv_server *sv, const wv_server_request *r, uint64_t *ticket);

/* 1 while the request is pending or on the GPU; WV_OK once its output is
 * written (the ticket is then released and *latency_ms, if not NULL, holds
 * the time from submission to completion); a negative code if it failed. */
int wv_server_poll(wv_server *sv, uint64_t ticket, double *latency_ms);

/* As wv_server_poll, blocking up to timeout_ms (WV_ERR_TIMEOUT after). */
int wv_server_wait(wv_server *sv, uint64_t ticket, double timeout_ms, double *latency_ms);

/* Wait until no request is pending or in flight (WV_ERR_TIMEOUT after
 * timeout_ms). */
int wv_server_drain(wv_server *sv, double timeout_ms);

int wv_server_get_stats(wv_server *sv, wv_server_stats *out);

/* Latencies (ms, submission to completion) of the requests completed since
 * the start or the last wv_server_reset_stats, in completion order: the
 * first min(cap, *n) are copied to out; *n receives their number. */
int wv_server_latencies(wv_server *sv, double *out, int cap, int *n);
int wv_server_reset_stats(wv_server *sv);

/* Stop the worker, wait for batches in flight, free everything. */
void wv_server_close(wv_server *sv);

/* ---------------------------------------------------------------------------
 * Learned post-filter (an extension; the paper has no learned component)
 * ------------------------------------------------------------------------- */

/* A residual CNN on the decoded viewport's luma that removes quantisation
 * artefacts.  Input x = Y / 255 (float, n images of h x w, row-major); five
 * 3x3 convolutions with zero padding: 1 -> 32 channels (ReLU), three
 * 32 -> 32 (ReLU), 32 -> 1; output y = x + that residual.  Parameters are a
 * flat float array, layer by layer: weights [c_out][c_in][3][3] (row dy,
 * column dx; cross-correlation), then biases [c_out]; wv_cnn_param_count()
 * floats in all.  Weights run as bf16 with fp32 accumulation on the tensor
 * cores (tcgen05); activations between layers are bf16.  Training (MSE loss,
 * Adam on fp32 master parameters) runs on the same kernels.  Calls are
 * enqueued on cuda_stream (NULL = legacy default stream); a network object
 * is used by one host thread at a time. */
typedef struct wv_cnn wv_cnn;

/* Number of floats in the parameter array (all layers). */
size_t wv_cnn_param_count(void);

/* Create a network with the given parameters (host, wv_cnn_param_count()
 * floats) on the current device. */
int wv_cnn_create(const float *params_host, wv_cnn **out);
void wv_cnn_close(wv_cnn *c);
int wv_cnn_get_params(wv_cnn *c, float *params_host);
/* Replace the parameters (and reset the optimiser state). */
int wv_cnn_set_params(wv_cnn *c, const float *params_host);

/* Optimiser state, for checkpointing and resuming training (no counterpart
 * in the paper): the Adam first and second moments (host, wv_cnn_param_count()
 * floats each, in the parameter layout) and the number of Adam steps taken
 * (its bias correction).  get waits for the device; set must follow
 * wv_cnn_set_params, which clears the state. */
int wv_cnn_get_state(wv_cnn *c, float *m_host, float *v_host, int *steps);
int wv_cnn_set_state(wv_cnn *c, const float *m_host, const float *v_host, int steps);

/* y = network(x) for n images of h x w (device float planes). */
int wv_cnn_forward(wv_cnn *c, const float *x_dev, float *y_dev, int n, int h, int w, void *cuda_stream);

/* Loss mean((y - t)^2) and its gradient with respect to every parameter
 * (host, wv_cnn_param_count() floats, same layout as the parameters);
 * synchronises cuda_stream. */
int wv_cnn_gradients(wv_cnn *c, const float *x_dev, const float *t_dev, int n, int h, int w,
                     float *grads_host, float *loss_host, void *cuda_stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
 * batch (x, t).  loss_host != NULL receives the batch loss before the step
 * (synchronises cuda_stream). */
int wv_cnn_train_step(wv_cnn *c, const float *x_dev, const float *t_dev, int n, int h, int w, float lr,
                      float *loss_host, void *cuda_stream);

/* Synchronise the device and read the network's error word (WV_ERR_TIMEOUT:
 * a bounded tensor-core wait gave up). */
int wv_cnn_sync_status(wv_cnn *c);

/* wv_decode_viewport with the post-filter: the decoded region is reprojected
 * into the viewport's luma and chroma, the network filters the luma, and the
 * last layer's epilogue converts to RGBA (8-bit luma: floor(255 y + 1/2),
 * clamped).  Enqueued on the stream's CUDA stream. */
int wv_decode_viewport_filtered(wv_stream *s, int frame, float yaw, float pitch, float fov, wv_cnn *c,
                                const wv_image *out);

/* Decode a whole plane of one frame (all tiles) -- the full-frame case, used
 * for the lossless workload and for parity checks.  dptr receives width x
 * height samples of the plane, row-major and tightly packed: uint8
 * (as_float = 0) or float32 values before rounding (as_float = 1, 8-bit
 * units, DC offset included; always the square-tile passes).  dptr == NULL
 * decodes into the stream's own reconstruction plane (as uint8, in the
 * layout of the current decode mode) for wv_resample_at. */
int wv_decode_full(wv_stream *s, int frame, int plane, void *dptr, int as_float);

/* Decode one whole plane without allocating any device memory.  The paper
 * has no counterpart: this entry point exists for callers that must not
 * allocate GPU memory themselves -- for example a plug-in whose host
 * application owns every device allocation -- but already hold a stream's
 * block table (int32 [num_frames][blocks per frame], the stream's table) and
 * coefficient payload (int16 blocks, payload_blocks of them) in device
 * memory they own.
 * desc describes the stream (host memory).  out_dev receives the plane's
 * width x height samples, row-major and tightly packed: uint8 (as_float = 0)
 * or float32 before rounding (as_float = 1), as in wv_decode_full.  Work is
 * enqueued on cuda_stream (NULL = legacy default stream).  status == NULL:
 * the call returns before the work finishes; otherwise it waits for it and
 * stores the device error word in *status (host memory): WV_OK, or
 * WV_ERR_FORMAT when a table entry was at or above payload_blocks (such an
 * entry reads as an all-zero block, never outside the payload).
 * Scratch: the tile list and counters live in one static device array of
 * 16 KB + 256 bytes that every GPU loading the library holds until the
 * process exits; planes of more than 4096 tiles of 128 x 128 samples (larger
 * than 8192 x 8192) are rejected with WV_ERR_RANGE.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress, with
 * the device current); make that first call before any stream capture.
 * All calls share the array (the error word included): calls whose work
 * overlaps on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  Returns WV_ERR_ARG for payload_blocks == 0.
 * Calls no cudaMalloc, cudaFree or other allocating routine. */
int wv_decode_plane_static(const wv_stream_desc *desc, const void *payload_dev,
                           size_t payload_blocks, const void *table_dev, int frame, int plane,
                           void *out_dev, int as_float, void *cuda_stream, int *status);

/* Wait for the stream's CUDA stream and read the device error word: WV_OK,
 * or the first error a kernel recorded since the previous call (the word is
 * then cleared). */
int wv_stream_sync_status(wv_stream *s);

/* ---------------------------------------------------------------------------
 * Inspection and measurement (tests, benchmark)
 * ------------------------------------------------------------------------- */

/* Footprint of a viewport: runs step 1 of wv_decode_viewport and copies the
 * cell mask (height/32 rows x width/32 columns of 0/1 bytes) to mask_host
 * (host memory) and the number of tiles step 2 selects to *tiles.
 * Synchronises the stream's CUDA stream. */
int wv_debug_footprint(wv_stream *s, float yaw, float pitch, float fov,
                       int out_w, int out_h, uint8_t *mask_host, int *tiles);

/* Equirectangular positions (u, v) that the viewport's pixels sample, as
 * computed on the device (float32 pairs, out_h x out_w x 2, device memory). */
int wv_debug_project(wv_stream *s, float yaw, float pitch, float fov,
                     int out_w, int out_h, float *uv_dev);

/* Resample and colour-convert the stream's reconstruction planes (filled by
 * wv_decode_full with dptr == NULL) at caller-given luma positions uv_dev
 * (device float32 pairs, out->height x out->width x 2) into out. */
int wv_resample_at(wv_stream *s, const float *uv_dev, const wv_image *out);

/* Bytes of quantised coefficients the masked iFWT of frame `frame` needs for
 * the cell mask mask_host (height/32 x width/32 bytes, host): the exact
 * dependency cone of the marked pixels through every level (synthesis
 * filter supports, symmetric extension), restricted to stored blocks,
 * 2 bytes per coefficient, summed over the coefficient frames the
 * inter-frame rebuild reads.  Host computation. */
int wv_cone_bytes(wv_stream *s, int frame, const uint8_t *mask_host,
                  unsigned long long *bytes);

/* As wv_cone_bytes with foveation: fovea_host (one byte per mask cell, host;
 * bit 0 keeps the level-1 details of the cell, bit 1 the level-2 details;
 * NULL keeps everything) drops the detail coefficients of levels 1 and 2
 * whose nominal position (coefficient index x 2^level, in luma pixels) lies
 * in a cell without the bit. */
int wv_cone_bytes_fovea(wv_stream *s, int frame, const uint8_t *mask_host,
                        const uint8_t *fovea_host, unsigned long long *bytes);

/* wv_cone_bytes split by the pass that reads the coefficients: *fine =
 * levels 1 and 2 (the fine pass; for streams of one or two levels the LL
 * band too), *coarse = levels 3 and above with the LL band (the coarse
 * pass).  Host computation. */
int wv_cone_bytes_split(wv_stream *s, int frame, const uint8_t *mask_host, unsigned long long *fine,
                        unsigned long long *coarse);

/* Algorithmic bytes of one request: runs the request's footprint on the
 * stream's CUDA stream (synchronising it), then on the host the coefficient
 * bytes its cone reads (with the request's foveation, decided in double
 * precision) and the bytes of the decoded region (marked cells x samples per
 * cell over the planes). */
int wv_request_bytes(const wv_request *r, unsigned long long *cone, unsigned long long *region);

/* Per-kernel device time of the calls since the last wv_profile_begin,
 * measured with CUDA events recorded on the stream's CUDA stream around
 * each launch. */
typedef struct {
    double ms[8];        /* footprint, select tiles, coarse decode, fine decode, resample */
    int launches[8];
    int tiles;           /* tiles decoded by the last viewport (an edge strip
                            counts as its two halves) */
} wv_profile;

/* Start recording: the following decode calls on s record events around
 * each launch and run all their steps serially on the stream's CUDA stream
 * (no overlap between viewports, so that each interval is one kernel). */
int wv_profile_begin(wv_stream *s);
/* Synchronises, sums the recorded event intervals into *out and stops. */
int wv_profile_end(wv_stream *s, wv_profile *out);

/* Number of kernel launches a wv_decode_viewport call on s makes. */
int wv_launches_per_viewport(const wv_stream *s);

/* Tile-decode organisation.  Mode 0 (default): levels L..3 of the needed
 * coarse tiles go into float LL_2 planes in one kernel (streams of three or
 * more levels), then levels 2 and 1 of the needed output tiles in a second;
 * for dead-zone streams of three or more levels the second kernel streams
 * each 224-column strip of the region down its rows in one warp (strip
 * tiles; 8-bit output only: float whole-plane decodes take mode 2), with
 * the reconstruction's chroma held as alternating Cb and Cr groups of four
 * samples; otherwise it decodes square 128-sample tiles.  Mode 1: all
 * levels of each square output tile in one kernel, repeating the coarse
 * levels per tile.  Mode 2: the coarse pass, then levels 2 and 1 of square
 * output tiles (mode 0 for streams without strip tiles).  8-bit results are
 * identical in all modes; float results identical up to float rounding
 * order for 9/7 and bit-exact for 5/3.  The reconstruction planes follow
 * the mode: decode again after changing it before wv_resample_at. */
int wv_set_decode_mode(wv_stream *s, int mode);

/* ---------------------------------------------------------------------------
 * Encoder (offline; not part of the decode path)
 * ------------------------------------------------------------------------- */

/* Device scratch (bytes) and the largest stream (bytes) wv_encode may need
 * for frames of this description. */
int wv_encode_sizes(const wv_stream_desc *desc, size_t *scratch_bytes,
                    size_t *max_stream_bytes);

/* Encode desc->num_frames frames on the GPU: DC shift and 2D FWT per frame
 * and plane (Sec. 3.1, float32 for 9/7 as in Sec. 3.3, int32 for 5/3),
 * inter-frame Haar per set (Sec. 3.2), dead-zone quantisation, blocking with
 * all-zero blocks omitted (Sec. 3.4).  planes_dev holds num_frames * planes
 * device pointers to tightly packed uint8 planes (frame-major).  The stream
 * is written to host memory out (capacity cap); *out_len receives its
 * length.  Returns WV_ERR_OOM if cap or scratch_bytes is too small and
 * WV_ERR_RANGE if a quantised coefficient does not fit in int16.
 * Synchronises cuda_stream. */
int wv_encode(const wv_stream_desc *desc, const void *const *planes_dev,
              void *scratch_dev, size_t scratch_bytes, void *out, size_t cap,
              size_t *out_len, void *cuda_stream);

/* Encode into the paper-faithful format ("WVP1", Sec. 3.3 / 3.4) on the GPU.
 * desc: quant = 1, wavelet = 9/7, block = 32 (width, height, planes,
 * chroma_420, levels, num_frames, tlevels as for wv_encode; step unused).
 * Samples are normalised to [0, 1] around 128; after the frame-wise FWT every
 * coefficient with |W| <= alpha ((l_max - l) / l_max)^2 + H(y) is dropped
 * (Eq. 3; H(y) = 1 - sin(pi y / S_y), Sec. 3.6, y the row inside the
 * subband; the approximation band uses l = l_max); after the inter-frame Haar
 * (sets of 2^tlevels frames, to the last level) the same with alpha_t and the
 * temporal level; the survivors of each coefficient frame, plane and class
 * (approximation band / detail bands) are quantised to one byte between
 * their extremes.  Output: header, per-frame offsets, per coefficient frame
 * the extremes, the BlockEnd pointers of the 32 x 32 blocks and the records
 * (index in the block | byte << 16).  Scratch and capacity from
 * wv_encode_sizes with the same desc.  Synchronises cuda_stream. */
int wv_encode_paper(const wv_stream_desc *desc, const void *const *planes_dev, void *scratch_dev,
                    size_t scratch_bytes, float alpha, float alpha_t, void *out, size_t cap,
                    size_t *out_len, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* WV_H */
