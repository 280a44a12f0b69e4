/*
 * wrls.h -- C ABI of libwrls.so, a GB300 (sm_103a) implementation of the weighted
 * recursive least squares (wRLS) temporal / spatio-temporal denoiser of
 * Iglesias-Guitian, Mane, Moon, "Real-Time Denoising of Volumetric Path Tracing for
 * Direct Volume Rendering", IEEE TVCG 2020 (Sec. 4-5).
 *
 * The problem (Sec. 4, Fig. 5): a renderer produces one noisy frame per time step; the
 * denoiser keeps a persistent per-pixel state -- a linear model beta (Eq. 5), its inverse
 * covariance P (Eq. 10-11) and a temporal feature z (Eq. 12) -- reprojects it along
 * per-pixel motion (Table 2, pi(v_j) = j + v_j), updates it by wRLS against the new noisy
 * radiance (Eq. 8, 9, 11, 13, 14) and outputs a colour blended from the predictions of a
 * 5x5 neighbourhood of models (Sec. 5.3, "Spatio-temporal denoising using wRLS").
 *
 * Conventions for every entry point:
 *  - Every call returns a wrls_status; nothing throws across the ABI. On an error the
 *    call has no effect on the stream's state and wrls_last_error() describes it.
 *  - Image buffers are planar, channel-major, row-major, tightly packed:
 *    element (c, y, x) of a C-channel W x H image is at index (c * H + y) * W + x.
 *    All are binary32 (float).
 *  - Device buffers are CUDA device pointers of the current device. The caller owns
 *    every input and output buffer; the stream owns its state.
 *  - Work is enqueued asynchronously on the stream's CUDA stream (see
 *    wrls_stream_set_cuda_stream); an output is complete once that stream is
 *    synchronised. The library never allocates per frame.
 *  - A stream object may be used by one host thread at a time.
 */
#ifndef WRLS_H
#define WRLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WRLS_OK = 0,
    WRLS_ERR_INVALID_ARG = 1, /* a null/misaligned pointer, a bad size or parameter */
    WRLS_ERR_OOM = 2,         /* device allocation failed at create time */
    WRLS_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
    WRLS_ERR_STATE = 4,       /* the object is in a state that forbids the call */
    WRLS_ERR_TIMEOUT = 5      /* a bounded device-side wait gave up */
} wrls_status;

/* Storage format of the per-pixel state (computation is always binary32). The 16-bit formats
 * store beta, z and the Cholesky factor of P / s (s a per-pixel power of two, P / s = L L^T,
 * so the decoded P is positive semi-definite) as 16-bit values, two per 32-bit word, with the
 * exponent of s in the last word (52 B). With the paper's forgetting factor a frame changes the
 * state by about (1 - lambda) = 0.2 % relative, less than BF16's rounding step and a few of
 * FP16's: over long static histories the 16-bit states lag the binary32 one (FP16 by about
 * 1e-2 of the colour, BF16 by several 1e-2); see the precision tests. */
typedef enum {
    WRLS_STATE_F32 = 0,   /* 25 binary32 values per pixel (100 B) */
    WRLS_STATE_BF16 = 1,  /* 25 bfloat16 values, P as a scaled Cholesky factor (52 B) */
    WRLS_STATE_F16 = 2    /* 25 binary16 values, P as a scaled Cholesky factor (52 B); beta and z
                             (and so the radiance) must stay below 65504 in magnitude */
} wrls_state_precision;

/*
 * Parameters. Fill with wrls_params_default() and change fields as needed;
 * struct_size must stay sizeof(wrls_params) (ABI versioning).
 */
typedef struct wrls_params {
    uint32_t struct_size;
    float lambda;        /* forgetting factor, Sec. 5.2 (Eq. 10-11); default 0.998 */
    float h;             /* wRLS bandwidth, Sec. 5.3 (Eq. 13); default 0.75 */
    float alpha;         /* temporal-feature history weight, Eq. 12 (Sec. 6); default 0.75 */
    float eps;           /* Eq. 13 epsilon; default 1e-4 */
    float p0_delta;      /* P of a (re)started pixel = p0_delta * I; default 1 */
    float sigma_s;       /* blend: spatial Gaussian std (pixels); default 1 */
    float h_s;           /* blend: bandwidth on the Eq. 13 distance of features; default 0.75 */
    float p_trace_max;   /* wind-up guard: P <- P0 when trace(P) > p_trace_max or a
                            diagonal entry <= 0; 0 (default) = off */
    int32_t radius;      /* blend window radius: 2 = 5x5 (Sec. 5.3, default); 0 = temporal only */
    int32_t weight_mode; /* 0 = wRLS weight Eq. 13 (default); 1 = RLS, w = 1 (Eq. 10);
                            2 = sample-variance weight, the alternative Sec. 5.3 sets aside:
                            w = exp(-3 sigma_j^2 / ((min(|I~_j|, |z_j|) + eps)^2 h^2)), the
                            Eq. 13 form with ||I~ - z||^2 replaced by its expectation
                            3 sigma^2 under the caller's per-pixel variance sigma_j^2 (the
                            variance plane is then required; a negative or non-finite
                            variance gives w = 0) */
    int32_t clamp_mode;  /* 0 = clamp history to the 3x3 min/max of I~ (Eq. 12 Psi); 1 = off */
    int32_t blend_mode;  /* 0 = neighbour k's model predicts pixel i: p_i . beta_k (default);
                            1 = bilateral average of the neighbours' own predictions */
    int32_t feature_mode;/* 0 = p = [1, z] (Sec. 5.1, d = 4, default); 1 = p = [1] (no feature) */
    int32_t init_mode;   /* 0 = restarted pixels start from beta = 0 (default);
                            1 = feature pass-through, beta_c = e_{c+1} (prediction = z_c) */
    int32_t state_precision; /* wrls_state_precision; default WRLS_STATE_F32 */
    int32_t n_features;  /* G-buffer feature planes the caller passes (features argument);
                            the paper's predictor uses none of them (Sec. 4, 5.3) */
    int32_t n_gbuf;      /* 0 (default, the paper's predictor) .. 4: the first n_gbuf feature
                            planes are appended to the predictor, p = [1, z, g_1..g_n]
                            (d = 4 + n), or [1, g_1..g_n] (d = 1 + n) with feature_mode 1 --
                            the G-buffer regression of RLS denoisers that Sec. 2.1 and
                            Sec. 5.2-5.3 discuss. Requires n_features >= n_gbuf. A non-finite
                            G-buffer value enters p as 0 and gives the sample weight 0 */
    int32_t reproj_filter; /* 0 = bilinear fetch of the reprojected model (default);
                              1 = the model of the nearest pixel, floor(q + 0.5) per axis */
} wrls_params;

/*
 * Extended path. Parameters with n_gbuf > 0, weight_mode 2 or reproj_filter 1 run on a
 * separate pair of kernels (one thread per pixel, binary32 state of 3d + d(d+1)/2 + 3 planes
 * per pixel: beta[c][a] at plane c*d + a, the upper triangle of P row by row, then z). They
 * need state_precision WRLS_STATE_F32 (WRLS_ERR_INVALID_ARG otherwise), take no blend tile
 * configuration other than 0, and are not accepted by the batched ticks.
 */

typedef struct wrls_stream wrls_stream;
struct wrls_frame_io; /* one frame's buffers, defined with the batched tick below */

/* Fill *p with the defaults above (the paper's constants where it gives them: lambda, h,
 * alpha and the 5x5 window of Sec. 5.2-6). */
void wrls_params_default(wrls_params* p);

/* Device bytes a stream of w x h pixels holds for its state (two copies: the
 * reprojection of Sec. 5.3 reads frame t-1 while frame t is written). 0 on bad args.
 * Used for admission by device memory. */
size_t wrls_state_bytes(int width, int height, const wrls_params* p);

/* Create a stream for w x h frames (1 <= w, h <= 16384). Allocates the per-pixel state of
 * Sec. 5.3 (beta of Eq. 5, P of Eq. 10-11, z of Eq. 12; two copies, the history buffer) with
 * cudaMalloc on the current device (WRLS_ERR_OOM on failure). The first frame after
 * create (or after wrls_stream_reset) restarts every pixel. On success *out owns the
 * stream; release it with wrls_stream_destroy. */
wrls_status wrls_stream_create(int width, int height, const wrls_params* p, wrls_stream** out);

/* Set the CUDA stream (a cudaStream_t passed as void*) that later calls enqueue on (not in
 * the paper).
 * NULL selects the legacy default stream (the default after create). */
wrls_status wrls_stream_set_cuda_stream(wrls_stream* s, void* cuda_stream);

/*
 * Denoise one frame (Sec. 5.3): reproject, Eq. 12 feature, Eq. 13 weight, Eq. 8/14/9/11
 * update, 5x5 blend. All pointers are device pointers:
 *   radiance  3 x H x W, noisy linear HDR colour I~(t); required. A pixel with a
 *             non-finite channel is a missing sample (weight 0, it leaves its model
 *             unchanged apart from the forgetting factor).
 *   variance  H x W per-pixel variance sigma^2 of the sample, or NULL; used only by
 *             weight_mode 2 (required there).
 *   features  n_features x H x W G-buffer planes, or NULL; the first n_gbuf planes enter
 *             the predictor (required when n_gbuf > 0).
 *   motion    2 x H x W (v_x plane, then v_y plane) in pixels, backward: the previous
 *             position of pixel j is j + v_j (Table 2). Non-finite or out-of-image
 *             previous positions restart the pixel.
 *   out       3 x H x W denoised colour; must not overlap any input.
 * Pointers must be 4-byte aligned. Asynchronous on the stream's CUDA stream.
 */
wrls_status wrls_denoise_frame(wrls_stream* s, const float* radiance, const float* variance,
                               const float* features, const float* motion, float* out);

/*
 * Same as wrls_denoise_frame (Sec. 5.3) with HOST buffers (pinned memory gives asynchronous copies):
 * copies radiance and motion to device buffers the stream owns (allocated on the first
 * call and kept until destroy), denoises, and copies the result back to `out`. Returns
 * after enqueuing; `out` is valid once the stream's CUDA stream is synchronised.
 * variance and features may be NULL unless weight_mode 2 or n_gbuf > 0 needs them (then
 * the variance plane and the first n_gbuf feature planes are copied as well).
 */
wrls_status wrls_denoise_frame_host(wrls_stream* s, const float* radiance, const float* variance,
                                    const float* features, const float* motion, float* out);

/*
 * Denoise n consecutive frames of one stream in one call (the per-frame computation of
 * Sec. 5.3; running the blend of one frame beside the update of the next is not in the
 * paper), for callers that hold several frames at once (offline denoising of a recorded
 * sequence, throughput runs). Results are
 * those of n calls of wrls_denoise_frame. The frames' updates run in order on the stream's
 * CUDA stream; the blend of frame t runs on a second CUDA stream that the library creates
 * on the first call, so it overlaps the update of frame t+1 (both read the state of frame t).
 * The first call also adds a third state copy (one more wrls_state_bytes / 2 of device
 * memory; synchronises the stream once), so that the update of frame t+2 need not wait for
 * the blend of frame t; the update of frame t+3, which overwrites that copy, waits for it
 * through an event (t+2 with two copies, if the allocation failed).
 * The memory-bound update and the arithmetic-bound blend then share the GPU. Before
 * returning, the stream's CUDA stream is made to wait for the last blend, so all n outputs
 * are complete once it is synchronised. frames[i].stream must be s or NULL; each frame
 * follows the rules of wrls_denoise_frame, and the output of frame i must not overlap any
 * buffer of frame i+1. With n = 1 the frame runs as wrls_denoise_frame. Kernel timing (wrls_stream_enable_timing) records each kernel on the CUDA stream
 * it runs on. Asynchronous.
 */
wrls_status wrls_denoise_sequence(wrls_stream* s, const struct wrls_frame_io* frames, int n);

/*
 * wrls_denoise_sequence (Sec. 5.3 per frame) with HOST buffers (pinned memory gives
 * asynchronous copies): for
 * each frame the inputs (radiance, motion; variance and G-buffer planes when the parameters
 * use them) are copied to one of three device slots on a copy stream, the frame is denoised
 * as by wrls_denoise_sequence, and the output is copied back on a second copy stream, so
 * that the input copy of frame t+1, the kernels of frame t and the output copy of frame t-1
 * can run at once. Events keep a slot from being refilled before the kernels that read it
 * (and its output from being overwritten before it was copied back). The first call
 * allocates the three slots (kept until destroy) and the copy streams. Before returning,
 * the stream's CUDA stream is made to wait for the last output copy and the last blend, so
 * every host output is complete once it is synchronised; the host buffers must stay valid
 * until then. frames[i].stream must be s or NULL. Kernel timing is not recorded for these
 * frames. Asynchronous.
 */
wrls_status wrls_denoise_sequence_host(wrls_stream* s, const struct wrls_frame_io* frames, int n);

/* Not in the paper: CTAs per SM of the persistent blend kernels (blend configurations 4-9)
 * when they overlap an update in wrls_denoise_sequence: fewer leave the update room on every SM. 0 = as many
 * as fit; default 3 (measured at 1080p, binary32 state, configuration 9: 120.7 us per frame with
 * 3, 123.6 us with 2, about 235 us with 1; 16-bit state, configuration 8, whose CTAs are twice
 * as large: the same with 2 and 3). */
wrls_status wrls_stream_set_overlap(wrls_stream* s, int blend_ctas_per_sm);

/* The next frame restarts every pixel (frame-0 behaviour: beta and P at their initial
 * values, z from the sample; the paper restarts a pixel only on disocclusion, Sec. 5.3). */
wrls_status wrls_stream_reset(wrls_stream* s);

/* Synchronise the stream's pending work and free it. NULL is a no-op. */
void wrls_stream_destroy(wrls_stream* s);

/*
 * Copy the current per-pixel state of Sec. 5.3 (beta Eq. 5, P Eq. 10-11, z Eq. 12), decoded
 * to binary32, into `dst` (device,
 * 25 x H x W planar): planes 0-11 beta[c][a] (channel c, coefficient a, plane c*4+a),
 * planes 12-21 the upper triangle of P row by row (00,01,02,03,11,12,13,22,23,33),
 * planes 22-24 z. Streams on the extended path write 3d + d(d+1)/2 + 3 planes in the
 * same order (beta[c][a] at plane c*d + a). WRLS_ERR_STATE before the first frame.
 */
wrls_status wrls_stream_read_state(wrls_stream* s, float* dst);

/*
 * Load a per-pixel state (checkpoint / resume, session migration; not in the paper): `src`
 * (device, caller-owned, same planar layout and plane count as wrls_stream_read_state) becomes
 * the stream's current state, encoded in its format (the 16-bit formats round beta and z and
 * store the Cholesky factor of P scaled by a power of two, as the update does); the next frame reprojects
 * from it instead of starting over. Asynchronous on the stream's CUDA stream; `src` may be
 * reused once that stream has passed this call. A state read from a stream with the same
 * size and parameters resumes it exactly with the binary32 format.
 */
wrls_status wrls_stream_write_state(wrls_stream* s, const float* src);

/*
 * State health (not in the paper): the covariance wind-up that the optional reset guard
 * p_trace_max bounds, positive definiteness of P and non-finite values, computed from the
 * current state copy on the stream's CUDA stream; the call waits for the result. trace(P) and
 * the diagonal are taken over the block the predictor uses (the 1 x 1 block with
 * feature_mode 1). WRLS_ERR_STATE before the first frame; a small device buffer is allocated
 * on the first call (WRLS_ERR_OOM if that fails).
 */
typedef struct wrls_state_stats {
    uint64_t frames;        /* frames denoised since create */
    double p_trace_max;     /* max over pixels of trace(P) */
    double p_trace_mean;    /* mean over pixels of trace(P) */
    double p_diag_min;      /* min over pixels of the smallest diagonal entry of P (> 0 for SPD P) */
    uint64_t nonfinite;     /* state values (beta, P, z) that are NaN or infinite */
} wrls_state_stats;
wrls_status wrls_stream_state_stats(wrls_stream* s, wrls_state_stats* out);

/* Frames denoised since create (0 for NULL). */
uint64_t wrls_stream_frames(const wrls_stream* s);

/*
 * Autotuner of the blend kernel's tile shape (not in the paper): times every blend tile
 * configuration on the
 * stream's current state, `reps` launches each (>= 1), on the stream's CUDA stream, and
 * keeps the fastest for later frames. Configurations (output tile rows x output rows per
 * thread): 0: 16x4, 1: 8x4, 2: 16x2, 3: 32x4 with one CTA per tile; 4: 16x2, 5: 16x2,
 * 6: 8x2, 7: 16x4 with persistent CTAs whose windows are filled by TMA bulk tensor copies,
 * double-buffered (4, 6: the next window arrives while the current one is blended) or single
 * (5, 7: more CTAs per SM) (binary32 state, images of at least 40 x 20 pixels); 8: 16 rows,
 * 9: 8 rows, with each thread blending 2 adjacent columns x 2 rows from a TMA-filled window
 * (64-column tiles; images of at least 72 x 20 pixels; with a 16-bit state the packed
 * words are copied as they are and decoded in shared memory). All configurations give bitwise identical outputs. Requires one
 * denoised frame; `out` (device, 3 x H x W) is overwritten and ends up holding the current
 * frame's output. times_ms (optional, WRLS_BLEND_CONFIGS entries) receives the mean time per
 * launch (-1 for a configuration the state format does not offer) and *chosen (optional)
 * the selected configuration. Synchronises the stream. After wrls_stream_create the
 * configuration is 9 for binary32 state on images of at least 2^19 pixels (and 72 x 20), else
 * 2. wrls_batch_tick uses each stream's configuration; wrls_batch_tick_static uses a
 * one-CTA-per-tile configuration of the same tile rows (2 for configurations 8 and 9).
 * Streams on the extended path have
 * one blend configuration: every time is reported as -1 and 0 is chosen, without a launch.
 */
#define WRLS_BLEND_CONFIGS 10
wrls_status wrls_stream_autotune(wrls_stream* s, float* out, int reps, float* times_ms, int* chosen);

/* Select a blend tile configuration (0..WRLS_BLEND_CONFIGS-1; kernel tiling, not in the
 * paper) directly; configurations
 * 4-7 need the binary32 state (WRLS_ERR_INVALID_ARG otherwise). */
wrls_status wrls_stream_set_blend_config(wrls_stream* s, int config);

/*
 * Test hooks (not in the paper); `flags` replaces the previous set, 0 clears them.
 * WRLS_DEBUG_WITHHOLD_STAGE_COPY: the failure path of the bounded device-side waits. The
 * update kernel arms the mbarrier of each tile's state-window copy but does not issue the
 * copy, so the tile's bounded wait runs out (about one second of SM clocks); the kernel then
 * records WRLS_ERR_TIMEOUT in the stream's error word (read by wrls_stream_check) and
 * returns. The frame's output and state are unreliable; the CUDA context stays usable.
 * WRLS_DEBUG_NO_THIRD_COPY: the sequence entries keep two state copies, as when the
 * allocation of the third fails (the update of frame t+2 then waits for the blend of frame
 * t). Takes effect if set before the stream's first wrls_denoise_sequence or
 * wrls_denoise_sequence_host call; outputs are unchanged.
 * Returns WRLS_ERR_INVALID_ARG for a NULL stream or an unknown flag.
 */
#define WRLS_DEBUG_WITHHOLD_STAGE_COPY 1u
#define WRLS_DEBUG_NO_THIRD_COPY 2u
wrls_status wrls_stream_set_debug(wrls_stream* s, uint32_t flags);

/* Not in the paper: synchronise the stream's CUDA stream and report device-side failures of the frames
 * since the last check: WRLS_ERR_TIMEOUT if a kernel's bounded wait for its own bulk
 * copy gave up (that frame's output and state are then unreliable). Clears the record. */
wrls_status wrls_stream_check(wrls_stream* s);

/*
 * Kernel tracing (not in the paper). With timing enabled, every frame records CUDA events on the stream's
 * CUDA stream before and after each of its kernels (temporal update, spatial blend).
 * wrls_stream_kernel_times synchronises the recorded events, adds their durations to
 * *update_ms and *blend_ms (milliseconds, summed over frames), sets *frames to the number
 * of frames summed, and clears the record. Up to 8192 frames are held; older ones are
 * folded into the totals as the record fills. Enabling allocates the events; disabling
 * frees them.
 */
wrls_status wrls_stream_enable_timing(wrls_stream* s, int enable);
wrls_status wrls_stream_kernel_times(wrls_stream* s, double* update_ms, double* blend_ms,
                                     uint64_t* frames);

/* Message of the last error on the calling thread ("" if none). */
const char* wrls_last_error(void);

/*
 * ---- Batched tick: all ready frames of many streams in one graph launch ----
 *
 * One tick processes one frame of each of n streams (of any sizes) with a single CUDA
 * graph launch. The graph holds each stream's own update and blend kernels (with the
 * stream's tuned blend tile), the streams spread over four parallel branches so that the
 * blend of one stream overlaps the update of another; it is captured each tick and applied to
 * the instantiated graph with cudaGraphExecUpdate. Results are identical to calling
 * wrls_denoise_frame on each stream alone.
 */
typedef struct wrls_frame_io {
    wrls_stream* stream;
    const float* radiance;  /* device, 3 x H x W */
    const float* variance;  /* device or NULL (unused) */
    const float* features;  /* device or NULL (unused) */
    const float* motion;    /* device, 2 x H x W */
    float* out;             /* device, 3 x H x W */
} wrls_frame_io;

typedef struct wrls_batch wrls_batch;

/* Create a batch executor for up to max_streams frames per tick (batching is not in the
 * paper; each frame is the computation of Sec. 5.3). WRLS_ERR_INVALID_ARG outside
 * [1, 4096], WRLS_ERR_OOM / WRLS_ERR_CUDA if its buffers, streams or events fail. */
wrls_status wrls_batch_create(int max_streams, wrls_batch** out);

/* Set the CUDA stream (cudaStream_t as void*) ticks run on; NULL = legacy default. */
wrls_status wrls_batch_set_cuda_stream(wrls_batch* b, void* cuda_stream);

/* Run one tick over n frames (1 <= n <= max_streams; each stream at most once, all
 * streams of the same state precision and blend mode, none on the extended path). Every
 * stream uses its own blend tile configuration. Asynchronous. */
wrls_status wrls_batch_tick(wrls_batch* b, const wrls_frame_io* frames, int n);

/* Synchronise and free. NULL is a no-op. */
void wrls_batch_destroy(wrls_batch* b);

/*
 * One batched tick without an executor object (the per-frame computation of Sec. 5.3 for the
 * frames of many streams; batching itself is not in the paper): frame io[i] of stream
 * streams[i] (io[i].stream may be NULL or must equal streams[i]), 1 <= n <= 256, with the
 * rules of wrls_batch_tick. Errors: WRLS_ERR_INVALID_ARG for a NULL or mismatched stream, a
 * repeated stream or n outside [1, 256] (nothing is launched), WRLS_ERR_OOM / WRLS_ERR_CUDA
 * from creating the executor or launching.
 * The library keeps one executor per device, created on the first call on that device
 * (allocation as in wrls_batch_create) and kept until the process exits; calls are
 * serialised by a lock. The tick runs on streams[0]'s CUDA stream. Asynchronous.
 */
wrls_status wrls_denoise_batch(wrls_stream* const* streams, const struct wrls_frame_io* io, int n);

/*
 * wrls_batch_tick_static: the batched tick for callers that cannot allocate device memory.
 * The paper has no counterpart; this is an integration entry point.
 *
 * Some callers must not call cudaMalloc: a plugin living inside a host application that
 * owns the device memory budget (allocating would break its accounting or fail under its
 * cap), or a frame loop that cannot afford the implicit device synchronisation that an
 * allocation may cause. wrls_batch_create allocates a device work table, work counters and
 * pinned host buffers; this entry point allocates nothing. Its work table and its two work
 * counters live in one statically sized device array compiled into the library (10,752
 * bytes, for at most WRLS_STATIC_BATCH_MAX frames per call); every GPU that loads the
 * library holds that array until the process exits. The streams passed in were created
 * with wrls_stream_create beforehand and keep their own state; the caller passes all
 * inputs and outputs as with wrls_batch_tick.
 *
 *   frames, n      one frame of each of n streams, 1 <= n <= WRLS_STATIC_BATCH_MAX (larger n
 *                  is rejected with WRLS_ERR_INVALID_ARG); same rules as wrls_batch_tick.
 *   cuda_stream    the cudaStream_t (as void*) to enqueue on; NULL = legacy default stream.
 *
 * The first call on a device looks up the device address of the static array
 * (cudaGetSymbolAddress) with that device current and caches it for the life of the process;
 * make that first call before any stream capture. The cached address, like every stream's
 * state, belongs to the device's current context: after cudaDeviceReset do not call this
 * entry point again in the same process. Each call writes its work table into the array
 * with one small kernel whose parameter carries the table (no host buffer is read after the
 * call returns, and no host-to-device copy is made) and clears the work counters there.
 * Every call reuses the same array and overwrites what the previous call left there, so
 * calls whose work overlaps on the GPU (on different CUDA streams, or from different host
 * threads without ordering) race: serialise them on one CUDA stream. Outputs equal those of
 * wrls_batch_tick bit for bit. Asynchronous.
 */
#define WRLS_STATIC_BATCH_MAX 16
wrls_status wrls_batch_tick_static(const wrls_frame_io* frames, int n, void* cuda_stream);

/*
 * ---- The denoiser's inputs from the renderer's raw data (stateless calls) ----
 */

/* Pixel reconstruction filter parameters. Fill with wrls_recon_params_default. */
typedef struct wrls_recon_params {
    uint32_t struct_size;  /* must equal sizeof(wrls_recon_params) */
    float sigma;           /* Gaussian std in pixels; default 0.5 */
    float radius;          /* support half-width in pixels, (0, 1.5]; default 1.5 */
} wrls_recon_params;

void wrls_recon_params_default(wrls_recon_params* p);

/*
 * Pixel reconstruction filter (Sec. 4, Table 2: a pixel's light-path samples are filtered
 * into its estimate I~_j; Sec. 6: a separable Gaussian kernel):
 *   I~_j = sum_k g(x_k - x_j) g(y_k - y_j) f_k / sum_k g(x_k - x_j) g(y_k - y_j)
 * over the samples k of the 3 x 3 pixels around j at their positions (pixel centre plus
 * offset), g(d) = exp(-d^2 / (2 sigma^2)) for |d| <= radius (tested in binary32), else 0.
 *   samples   device, spp x 5 x H x W planar: element (s, k, y, x) at
 *             ((s * 5 + k) * H + y) * W + x with k = r, g, b, ox, oy; (ox, oy) is the
 *             sample's offset from the pixel centre in pixels, in [-0.5, 0.5]. A sample
 *             with a non-finite colour or offset is skipped.
 *   radiance  device, 3 x H x W output; a pixel whose window holds no weight gets NaN
 *             (the denoiser treats it as a missing sample).
 *   variance  device, H x W output or NULL: the unbiased sample variance of the pixel's own
 *             valid samples, averaged over the channels and divided by their count (the
 *             variance of the pixel's sample mean, an input of weight_mode 2); NaN with
 *             fewer than two valid samples.
 * 1 <= spp <= 1024; outputs must not overlap the samples or each other; 4-byte aligned.
 * Asynchronous on cuda_stream (a cudaStream_t as void*, NULL = legacy default).
 */
wrls_status wrls_reconstruct(int width, int height, int spp, const float* samples, const wrls_recon_params* p,
                             float* radiance, float* variance, void* cuda_stream);

/*
 * Per-pixel backward motion from the world position of the first real collision along each
 * pixel's ray (Sec. 5.3: velocities from the view matrix and per-pixel world coordinates;
 * Sec. 6 "Optical flow estimation": the collision closest to the viewer). The position is
 * projected with the previous frame's view-projection matrix:
 *   clip = M [X, Y, Z, 1]^T, q = ((clip_x / clip_w + 1) W / 2 - 0.5, (1 - clip_y / clip_w) H / 2 - 0.5),
 *   v_j = q - j  (pixel centres at integer coordinates, row 0 at the top).
 *   world           device, 3 x H x W (X, Y, Z planes) of frame t; a non-finite position
 *                   means the ray had no collision.
 *   prev_view_proj  HOST array of 16 floats, row-major M of frame t-1 (OpenGL-style clip
 *                   space); all finite.
 *   miss_policy     0: no collision -> v = 0; 1: -> NaN (the denoiser restarts the pixel).
 *                   A position behind the previous camera (clip_w <= 0) always gives NaN.
 *   motion          device, 2 x H x W output (v_x plane, v_y plane), the layout
 *                   wrls_denoise_frame takes.
 * Asynchronous on cuda_stream.
 */
wrls_status wrls_velocity_from_world(int width, int height, const float* world, const float* prev_view_proj,
                                     int miss_policy, float* motion, void* cuda_stream);

/*
 * ---- Volumetric path tracer producing the denoiser's inputs ----
 *
 * Progressive path tracing of a procedural heterogeneous volume (Sec. 3, Sec. 6): delta
 * tracking with the majorant mu_max (Eq. 4), the collision estimator of Eq. 3 (throughput
 * times the albedo colour at each real collision), next-event estimation to a directional
 * light with delta-tracked visibility and the isotropic phase function 1 / (4 pi), and the
 * environment radiance for paths that leave the volume (Eq. 1). Volume: the box [-1, 1]^3,
 * density rho(x) = min(1, sum_i a_i exp(-|x - c_i|^2 / (2 r_i^2))); transfer function:
 * mu_t = mu_max clamp((rho - tf_lo) / (tf_hi - tf_lo), 0, 1), albedo colour
 * albedo (color_lo + rho (color_hi - color_lo)). A path ends after max_bounces real
 * collisions or 2^20 tentative collisions. Random numbers: Philox4x32-10 with counter
 * (pixel index, sample index, frame, block) and key seed.
 */
typedef struct wrls_vpt_scene {
    uint32_t struct_size;     /* must equal sizeof(wrls_vpt_scene) */
    uint32_t seed[2];         /* Philox key */
    float eye[3];             /* camera position */
    float inv_view_proj[16];  /* row-major inverse view-projection: rays go from eye through
                                 inv_view_proj [ndc_x, ndc_y, 1, 1] (dehomogenised) */
    int32_t n_blobs;          /* 0..16 */
    float blobs[16][5];       /* cx, cy, cz, radius (> 0), amplitude */
    float mu_max;             /* > 0 */
    float tf_lo, tf_hi;       /* opacity ramp, tf_hi > tf_lo */
    float albedo;             /* single-scattering albedo >= 0 */
    float color_lo[3], color_hi[3];
    float light_dir[3];       /* unit vector towards the directional light */
    float light_rgb[3];       /* its radiance */
    float env_rgb[3];         /* environment radiance */
    int32_t max_bounces;      /* >= 1 */
} wrls_vpt_scene;

/*
 * Render one frame with spp samples per pixel (1..1024), all outputs device, planar:
 *   samples   spp x 5 x H x W: r, g, b and the sub-pixel offsets ox, oy of each sample (the
 *             layout wrls_reconstruct takes); ndc = ((x + 0.5 + ox) / W * 2 - 1,
 *             1 - (y + 0.5 + oy) / H * 2), offsets from the first two random numbers - 0.5.
 *   world     3 x H x W: the first real collision closest to the eye among the pixel's
 *             samples (the input of wrls_velocity_from_world); NaN where none.
 *   features  7 x H x W or NULL: depth (distance from the eye), normal (-grad rho / |grad rho|)
 *             and albedo colour at that collision; 0 where none (noisy G-buffers, Fig. 4).
 * Outputs must not overlap. Asynchronous on cuda_stream.
 */
wrls_status wrls_render_vpt(const wrls_vpt_scene* scene, int width, int height, int spp, uint32_t frame,
                            float* samples, float* world, float* features, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* WRLS_H */
