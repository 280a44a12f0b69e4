// C ABI of libwrls.so (declared in include/wrls.h): parameter handling, stream objects
// owning the per-pixel state, and the per-frame entry points.
#include <math.h>
#include <stdlib.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cudaTypedefs.h>

#include <new>

#include "wrls_internal.h"

namespace wrls {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

static size_t round_up(size_t v, size_t m) { return (v + m - 1) / m * m; }

size_t state_copy_layout(int W, int H, int precision, int* pitch, size_t* plane_stride, int nplanes) {
  const size_t p = round_up((size_t)W, 32);
  const size_t ps = round_up(p * (size_t)H, 64);
  const size_t bytes = ps * 4 * (size_t)copy_planes(precision, nplanes);
  if (pitch) *pitch = (int)p;
  if (plane_stride) *plane_stride = ps;
  return round_up(bytes, 256);
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  }
  return fn;
}

bool encode_stage_maps(StateDesc& d, const char** why) {
  d.stage_ok = false;
  d.blend_tma_ok = false;
  d.blend_tma2_ok = false;
  memset(&d.maps, 0, sizeof(d.maps));
  memset(&d.bmaps, 0, sizeof(d.bmaps));
  if (d.pitch < kStageW || d.H < kStageH) return true;  // smaller images read taps from global memory
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) { *why = "cuTensorMapEncodeTiled is not available from the driver"; return false; }
  const bool f32 = d.precision == 0;
  const cuuint32_t np = (cuuint32_t)copy_planes(d.precision, kNState);
  // 32-bit elements in every format (binary32 values or packed 16-bit pairs)
  const cuuint64_t dims[3] = {(cuuint64_t)d.pitch, (cuuint64_t)d.H, (cuuint64_t)np};
  const cuuint64_t strides[2] = {(cuuint64_t)d.pitch * 4, (cuuint64_t)d.plane_stride * 4};
  const cuuint32_t box[3] = {(cuuint32_t)kStageW, (cuuint32_t)kStageH, np};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapDataType dt = f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT32;
  auto encode = [&](CUtensorMap* m, const cuuint32_t* bx) {
    return enc(m, dt, 3, d.base, dims, strides, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  };
  if (encode(&d.maps.planes, box) != CUDA_SUCCESS) {
    *why = "cuTensorMapEncodeTiled failed for the state planes";
    return false;
  }
  d.stage_ok = true;
  if (d.H < 20) return true;
  // blend windows: binary32 12 beta + 3 z planes; 16-bit formats 6 beta + 2 z word planes
  const cuuint32_t nb = f32 ? 12 : 6, nz = f32 ? 3 : 2;
  if (f32) {
    const cuuint32_t bb16[3] = {(cuuint32_t)kBlendBoxW, 20, nb}, bz16[3] = {(cuuint32_t)kBlendBoxW, 20, nz};
    const cuuint32_t bb8[3] = {(cuuint32_t)kBlendBoxW, 12, nb}, bz8[3] = {(cuuint32_t)kBlendBoxW, 12, nz};
    CUtensorMap* m[4] = {&d.bmaps.beta16, &d.bmaps.z16, &d.bmaps.beta8, &d.bmaps.z8};
    const cuuint32_t* bx[4] = {bb16, bz16, bb8, bz8};
    for (int i = 0; i < 4; ++i)
      if (encode(m[i], bx[i]) != CUDA_SUCCESS) { *why = "cuTensorMapEncodeTiled failed for a blend window"; return false; }
    d.blend_tma_ok = true;
  }
  if (d.pitch >= kBlendBoxW2) {
    const cuuint32_t wb16[3] = {(cuuint32_t)kBlendBoxW2, 20, nb}, wz16[3] = {(cuuint32_t)kBlendBoxW2, 20, nz};
    const cuuint32_t wb8[3] = {(cuuint32_t)kBlendBoxW2, 12, nb}, wz8[3] = {(cuuint32_t)kBlendBoxW2, 12, nz};
    CUtensorMap* m2[4] = {&d.bmaps.beta16w, &d.bmaps.z16w, &d.bmaps.beta8w, &d.bmaps.z8w};
    const cuuint32_t* bx2[4] = {wb16, wz16, wb8, wz8};
    for (int i = 0; i < 4; ++i)
      if (encode(m2[i], bx2[i]) != CUDA_SUCCESS) {
        *why = "cuTensorMapEncodeTiled failed for a two-wide blend window";
        return false;
      }
    d.blend_tma2_ok = true;
  }
  return true;
}

bool make_kparams(const wrls_params& p, KParams* kp, const char** why) {
  if (p.struct_size != sizeof(wrls_params)) { *why = "params.struct_size != sizeof(wrls_params)"; return false; }
  if (!(p.lambda > 0.0f && p.lambda <= 1.0f)) { *why = "lambda must be in (0, 1]"; return false; }
  if (!(p.h > 0.0f) || !(p.alpha >= 0.0f && p.alpha <= 1.0f) || !(p.eps > 0.0f) ||
      !(p.p0_delta > 0.0f) || !(p.sigma_s > 0.0f) || !(p.h_s > 0.0f) || !(p.p_trace_max >= 0.0f)) {
    *why = "h, eps, p0_delta, sigma_s, h_s must be > 0, alpha in [0,1], p_trace_max >= 0";
    return false;
  }
  if (p.radius < 0 || p.radius > kMaxRadius) { *why = "radius must be in [0, 2]"; return false; }
  if ((unsigned)p.weight_mode > 2u || (unsigned)p.clamp_mode > 1u || (unsigned)p.blend_mode > 1u ||
      (unsigned)p.feature_mode > 1u || (unsigned)p.init_mode > 1u || (unsigned)p.state_precision > 2u ||
      p.n_features < 0 || (unsigned)p.reproj_filter > 1u) {
    *why = "a mode field is out of range";
    return false;
  }
  if (p.n_gbuf < 0 || p.n_gbuf > 4 || p.n_gbuf > p.n_features) {
    *why = "n_gbuf must be in [0, 4] and at most n_features";
    return false;
  }
  if (uses_ext(p) && p.state_precision != WRLS_STATE_F32) {
    *why = "G-buffer predictor entries, weight_mode 2 and reproj_filter 1 need the binary32 state";
    return false;
  }
  const double log2e = 1.4426950408889634;
  kp->lambda = p.lambda;
  kp->inv_lambda = (float)(1.0 / (double)p.lambda);
  kp->alpha = p.alpha;
  kp->one_m_alpha = (float)(1.0 - (double)p.alpha);
  kp->eps = p.eps;
  kp->w_k = (float)(log2e / ((double)p.h * (double)p.h));
  kp->p0_delta = p.p0_delta;
  kp->p_trace_max = p.p_trace_max;
  kp->range_k = (float)(log2e / ((double)p.h_s * (double)p.h_s));
  // Offsets beyond the window radius get -inf: their blend weight is exactly 0.
  for (int dy = -kMaxRadius; dy <= kMaxRadius; ++dy)
    for (int dx = -kMaxRadius; dx <= kMaxRadius; ++dx)
      kp->spatial[(dy + kMaxRadius) * (2 * kMaxRadius + 1) + dx + kMaxRadius] =
          (abs(dx) > p.radius || abs(dy) > p.radius)
              ? -INFINITY
              : (float)(-(double)(dx * dx + dy * dy) / (2.0 * (double)p.sigma_s * (double)p.sigma_s) * log2e);
  kp->radius = p.radius;
  kp->weight_mode = p.weight_mode;
  kp->clamp_mode = p.clamp_mode;
  kp->blend_mode = p.blend_mode;
  kp->feature_mode = p.feature_mode;
  kp->init_mode = p.init_mode;
  kp->debug_withhold_copy = 0;
  kp->blend_ctas_cap = 0;
  return true;
}

}  // namespace wrls

using namespace wrls;


static bool aligned4(const void* p) { return ((uintptr_t)p & 3u) == 0; }

static bool dims_ok(int w, int h) { return w >= 1 && h >= 1 && w <= 16384 && h <= 16384; }

// Add the durations of the recorded frames to the totals and clear the record.
static wrls_status fold_timing(wrls_stream* s) {
  for (int i = 0; i < s->t_pending; ++i) {
    cudaEvent_t* ev = s->tev + 4 * i;
    float a = 0.0f, b = 0.0f;
    WRLS_CHECK_CUDA(cudaEventSynchronize(ev[1]), "kernel timing: event synchronize");
    WRLS_CHECK_CUDA(cudaEventSynchronize(ev[3]), "kernel timing: event synchronize");
    WRLS_CHECK_CUDA(cudaEventElapsedTime(&a, ev[0], ev[1]), "kernel timing: elapsed time");
    WRLS_CHECK_CUDA(cudaEventElapsedTime(&b, ev[2], ev[3]), "kernel timing: elapsed time");
    s->t_update_ms += a;
    s->t_blend_ms += b;
    s->t_frames++;
  }
  s->t_pending = 0;
  return WRLS_OK;
}

static void free_timing(wrls_stream* s) {
  if (!s->tev) return;
  for (int i = 0; i < 4 * wrls_stream::kTimingCap; ++i)
    if (s->tev[i]) cudaEventDestroy(s->tev[i]);
  delete[] s->tev;
  s->tev = nullptr;
  s->t_pending = 0;
}

static bool overlaps(const void* a, size_t a_floats, const void* b, size_t b_floats) {
  if (!a || !b) return false;
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x < y + b_floats * 4 && y < x + a_floats * 4;
}

// Argument checks of one frame (per-frame and sequence entries).
static wrls_status check_frame(const wrls_stream* s, const float* radiance, const float* variance,
                               const float* features, const float* motion, const float* out, const char* who) {
  if (!radiance || !motion || !out) {
    set_error("%s: radiance, motion and out must be non-NULL", who);
    return WRLS_ERR_INVALID_ARG;
  }
  if (!aligned4(radiance) || !aligned4(motion) || !aligned4(out)) {
    set_error("%s: buffers must be 4-byte aligned", who);
    return WRLS_ERR_INVALID_ARG;
  }
  const size_t n = (size_t)s->W * s->H;
  if (overlaps(out, 3 * n, radiance, 3 * n) || overlaps(out, 3 * n, motion, 2 * n)) {
    set_error("%s: out overlaps an input", who);
    return WRLS_ERR_INVALID_ARG;
  }
  if (s->ext) {
    const bool need_var = s->prm.weight_mode == 2, need_g = s->prm.n_gbuf > 0;
    if ((need_var && (!variance || !aligned4(variance))) || (need_g && (!features || !aligned4(features)))) {
      set_error("%s: weight_mode 2 needs the variance plane and n_gbuf > 0 the feature planes "
                "(4-byte aligned device pointers)", who);
      return WRLS_ERR_INVALID_ARG;
    }
    if ((need_var && overlaps(out, 3 * n, variance, n)) ||
        (need_g && overlaps(out, 3 * n, features, (size_t)s->prm.n_gbuf * n))) {
      set_error("%s: out overlaps an input", who);
      return WRLS_ERR_INVALID_ARG;
    }
  }
  return WRLS_OK;
}

// The timing events of the next frame (NULL when timing is off).
static wrls_status timing_slot(wrls_stream* s, cudaEvent_t** ev) {
  *ev = nullptr;
  if (!s->tev) return WRLS_OK;
  if (s->t_pending == wrls_stream::kTimingCap) {
    wrls_status st = fold_timing(s);
    if (st != WRLS_OK) return st;
  }
  *ev = s->tev + 4 * s->t_pending;
  return WRLS_OK;
}

// Update of the next frame (state copy cur -> next_copy) on the stream's CUDA stream.
static wrls_status enqueue_update(wrls_stream* s, const float* radiance, const float* variance,
                                  const float* features, const float* motion, const char* who) {
  const StateDesc& prev = s->state[s->cur];
  const StateDesc& next = s->state[next_copy(s)];
  cudaError_t e;
  if (s->ext)
    e = launch_ext_update(s->ep, s->dim, prev, next, s->need_reset, radiance, motion,
                          s->prm.weight_mode == 2 ? variance : nullptr, s->prm.n_gbuf > 0 ? features : nullptr,
                          s->cs);
  else
    e = launch_update(s->kp, prev, next, s->need_reset, radiance, motion, s->err, s->cs);
  if (e != cudaSuccess) {
    set_error("%s: update kernel launch: %s", who, cudaGetErrorString(e));
    return WRLS_ERR_CUDA;
  }
  return WRLS_OK;
}

// Blend of the state copy the last update wrote (next_copy) into out, on CUDA stream cs.
static wrls_status enqueue_blend(wrls_stream* s, const KParams& kp, const float* features, float* out,
                                 cudaStream_t cs, const char* who) {
  const StateDesc& next = s->state[next_copy(s)];
  cudaError_t e;
  if (s->ext) {
    ExtParams ep = s->ep;
    ep.kp = kp;
    e = launch_ext_blend(ep, s->dim, next, s->prm.n_gbuf > 0 ? features : nullptr, out, cs);
  } else {
    e = launch_blend(kp, s->blend_cfg, next, out, s->err, cs);
  }
  if (e != cudaSuccess) {
    set_error("%s: blend kernel launch: %s", who, cudaGetErrorString(e));
    return WRLS_ERR_CUDA;
  }
  return WRLS_OK;
}

// A third state copy for wrls_denoise_sequence (same geometry as the other two); false if
// the allocation or the tensor-map encoding fails, and the stream keeps two copies.
static bool add_third_copy(wrls_stream* s) {
  int pitch;
  size_t ps;
  const int nplanes = s->state[0].nplanes;
  const size_t copy = state_copy_layout(s->W, s->H, s->prm.state_precision, &pitch, &ps, nplanes);
  void* mem = nullptr;
  if (cudaMalloc(&mem, copy) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  StateDesc d = s->state[0];
  d.base = mem;
  const char* why = "";
  if (!s->ext && !encode_stage_maps(d, &why)) {
    cudaFree(mem);
    return false;
  }
  s->state[2] = d;
  s->mem3 = mem;
  s->ncopies = 3;
  return true;
}

static void advance(wrls_stream* s) {
  s->cur = next_copy(s);
  s->need_reset = false;
  s->has_frame = true;
  s->frames++;
}

extern "C" {

void wrls_params_default(wrls_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->struct_size = sizeof(wrls_params);
  p->lambda = 0.998f;   // Sec. 5.2
  p->h = 0.75f;         // Sec. 5.3
  p->alpha = 0.75f;     // Sec. 6
  p->eps = 1e-4f;
  p->p0_delta = 1.0f;
  p->sigma_s = 1.0f;
  p->h_s = 0.75f;
  p->p_trace_max = 0.0f;
  p->radius = 2;        // 5x5, Sec. 5.3
  p->weight_mode = 0;
  p->clamp_mode = 0;
  p->blend_mode = 0;
  p->feature_mode = 0;
  p->init_mode = 0;
  p->state_precision = WRLS_STATE_F32;
  p->n_features = 0;
  p->n_gbuf = 0;
  p->reproj_filter = 0;
}

size_t wrls_state_bytes(int width, int height, const wrls_params* p) {
  if (!p || !dims_ok(width, height) || (unsigned)p->state_precision > 2u) return 0;
  if (p->struct_size != sizeof(wrls_params)) return 0;
  const int np = uses_ext(*p) ? ext_planes(ext_dim(*p)) : kNState;
  return 2 * state_copy_layout(width, height, p->state_precision, nullptr, nullptr, np);
}

const char* wrls_last_error(void) { return g_err; }

wrls_status wrls_stream_create(int width, int height, const wrls_params* p, wrls_stream** out) {
  if (!out) { set_error("wrls_stream_create: out is NULL"); return WRLS_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!p) { set_error("wrls_stream_create: params is NULL"); return WRLS_ERR_INVALID_ARG; }
  if (!dims_ok(width, height)) {
    set_error("wrls_stream_create: width/height %d x %d outside [1, 16384]", width, height);
    return WRLS_ERR_INVALID_ARG;
  }
  KParams kp;
  const char* why = "";
  if (!make_kparams(*p, &kp, &why)) { set_error("wrls_stream_create: %s", why); return WRLS_ERR_INVALID_ARG; }
  int pitch;
  size_t ps;
  const bool ext = uses_ext(*p);
  const int dim = ext ? ext_dim(*p) : 4;
  const int nplanes = ext ? ext_planes(dim) : kNState;
  const size_t copy = state_copy_layout(width, height, p->state_precision, &pitch, &ps, nplanes);
  wrls_stream* s = new (std::nothrow) wrls_stream();
  if (!s) { set_error("wrls_stream_create: host allocation failed"); return WRLS_ERR_OOM; }
  s->W = width;
  s->H = height;
  s->prm = *p;
  s->kp = kp;
  s->ext = ext;
  s->dim = dim;
  s->ep.kp = kp;
  s->ep.n_gbuf = p->n_gbuf;
  s->ep.reproj_filter = p->reproj_filter;
  s->ep.wv_k = (float)(3.0 * 1.4426950408889634 / ((double)p->h * (double)p->h));
  cudaGetDevice(&s->device);
  // both state copies, then the device error word
  const size_t scratch = 256;
  cudaError_t e = cudaMalloc(&s->mem, 2 * copy + scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("wrls_stream_create: cudaMalloc(%zu) failed: %s", 2 * copy + scratch, cudaGetErrorString(e));
    delete s;
    return e == cudaErrorMemoryAllocation ? WRLS_ERR_OOM : WRLS_ERR_CUDA;
  }
  s->mem_bytes = 2 * copy + scratch;
  s->err = (int*)((char*)s->mem + 2 * copy);
  e = cudaMemset(s->err, 0, scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(s->mem);
    set_error("wrls_stream_create: cudaMemset failed: %s", cudaGetErrorString(e));
    delete s;
    return WRLS_ERR_CUDA;
  }
  for (int i = 0; i < 2; ++i) {
    StateDesc& d = s->state[i];
    d.base = (char*)s->mem + i * copy;
    d.precision = p->state_precision;
    d.W = width;
    d.H = height;
    d.pitch = pitch;
    d.plane_stride = ps;
    d.nplanes = nplanes;
    if (!ext && !encode_stage_maps(d, &why)) {
      cudaFree(s->mem);
      set_error("wrls_stream_create: %s", why);
      delete s;
      return WRLS_ERR_CUDA;
    }
  }
  // Default blend configuration, from the measured ranking: on images of at least 2^19 pixels
  // the two-wide packed blend, 64 x 8 tiles (9) for the binary32 state, 64 x 16 tiles (8) for
  // the 16-bit formats (some 1000 tiles, several per SM); on smaller images the
  // one-CTA-per-tile 16 x 2 blend (2), where one tile per CTA spreads the work over more SMs.
  if (!ext) {
    const bool big = (long long)width * height >= (1ll << 19);
    s->blend_cfg = (big && s->state[0].blend_tma2_ok) ? (p->state_precision == 0 ? 9 : 8) : 2;
  }
  *out = s;
  return WRLS_OK;
}

wrls_status wrls_stream_set_cuda_stream(wrls_stream* s, void* cuda_stream) {
  if (!s) { set_error("wrls_stream_set_cuda_stream: stream is NULL"); return WRLS_ERR_INVALID_ARG; }
  s->cs = (cudaStream_t)cuda_stream;
  return WRLS_OK;
}

wrls_status wrls_denoise_frame(wrls_stream* s, const float* radiance, const float* variance,
                               const float* features, const float* motion, float* out) {
  NvtxRange nvtx("wrls_denoise_frame");
  if (!s) { set_error("wrls_denoise_frame: stream is NULL"); return WRLS_ERR_INVALID_ARG; }
  wrls_status st = check_frame(s, radiance, variance, features, motion, out, "wrls_denoise_frame");
  if (st != WRLS_OK) return st;
  cudaEvent_t* ev = nullptr;
  st = timing_slot(s, &ev);
  if (st != WRLS_OK) return st;
  if (ev) WRLS_CHECK_CUDA(cudaEventRecord(ev[0], s->cs), "wrls_denoise_frame: event record");
  st = enqueue_update(s, radiance, variance, features, motion, "wrls_denoise_frame");
  if (st != WRLS_OK) return st;
  if (ev) {
    WRLS_CHECK_CUDA(cudaEventRecord(ev[1], s->cs), "wrls_denoise_frame: event record");
    WRLS_CHECK_CUDA(cudaEventRecord(ev[2], s->cs), "wrls_denoise_frame: event record");
  }
  st = enqueue_blend(s, s->kp, features, out, s->cs, "wrls_denoise_frame");
  if (st != WRLS_OK) return st;
  if (ev) {
    WRLS_CHECK_CUDA(cudaEventRecord(ev[3], s->cs), "wrls_denoise_frame: event record");
    s->t_pending++;
  }
  advance(s);
  return WRLS_OK;
}

static wrls_status sequence_setup(wrls_stream* s, const char* who);

wrls_status wrls_denoise_sequence(wrls_stream* s, const wrls_frame_io* frames, int n) {
  NvtxRange nvtx("wrls_denoise_sequence");
  if (!s || !frames || n < 1) {
    set_error("wrls_denoise_sequence: NULL stream or frames, or n < 1");
    return WRLS_ERR_INVALID_ARG;
  }
  const size_t np = (size_t)s->W * s->H;
  for (int i = 0; i < n; ++i) {
    const wrls_frame_io& f = frames[i];
    if (f.stream && f.stream != s) {
      set_error("wrls_denoise_sequence: frame %d names another stream", i);
      return WRLS_ERR_INVALID_ARG;
    }
    wrls_status st = check_frame(s, f.radiance, f.variance, f.features, f.motion, f.out, "wrls_denoise_sequence");
    if (st != WRLS_OK) return st;
    if (i + 1 < n) {  // the blend of frame i runs while the update of frame i+1 reads its inputs
      const wrls_frame_io& g = frames[i + 1];
      const bool need_var = s->ext && s->prm.weight_mode == 2, need_g = s->ext && s->prm.n_gbuf > 0;
      if (overlaps(f.out, 3 * np, g.radiance, 3 * np) || overlaps(f.out, 3 * np, g.motion, 2 * np) ||
          (need_var && overlaps(f.out, 3 * np, g.variance, np)) ||
          (need_g && overlaps(f.out, 3 * np, g.features, (size_t)s->prm.n_gbuf * np)) ||
          overlaps(f.out, 3 * np, g.out, 3 * np)) {
        set_error("wrls_denoise_sequence: the output of frame %d overlaps a buffer of frame %d", i, i + 1);
        return WRLS_ERR_INVALID_ARG;
      }
    }
  }
  if (n == 1) {
    for (int i = 0; i < n; ++i) {
      const wrls_frame_io& f = frames[i];
      wrls_status st = wrls_denoise_frame(s, f.radiance, f.variance, f.features, f.motion, f.out);
      if (st != WRLS_OK) return st;
    }
    return WRLS_OK;
  }
  // first use: side stream, events, and a third state copy, which lets the update of frame
  // t+2 run while the blend of frame t still reads its copy (without it, when the
  // allocation fails, that update waits for that blend)
  {
    wrls_status st0 = sequence_setup(s, "wrls_denoise_sequence");
    if (st0 != WRLS_OK) return st0;
  }
  KParams kpo = s->kp;
  kpo.blend_ctas_cap = s->overlap_ctas;
  wrls_status st = WRLS_OK;
  auto ck = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == WRLS_OK) {
      set_error("wrls_denoise_sequence: %s: %s", what, cudaGetErrorString(e));
      st = WRLS_ERR_CUDA;
    }
    return st == WRLS_OK;
  };
  int last = -1;  // last frame whose blend was enqueued on the side stream
  for (int i = 0; i < n && st == WRLS_OK; ++i) {
    const wrls_frame_io& f = frames[i];
    // The update of frame i overwrites the state copy that the blend of frame i - ncopies reads.
    const int nc = s->ncopies;
    if (i >= nc && !ck(cudaStreamWaitEvent(s->cs, s->ev_b[(i - nc) % 3], 0), "wait")) break;
    cudaEvent_t* ev = nullptr;
    if ((st = timing_slot(s, &ev)) != WRLS_OK) break;
    if (ev && !ck(cudaEventRecord(ev[0], s->cs), "event record")) break;
    if ((st = enqueue_update(s, f.radiance, f.variance, f.features, f.motion, "wrls_denoise_sequence")) != WRLS_OK)
      break;
    if (ev && !ck(cudaEventRecord(ev[1], s->cs), "event record")) break;
    if (!ck(cudaEventRecord(s->ev_u, s->cs), "event record")) break;
    if (!ck(cudaStreamWaitEvent(s->side, s->ev_u, 0), "wait")) break;
    if (ev && !ck(cudaEventRecord(ev[2], s->side), "event record")) break;
    if ((st = enqueue_blend(s, kpo, f.features, f.out, s->side, "wrls_denoise_sequence")) != WRLS_OK) break;
    last = i;
    if (ev) {
      if (!ck(cudaEventRecord(ev[3], s->side), "event record")) break;
      s->t_pending++;
    }
    if (!ck(cudaEventRecord(s->ev_b[i % 3], s->side), "event record")) break;
    advance(s);
  }
  // join: later work on the stream's CUDA stream sees every output (also after an error)
  if (last >= 0) {
    cudaError_t e = cudaEventRecord(s->ev_b[last % 3], s->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->cs, s->ev_b[last % 3], 0);
    ck(e, "join");
  }
  return st;
}

// Side stream, its events and the third state copy of the sequence entries (first use).
static wrls_status sequence_setup(wrls_stream* s, const char* who) {
  if (s->side) return WRLS_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_u, cudaEventDisableTiming);
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&s->ev_b[k], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("%s: stream/event creation failed: %s", who, cudaGetErrorString(e));
    return WRLS_ERR_CUDA;
  }
  if (!s->debug_two_copies) add_third_copy(s);  // on failure the stream keeps two copies
  return WRLS_OK;
}

wrls_status wrls_denoise_sequence_host(wrls_stream* s, const wrls_frame_io* frames, int n) {
  NvtxRange nvtx("wrls_denoise_sequence_host");
  if (!s || !frames || n < 1) {
    set_error("wrls_denoise_sequence_host: NULL stream or frames, or n < 1");
    return WRLS_ERR_INVALID_ARG;
  }
  const bool need_var = s->ext && s->prm.weight_mode == 2, need_g = s->ext && s->prm.n_gbuf > 0;
  for (int i = 0; i < n; ++i) {
    const wrls_frame_io& f = frames[i];
    if ((f.stream && f.stream != s) || !f.radiance || !f.motion || !f.out || (need_var && !f.variance) ||
        (need_g && !f.features)) {
      set_error("wrls_denoise_sequence_host: frame %d names another stream or lacks a required buffer", i);
      return WRLS_ERR_INVALID_ARG;
    }
  }
  wrls_status st = sequence_setup(s, "wrls_denoise_sequence_host");
  if (st != WRLS_OK) return st;
  const size_t np = (size_t)s->W * s->H;
  const size_t slot_floats = (8 + (s->ext ? 1 + (size_t)s->prm.n_gbuf : 0)) * np;
  if (!s->ring) {
    cudaError_t e = cudaMalloc(&s->ring, wrls_stream::kHostSlots * slot_floats * sizeof(float));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->d2h, cudaStreamNonBlocking);
    for (int k = 0; k < wrls_stream::kHostSlots && e == cudaSuccess; ++k) {
      e = cudaEventCreateWithFlags(&s->ev_in[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_used[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_done[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_out[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("wrls_denoise_sequence_host: set-up failed: %s", cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? WRLS_ERR_OOM : WRLS_ERR_CUDA;
    }
    s->ring_slot = slot_floats;
    // the copy streams start behind everything already queued on the stream's CUDA stream
    WRLS_CHECK_CUDA(cudaStreamSynchronize(s->cs), "wrls_denoise_sequence_host: synchronize");
  }
  KParams kpo = s->kp;
  kpo.blend_ctas_cap = s->overlap_ctas;
  auto ck = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == WRLS_OK) {
      set_error("wrls_denoise_sequence_host: %s: %s", what, cudaGetErrorString(e));
      st = WRLS_ERR_CUDA;
    }
    return st == WRLS_OK;
  };
  // earlier work on the stream's CUDA stream comes first
  ck(cudaEventRecord(s->ev_u, s->cs), "event record");
  ck(cudaStreamWaitEvent(s->h2d, s->ev_u, 0), "wait");
  const int NS = wrls_stream::kHostSlots;
  int last = -1;
  for (int i = 0; i < n && st == WRLS_OK; ++i) {
    const wrls_frame_io& f = frames[i];
    const int k = i % NS;
    float* base = s->ring + (size_t)k * s->ring_slot;
    float *d_rad = base, *d_mot = base + 3 * np, *d_out = base + 5 * np;
    float* d_var = need_var ? base + 8 * np : nullptr;
    float* d_g = need_g ? base + 9 * np : nullptr;
    // inputs: after the kernels of frame i - NS are done with this slot
    if (i >= NS && !ck(cudaStreamWaitEvent(s->h2d, s->ev_used[k], 0), "wait")) break;
    if (!ck(cudaMemcpyAsync(d_rad, f.radiance, 3 * np * 4, cudaMemcpyHostToDevice, s->h2d), "radiance copy")) break;
    if (!ck(cudaMemcpyAsync(d_mot, f.motion, 2 * np * 4, cudaMemcpyHostToDevice, s->h2d), "motion copy")) break;
    if (d_var && !ck(cudaMemcpyAsync(d_var, f.variance, np * 4, cudaMemcpyHostToDevice, s->h2d), "variance copy"))
      break;
    if (d_g && !ck(cudaMemcpyAsync(d_g, f.features, (size_t)s->prm.n_gbuf * np * 4, cudaMemcpyHostToDevice, s->h2d),
                   "feature copy"))
      break;
    if (!ck(cudaEventRecord(s->ev_in[k], s->h2d), "event record")) break;
    // update on the stream's CUDA stream (after its inputs, and after the blend that last
    // read the state copy it overwrites)
    const int nc = s->ncopies;
    if (i >= nc && !ck(cudaStreamWaitEvent(s->cs, s->ev_b[(i - nc) % 3], 0), "wait")) break;
    if (!ck(cudaStreamWaitEvent(s->cs, s->ev_in[k], 0), "wait")) break;
    if ((st = enqueue_update(s, d_rad, d_var, d_g, d_mot, "wrls_denoise_sequence_host")) != WRLS_OK) break;
    if (!ck(cudaEventRecord(s->ev_u, s->cs), "event record")) break;
    // blend on the side stream (after the update, and after the output copy of frame i - NS)
    if (!ck(cudaStreamWaitEvent(s->side, s->ev_u, 0), "wait")) break;
    if (i >= NS && !ck(cudaStreamWaitEvent(s->side, s->ev_out[k], 0), "wait")) break;
    if ((st = enqueue_blend(s, kpo, d_g, d_out, s->side, "wrls_denoise_sequence_host")) != WRLS_OK) break;
    last = i;
    if (!ck(cudaEventRecord(s->ev_b[i % 3], s->side), "event record")) break;
    // the slot's inputs are free once the update (and, with G-buffer entries, the blend) ran
    if (!ck(cudaEventRecord(s->ev_used[k], need_g ? s->side : s->cs), "event record")) break;
    if (!ck(cudaEventRecord(s->ev_done[k], s->side), "event record")) break;
    if (!ck(cudaStreamWaitEvent(s->d2h, s->ev_done[k], 0), "wait")) break;
    if (!ck(cudaMemcpyAsync(f.out, d_out, 3 * np * 4, cudaMemcpyDeviceToHost, s->d2h), "output copy")) break;
    if (!ck(cudaEventRecord(s->ev_out[k], s->d2h), "event record")) break;
    advance(s);
  }
  // join: the stream's CUDA stream waits for the last output copy (the copy stream is in
  // order, so for all of them) and for the last blend
  if (last >= 0) {
    cudaError_t e = cudaEventRecord(s->ev_out[last % NS], s->d2h);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->cs, s->ev_out[last % NS], 0);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev_b[last % 3], s->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->cs, s->ev_b[last % 3], 0);
    ck(e, "join");
  }
  return st;
}

wrls_status wrls_stream_set_overlap(wrls_stream* s, int blend_ctas_per_sm) {
  if (!s || blend_ctas_per_sm < 0 || blend_ctas_per_sm > 32) {
    set_error("wrls_stream_set_overlap: bad stream or value %d (0..32)", blend_ctas_per_sm);
    return WRLS_ERR_INVALID_ARG;
  }
  s->overlap_ctas = blend_ctas_per_sm;
  return WRLS_OK;
}

wrls_status wrls_denoise_frame_host(wrls_stream* s, const float* radiance, const float* variance,
                                    const float* features, const float* motion, float* out) {
  NvtxRange nvtx("wrls_denoise_frame_host");
  if (!s || !radiance || !motion || !out) {
    set_error("wrls_denoise_frame_host: stream, radiance, motion and out must be non-NULL");
    return WRLS_ERR_INVALID_ARG;
  }
  const bool need_var = s->prm.weight_mode == 2, need_g = s->prm.n_gbuf > 0;
  if ((need_var && !variance) || (need_g && !features)) {
    set_error("wrls_denoise_frame_host: weight_mode 2 needs the variance plane and n_gbuf > 0 the feature planes");
    return WRLS_ERR_INVALID_ARG;
  }
  const size_t n = (size_t)s->W * s->H;
  // radiance 3, motion 2, output 3 planes, then the variance plane and the predictor's
  // G-buffer planes of the extended path
  const size_t extra = (size_t)(s->ext ? 1 + s->prm.n_gbuf : 0);
  if (!s->staging) {
    cudaError_t e = cudaMalloc(&s->staging, (8 + extra) * n * sizeof(float));
    if (e != cudaSuccess) {
      cudaGetLastError();
      s->staging = nullptr;
      set_error("wrls_denoise_frame_host: staging cudaMalloc failed: %s", cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? WRLS_ERR_OOM : WRLS_ERR_CUDA;
    }
  }
  float* d_rad = s->staging;
  float* d_mot = s->staging + 3 * n;
  float* d_out = s->staging + 5 * n;
  float* d_var = need_var ? s->staging + 8 * n : nullptr;
  float* d_g = need_g ? s->staging + 9 * n : nullptr;
  WRLS_CHECK_CUDA(cudaMemcpyAsync(d_rad, radiance, 3 * n * sizeof(float), cudaMemcpyHostToDevice, s->cs),
                  "wrls_denoise_frame_host: radiance copy");
  WRLS_CHECK_CUDA(cudaMemcpyAsync(d_mot, motion, 2 * n * sizeof(float), cudaMemcpyHostToDevice, s->cs),
                  "wrls_denoise_frame_host: motion copy");
  if (d_var)
    WRLS_CHECK_CUDA(cudaMemcpyAsync(d_var, variance, n * sizeof(float), cudaMemcpyHostToDevice, s->cs),
                    "wrls_denoise_frame_host: variance copy");
  if (d_g)
    WRLS_CHECK_CUDA(cudaMemcpyAsync(d_g, features, (size_t)s->prm.n_gbuf * n * sizeof(float),
                                    cudaMemcpyHostToDevice, s->cs),
                    "wrls_denoise_frame_host: feature copy");
  wrls_status st = wrls_denoise_frame(s, d_rad, d_var, d_g, d_mot, d_out);
  if (st != WRLS_OK) return st;
  WRLS_CHECK_CUDA(cudaMemcpyAsync(out, d_out, 3 * n * sizeof(float), cudaMemcpyDeviceToHost, s->cs),
                  "wrls_denoise_frame_host: output copy");
  return WRLS_OK;
}

wrls_status wrls_stream_reset(wrls_stream* s) {
  if (!s) { set_error("wrls_stream_reset: stream is NULL"); return WRLS_ERR_INVALID_ARG; }
  s->need_reset = true;
  return WRLS_OK;
}

void wrls_stream_destroy(wrls_stream* s) {
  if (!s) return;
  int prev_dev = 0;
  cudaGetDevice(&prev_dev);
  if (prev_dev != s->device) cudaSetDevice(s->device);
  cudaStreamSynchronize(s->cs);
  if (s->side) cudaStreamSynchronize(s->side);
  free_timing(s);
  if (s->ev_u) cudaEventDestroy(s->ev_u);
  for (int i = 0; i < 3; ++i)
    if (s->ev_b[i]) cudaEventDestroy(s->ev_b[i]);
  if (s->side) cudaStreamDestroy(s->side);
  if (s->h2d) cudaStreamSynchronize(s->h2d);
  if (s->d2h) cudaStreamSynchronize(s->d2h);
  for (int k = 0; k < wrls_stream::kHostSlots; ++k) {
    if (s->ev_in[k]) cudaEventDestroy(s->ev_in[k]);
    if (s->ev_used[k]) cudaEventDestroy(s->ev_used[k]);
    if (s->ev_done[k]) cudaEventDestroy(s->ev_done[k]);
    if (s->ev_out[k]) cudaEventDestroy(s->ev_out[k]);
  }
  if (s->h2d) cudaStreamDestroy(s->h2d);
  if (s->d2h) cudaStreamDestroy(s->d2h);
  if (s->ring) cudaFree(s->ring);
  cudaFree(s->mem);
  if (s->mem3) cudaFree(s->mem3);
  if (s->staging) cudaFree(s->staging);
  if (s->stats) cudaFree(s->stats);
  cudaGetLastError();
  if (prev_dev != s->device) cudaSetDevice(prev_dev);
  delete s;
}

wrls_status wrls_stream_read_state(wrls_stream* s, float* dst) {
  NvtxRange nvtx("wrls_stream_read_state");
  if (!s || !dst) { set_error("wrls_stream_read_state: NULL argument"); return WRLS_ERR_INVALID_ARG; }
  if (!aligned4(dst)) { set_error("wrls_stream_read_state: dst must be 4-byte aligned"); return WRLS_ERR_INVALID_ARG; }
  if (!s->has_frame) { set_error("wrls_stream_read_state: no frame denoised yet"); return WRLS_ERR_STATE; }
  if (s->ext)
    WRLS_CHECK_CUDA(launch_read_state_ext(s->state[s->cur], s->state[s->cur].nplanes, dst, s->cs),
                    "wrls_stream_read_state: launch");
  else
    WRLS_CHECK_CUDA(launch_read_state(s->state[s->cur], dst, s->cs), "wrls_stream_read_state: launch");
  return WRLS_OK;
}

wrls_status wrls_stream_write_state(wrls_stream* s, const float* src) {
  NvtxRange nvtx("wrls_stream_write_state");
  if (!s || !src) { set_error("wrls_stream_write_state: NULL argument"); return WRLS_ERR_INVALID_ARG; }
  if (!aligned4(src)) { set_error("wrls_stream_write_state: src must be 4-byte aligned"); return WRLS_ERR_INVALID_ARG; }
  if (s->ext)
    WRLS_CHECK_CUDA(launch_write_state_ext(s->state[s->cur], s->state[s->cur].nplanes, src, s->cs),
                    "wrls_stream_write_state: launch");
  else
    WRLS_CHECK_CUDA(launch_write_state(s->state[s->cur], src, s->cs), "wrls_stream_write_state: launch");
  s->has_frame = true;
  s->need_reset = false;
  return WRLS_OK;
}

uint64_t wrls_stream_frames(const wrls_stream* s) { return s ? s->frames : 0; }

wrls_status wrls_stream_set_blend_config(wrls_stream* s, int config) {
  if (!s || !blend_config_ok(config, s->prm.state_precision, s->state[0].blend_tma_ok, s->state[0].blend_tma2_ok) ||
      (s->ext && config != 0)) {
    set_error("wrls_stream_set_blend_config: bad stream or configuration %d for this state format", config);
    return WRLS_ERR_INVALID_ARG;
  }
  s->blend_cfg = config;
  return WRLS_OK;
}

wrls_status wrls_stream_autotune(wrls_stream* s, float* out, int reps, float* times_ms, int* chosen) {
  NvtxRange nvtx("wrls_stream_autotune");
  if (!s || !out || reps < 1) { set_error("wrls_stream_autotune: bad argument"); return WRLS_ERR_INVALID_ARG; }
  if (!s->has_frame) { set_error("wrls_stream_autotune: no frame denoised yet"); return WRLS_ERR_STATE; }
  if (s->ext) {  // one blend configuration on the extended path
    if (times_ms)
      for (int c = 0; c < kBlendConfigs; ++c) times_ms[c] = -1.0f;
    if (chosen) *chosen = 0;
    return WRLS_OK;
  }
  const StateDesc& cur = s->state[s->cur];
  cudaEvent_t e0, e1;
  WRLS_CHECK_CUDA(cudaEventCreate(&e0), "wrls_stream_autotune: event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    set_error("wrls_stream_autotune: event");
    return WRLS_ERR_CUDA;
  }
  int best = 0;
  float best_ms = 0.0f;
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < kBlendConfigs && e == cudaSuccess; ++c) {
    if (!blend_config_ok(c, cur.precision, cur.blend_tma_ok, cur.blend_tma2_ok)) {
      if (times_ms) times_ms[c] = -1.0f;
      continue;
    }
    e = launch_blend(s->kp, c, cur, out, s->err, s->cs);  // warm-up (and first-use setup)
    if (e == cudaSuccess) e = cudaEventRecord(e0, s->cs);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_blend(s->kp, c, cur, out, s->err, s->cs);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s->cs);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    ms /= (float)reps;
    if (times_ms) times_ms[c] = ms;
    if (c == 0 || ms < best_ms) { best = c; best_ms = ms; }
  }
  if (e == cudaSuccess) e = launch_blend(s->kp, best, cur, out, s->err, s->cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->cs);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) { set_error("wrls_stream_autotune: %s", cudaGetErrorString(e)); return WRLS_ERR_CUDA; }
  s->blend_cfg = best;
  if (chosen) *chosen = best;
  return WRLS_OK;
}

wrls_status wrls_stream_set_debug(wrls_stream* s, uint32_t flags) {
  if (!s || (flags & ~(WRLS_DEBUG_WITHHOLD_STAGE_COPY | WRLS_DEBUG_NO_THIRD_COPY))) {
    set_error("wrls_stream_set_debug: bad stream or unknown flags 0x%x", flags);
    return WRLS_ERR_INVALID_ARG;
  }
  s->kp.debug_withhold_copy = (flags & WRLS_DEBUG_WITHHOLD_STAGE_COPY) ? 1 : 0;
  s->debug_two_copies = (flags & WRLS_DEBUG_NO_THIRD_COPY) != 0;
  return WRLS_OK;
}

wrls_status wrls_stream_check(wrls_stream* s) {
  if (!s) { set_error("wrls_stream_check: stream is NULL"); return WRLS_ERR_INVALID_ARG; }
  WRLS_CHECK_CUDA(cudaStreamSynchronize(s->cs), "wrls_stream_check: synchronize");
  int flag = 0;
  WRLS_CHECK_CUDA(cudaMemcpy(&flag, s->err, sizeof(int), cudaMemcpyDeviceToHost), "wrls_stream_check: read");
  if (flag != 0) {
    WRLS_CHECK_CUDA(cudaMemset(s->err, 0, sizeof(int)), "wrls_stream_check: clear");
    set_error("wrls_stream_check: a bounded device-side wait gave up (status %d)", flag);
    return (wrls_status)flag;
  }
  return WRLS_OK;
}

wrls_status wrls_stream_enable_timing(wrls_stream* s, int enable) {
  if (!s) { set_error("wrls_stream_enable_timing: stream is NULL"); return WRLS_ERR_INVALID_ARG; }
  if (!enable) {
    cudaStreamSynchronize(s->cs);
    free_timing(s);
    return WRLS_OK;
  }
  if (s->tev) return WRLS_OK;
  s->tev = new (std::nothrow) cudaEvent_t[4 * wrls_stream::kTimingCap]();
  if (!s->tev) { set_error("wrls_stream_enable_timing: host allocation failed"); return WRLS_ERR_OOM; }
  for (int i = 0; i < 4 * wrls_stream::kTimingCap; ++i) {
    cudaError_t e = cudaEventCreate(&s->tev[i]);
    if (e != cudaSuccess) {
      free_timing(s);
      set_error("wrls_stream_enable_timing: cudaEventCreate: %s", cudaGetErrorString(e));
      return WRLS_ERR_CUDA;
    }
  }
  s->t_update_ms = s->t_blend_ms = 0.0;
  s->t_frames = 0;
  return WRLS_OK;
}

wrls_status wrls_stream_kernel_times(wrls_stream* s, double* update_ms, double* blend_ms,
                                     uint64_t* frames) {
  if (!s || !update_ms || !blend_ms || !frames) {
    set_error("wrls_stream_kernel_times: NULL argument");
    return WRLS_ERR_INVALID_ARG;
  }
  if (!s->tev) { set_error("wrls_stream_kernel_times: timing is not enabled"); return WRLS_ERR_STATE; }
  wrls_status st = fold_timing(s);
  if (st != WRLS_OK) return st;
  *update_ms = s->t_update_ms;
  *blend_ms = s->t_blend_ms;
  *frames = s->t_frames;
  s->t_update_ms = s->t_blend_ms = 0.0;
  s->t_frames = 0;
  return WRLS_OK;
}

}  // extern "C"
