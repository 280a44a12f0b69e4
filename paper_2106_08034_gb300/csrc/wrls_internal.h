// Internal declarations shared by the CUDA translation units of libwrls.so.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/wrls.h"
#include "wrls_device.cuh"

namespace wrls {

// Geometry of one state copy in device memory. Planar: `nplanes` planes of 32-bit elements
// (binary32 values: kNState, or the extended path's count; 16-bit formats: the 13 word
// planes of packed pairs), each plane pitch x H elements padded to a multiple of 64.
struct StateDesc {
  void* base = nullptr;
  int precision = 0;
  int nplanes = kNState;
  int W = 0, H = 0, pitch = 0;
  size_t plane_stride = 0;  // in values
  StageMaps maps{};          // TMA tensor map of this copy's planes
  bool stage_ok = false;     // maps encoded and the image is at least one staging box
  BlendMaps bmaps{};         // TMA tensor maps of the blend windows
  bool blend_tma_ok = false; // 40-column blend maps encoded (binary32 state, image >= one box)
  bool blend_tma2_ok = false; // 72-column blend maps encoded

  StateF32 f32() const { return StateF32{(float*)base, plane_stride, pitch}; }
  StateBF16 bf16() const { return StateBF16{(uint32_t*)base, plane_stride, pitch}; }
  StateF16 f16() const { return StateF16{(uint32_t*)base, plane_stride, pitch}; }
};

// 32-bit planes of one state copy: `nplanes` binary32 planes, or the 13 word planes of the
// 16-bit formats.
inline int copy_planes(int precision, int nplanes) { return precision == 0 ? nplanes : StateBF16::kPlanes; }
// Bytes of one state copy and its geometry.
size_t state_copy_layout(int W, int H, int precision, int* pitch, size_t* plane_stride, int nplanes = kNState);

// ---- extended predictor and weights (wrls_ext.cu) ----
// Kernel parameters of a stream whose predictor has G-buffer entries, that weights by the
// sample variance, or that reprojects to the nearest pixel.
struct ExtParams {
  KParams kp;
  int n_gbuf;         // G-buffer entries of p
  int reproj_filter;  // 0 bilinear, 1 nearest pixel
  float wv_k;         // 3 log2(e) / h^2: exponent of the sample-variance weight in base 2
};
// True if the parameters need the extended kernels.
inline bool uses_ext(const wrls_params& p) { return p.n_gbuf > 0 || p.weight_mode == 2 || p.reproj_filter == 1; }
int ext_dim(const wrls_params& p);  // predictor dimension d
int ext_planes(int d);              // state planes of dimension d: 3d + d(d+1)/2 + 3
cudaError_t launch_ext_update(const ExtParams& ep, int d, const StateDesc& prev, const StateDesc& next, bool reset,
                              const float* rad, const float* mot, const float* var, const float* gbuf,
                              cudaStream_t cs);
cudaError_t launch_ext_blend(const ExtParams& ep, int d, const StateDesc& cur, const float* gbuf, float* out,
                             cudaStream_t cs);
cudaError_t launch_read_state_ext(const StateDesc& cur, int nplanes, float* dst, cudaStream_t cs);
cudaError_t launch_write_state_ext(const StateDesc& cur, int nplanes, const float* src, cudaStream_t cs);

// Host-side conversion of the public parameters (validated) into kernel parameters.
bool make_kparams(const wrls_params& p, KParams* kp, const char** why);

cudaError_t launch_update(const KParams& kp, const StateDesc& prev, const StateDesc& next, bool reset,
                          const float* rad, const float* mot, int* err, cudaStream_t cs);
// Encode the TMA tensor maps of a state copy (sets stage_ok; false only on a driver error).
bool encode_stage_maps(StateDesc& d, const char** why);
// Blend tile configurations (tile rows TH x output rows per thread R):
// 0: 16x4, 1: 8x4, 2: 16x2, 3: 32x4 -- one CTA per tile, synchronous fill;
// 4: 16x2, 5: 16x2, 6: 8x2, 7: 16x4 -- persistent, TMA-filled windows, double-buffered (4, 6)
// or single (5, 7) (binary32 state, images of at least 40 x 20 pixels);
// 8: 16 rows x 2 x 2, 9: 8 rows x 2 x 2 -- persistent, TMA-filled, each thread 2 columns x
// 2 rows (any state format; images of at least 72 x 20 pixels).
constexpr int kBlendConfigs = 10;
constexpr int kBlendSyncConfigs = 4;
inline bool blend_config_ok(int cfg, int precision, bool tma_ok, bool tma2_ok) {
  if (cfg < 0 || cfg >= kBlendConfigs) return false;
  if (cfg < kBlendSyncConfigs) return true;
  return cfg < 8 ? (precision == 0 && tma_ok) : tma2_ok;
}
// The synchronous configuration wrls_batch_tick_static runs in place of a persistent one (the
// same tile rows and outputs per thread; 16 x 2 for the two-wide configurations).
inline int blend_sync_config(int cfg) {
  static const int map[kBlendConfigs] = {0, 1, 2, 3, 2, 2, 1, 0, 2, 2};
  return (cfg >= 0 && cfg < kBlendConfigs) ? map[cfg] : 0;
}
cudaError_t launch_blend(const KParams& kp, int cfg, const StateDesc& cur, float* out, int* err, cudaStream_t cs);
cudaError_t launch_blend_pipelined(const KParams& kp, int cfg, const StateDesc& cur, float* out, int* err,
                                   cudaStream_t cs);
cudaError_t launch_blend_two_wide(const KParams& kp, int cfg, const StateDesc& cur, float* out, int* err,
                                  cudaStream_t cs);
cudaError_t launch_read_state(const StateDesc& cur, float* dst, cudaStream_t cs);
cudaError_t launch_write_state(const StateDesc& cur, const float* src, cudaStream_t cs);

void set_error(const char* fmt, ...);

// Return WRLS_ERR_CUDA with a message from an entry point when a CUDA call fails.
#define WRLS_CHECK_CUDA(call, what)                      \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) {                             \
      set_error("%s: %s", what, cudaGetErrorString(e_)); \
      return WRLS_ERR_CUDA;                              \
    }                                                    \
  } while (0)

// NVTX range around an entry point (visible in Nsight timelines; a no-op call when no tool is
// attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace wrls

// The stream object behind the opaque C handle.
struct wrls_stream {
  int W = 0, H = 0;
  wrls_params prm{};
  wrls::KParams kp{};
  bool ext = false;             // extended predictor / weights (wrls_ext.cu kernels)
  int dim = 4;                  // predictor dimension of the extended kernels
  wrls::ExtParams ep{};
  wrls::StateDesc state[3];     // copies in rotation: state[cur] holds frame t-1
  int ncopies = 2;              // 2; 3 once wrls_denoise_sequence has added a copy
  void* mem3 = nullptr;         // the third copy (wrls_denoise_sequence)
  void* mem = nullptr;          // both state copies, then the device error word
  int* err = nullptr;           // device error word (WRLS_ERR_TIMEOUT from a bounded wait)
  size_t mem_bytes = 0;
  int cur = 0;                  // copy holding frame t-1 (the next frame writes next_copy())
  bool need_reset = true;
  bool has_frame = false;
  cudaStream_t cs = nullptr;
  int device = 0;
  uint64_t frames = 0;
  float* staging = nullptr;     // device I/O buffers of wrls_denoise_frame_host
  void* stats = nullptr;        // wrls_stream_state_stats accumulators (allocated on first use)
  // wrls_denoise_sequence_host: a ring of device I/O slots and copy streams
  static constexpr int kHostSlots = 3;
  float* ring = nullptr;        // kHostSlots slots of (radiance, motion, output, variance, G-buffers)
  size_t ring_slot = 0;         // floats per slot
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t ev_in[kHostSlots] = {};    // slot's inputs copied
  cudaEvent_t ev_used[kHostSlots] = {};  // slot's inputs no longer read by kernels
  cudaEvent_t ev_done[kHostSlots] = {};  // slot's output written
  cudaEvent_t ev_out[kHostSlots] = {};   // slot's output copied to the host
  int blend_cfg = 0;            // blend tile configuration
  // wrls_denoise_sequence: blends on a second CUDA stream, ordered by events
  cudaStream_t side = nullptr;
  cudaEvent_t ev_u = nullptr;          // update of frame t done (side stream waits)
  cudaEvent_t ev_b[3] = {nullptr, nullptr, nullptr};  // blend of frame t done, by t % 3: the update of
                                                      // frame t + ncopies, which overwrites its copy, waits
  int overlap_ctas = 3;                // CTAs per SM of a persistent blend that overlaps an update
  bool debug_two_copies = false;       // WRLS_DEBUG_NO_THIRD_COPY: sequence entries keep two copies
  // kernel tracing
  static constexpr int kTimingCap = 8192;
  cudaEvent_t* tev = nullptr;   // 4 events per recorded frame: update start/end, blend start/end
  int t_pending = 0;
  double t_update_ms = 0.0, t_blend_ms = 0.0;
  uint64_t t_frames = 0;
};

// The state copy the next frame writes: the one after `cur` in the rotation.
inline int next_copy(const wrls_stream* s) { return s->cur + 1 < s->ncopies ? s->cur + 1 : 0; }
