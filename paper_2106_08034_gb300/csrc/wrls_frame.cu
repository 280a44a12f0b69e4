// Single-frame kernels of the wRLS denoiser, one CTA per tile:
//   k_update     : reprojection + Eq. 12 + Eq. 13 + Eq. 8/14/9/11 (tile body update_tile)
//   k_blend      : 5x5 spatio-temporal blend of Sec. 5.3 (tile body blend_tile)
//   k_read_state : decode a state copy to 25 binary32 planes
#include "wrls_internal.h"
#include "wrls_tiles.cuh"

namespace wrls {

// CTAs per SM the update is compiled for (registers a thread <= 65536 / (256 x CTAs)), measured
// at 1080p: with a 16-bit state (issue-bound, 24 KB of shared memory a CTA) 6 CTAs (40
// registers, a small spill) took 70.6 us against 74.8 us at 4 (64 registers) and 71.7 at 5; 7
// (32 registers) spilled and took 87.7. With the binary32 state (44 KB a CTA) 5 CTAs (48
// registers) took 83.1 us against 88.0 at 4.
template <class SV>
__global__ void __launch_bounds__(kTileThreads, SV::kScaled ? 6 : 5)
    k_update(const KParams kp, const int W, const int H, const int reset, const int stage_ok,
             const SV prev, const SV next, const __grid_constant__ StageMaps maps,
             const float* __restrict__ rad, const float* __restrict__ mot, int* err) {
  extern __shared__ unsigned char dsmem[];
  __shared__ alignas(8) uint64_t bar;
  UpdateSmem<SV>& sm = *reinterpret_cast<UpdateSmem<SV>*>(align128(dsmem));
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  uint32_t phase = 0;
  update_tile(sm, &bar, phase, err, kp, W, H, reset != 0, stage_ok != 0, prev, next, &maps, rad, mot,
              blockIdx.x * kTW, blockIdx.y * kTH);
}

template <class SV, int TH, int R, int MODE>
__global__ void __launch_bounds__(kTW * TH / R)
    k_blend(const KParams kp, const int W, const int H, const SV cur, float* __restrict__ out) {
  extern __shared__ float4 sm_blend[];
  blend_tile<SV, TH, R, MODE>(sm_blend, kp, W, H, cur, out, blockIdx.x * kTW, blockIdx.y * TH);
}

template <class SV>
__global__ void k_read_state(const int W, const int H, const SV cur, float* __restrict__ dst) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W || y >= H) return;
  float v[kNState];
  cur.load((size_t)y * cur.pitch + x, v);
  const size_t npix = (size_t)W * H, j = (size_t)y * W + x;
#pragma unroll
  for (int p = 0; p < kNState; ++p) dst[p * npix + j] = v[p];
}

// Inverse of k_read_state: binary32 planes in, the state copy encoded in its format.
template <class SV>
__global__ void k_write_state(const int W, const int H, const SV cur, const float* __restrict__ src) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W || y >= H) return;
  const size_t npix = (size_t)W * H, j = (size_t)y * W + x;
  float v[kNState];
#pragma unroll
  for (int p = 0; p < kNState; ++p) v[p] = src[p * npix + j];
  cur.store((size_t)y * cur.pitch + x, v);
}

template <class SV>
static cudaError_t launch_update_t(const KParams& kp, const StateDesc& prev, const SV& pv, const SV& nx,
                                  bool reset, const float* rad, const float* mot, int* err,
                                  cudaStream_t cs) {
  constexpr int bytes = update_smem_bytes<SV>();
  static bool attr_set = false;  // per instantiation
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_update<SV>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const dim3 grid((prev.W + kTW - 1) / kTW, (prev.H + kTH - 1) / kTH);
  k_update<SV><<<grid, kTileThreads, bytes, cs>>>(kp, prev.W, prev.H, reset ? 1 : 0, prev.stage_ok ? 1 : 0,
                                                   pv, nx, prev.maps, rad, mot, err);
  return cudaGetLastError();
}

cudaError_t launch_update(const KParams& kp, const StateDesc& prev, const StateDesc& next, bool reset,
                          const float* rad, const float* mot, int* err, cudaStream_t cs) {
  switch (prev.precision) {
    case 0: return launch_update_t(kp, prev, prev.f32(), next.f32(), reset, rad, mot, err, cs);
    case 1: return launch_update_t(kp, prev, prev.bf16(), next.bf16(), reset, rad, mot, err, cs);
    case 2: return launch_update_t(kp, prev, prev.f16(), next.f16(), reset, rad, mot, err, cs);
  }
  return cudaErrorInvalidValue;
}

template <class SV, int TH, int R, int MODE>
static cudaError_t launch_blend_cfg(const KParams& kp, const SV& cur, int W, int H, float* out,
                                    cudaStream_t cs) {
  constexpr int bytes = BlendGeom<TH>::kSmemBytes;
  static bool attr_set = false;  // per instantiation
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_blend<SV, TH, R, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const dim3 grid((W + kTW - 1) / kTW, (H + TH - 1) / TH);
  k_blend<SV, TH, R, MODE><<<grid, kTW * TH / R, bytes, cs>>>(kp, W, H, cur, out);
  return cudaGetLastError();
}

template <class SV, int MODE>
static cudaError_t launch_blend_mode(const KParams& kp, int cfg, const SV& cur, int W, int H,
                                     float* out, cudaStream_t cs) {
  switch (cfg) {
    case 0: return launch_blend_cfg<SV, 16, 4, MODE>(kp, cur, W, H, out, cs);
    case 1: return launch_blend_cfg<SV, 8, 4, MODE>(kp, cur, W, H, out, cs);
    case 2: return launch_blend_cfg<SV, 16, 2, MODE>(kp, cur, W, H, out, cs);
    case 3: return launch_blend_cfg<SV, 32, 4, MODE>(kp, cur, W, H, out, cs);
  }
  return cudaErrorInvalidValue;
}

template <class SV>
static cudaError_t launch_blend_sv(const KParams& kp, int cfg, const SV& cur, int W, int H,
                                   float* out, cudaStream_t cs) {
  return kp.blend_mode == 0 ? launch_blend_mode<SV, 0>(kp, cfg, cur, W, H, out, cs)
                            : launch_blend_mode<SV, 1>(kp, cfg, cur, W, H, out, cs);
}

cudaError_t launch_blend(const KParams& kp, int cfg, const StateDesc& cur, float* out, int* err, cudaStream_t cs) {
  if (cfg >= 8) return launch_blend_two_wide(kp, cfg - 8, cur, out, err, cs);
  if (cfg >= kBlendSyncConfigs) return launch_blend_pipelined(kp, cfg - kBlendSyncConfigs, cur, out, err, cs);
  switch (cur.precision) {
    case 0: return launch_blend_sv(kp, cfg, cur.f32(), cur.W, cur.H, out, cs);
    case 1: return launch_blend_sv(kp, cfg, cur.bf16(), cur.W, cur.H, out, cs);
    case 2: return launch_blend_sv(kp, cfg, cur.f16(), cur.W, cur.H, out, cs);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_write_state(const StateDesc& cur, const float* src, cudaStream_t cs) {
  const dim3 grid((cur.W + 127) / 128, cur.H);
  switch (cur.precision) {
    case 0: k_write_state<<<grid, 128, 0, cs>>>(cur.W, cur.H, cur.f32(), src); break;
    case 1: k_write_state<<<grid, 128, 0, cs>>>(cur.W, cur.H, cur.bf16(), src); break;
    case 2: k_write_state<<<grid, 128, 0, cs>>>(cur.W, cur.H, cur.f16(), src); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_read_state(const StateDesc& cur, float* dst, cudaStream_t cs) {
  const dim3 grid((cur.W + 127) / 128, cur.H);
  switch (cur.precision) {
    case 0: k_read_state<<<grid, 128, 0, cs>>>(cur.W, cur.H, cur.f32(), dst); break;
    case 1: k_read_state<<<grid, 128, 0, cs>>>(cur.W, cur.H, cur.bf16(), dst); break;
    case 2: k_read_state<<<grid, 128, 0, cs>>>(cur.W, cur.H, cur.f16(), dst); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace wrls
