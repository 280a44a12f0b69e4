// Device side of the fused wavefront schedule (see wrls_fused.cu): one work item = the
// temporal update of one 32 x 8 tile plus, a few items behind, the blend of one 32 x 16 tile
// whose update dependencies all have smaller item indices.
#pragma once
#include "wrls_tiles.cuh"

namespace wrls {

constexpr int kFusedTH = 16;  // blend tile rows

__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Items of one frame when blends trail their last dependency by `lag` items.
__host__ __device__ inline int fused_items(int W, int H, int lag) {
  const int nx = (W + kTW - 1) / kTW;
  const int n_u = nx * ((H + kTH - 1) / kTH);
  const int nbb = (H + kFusedTH - 1) / kFusedTH;
  const int last_blend = 2 * nbb * nx + nx + 1 + lag;  // item of blend tile (nx-1, nbb-1)
  return n_u > last_blend + 1 ? n_u : last_blend + 1;
}

// Lag of the blends behind their dependencies: about twice the CTAs in flight (so the
// dependencies have finished, not merely started), at most the frame's update tiles.
__host__ __device__ inline int fused_lag(int W, int H, int ctas) {
  const int n_u = ((W + kTW - 1) / kTW) * ((H + kTH - 1) / kTH);
  return 2 * ctas < n_u ? 2 * ctas : n_u;
}

template <class SV>
constexpr int fused_smem_bytes() {
  return (update_smem_bytes<SV>() > BlendGeom<kFusedTH>::kSmemBytes + 128)
             ? update_smem_bytes<SV>()
             : BlendGeom<kFusedTH>::kSmemBytes + 128;
}

// Work item k of one frame: update tile k (if any) and publish its flag, then the blend tile
// scheduled at k (if any) once its dependencies' flags carry `epoch`. Blend tile (c, p) is
// scheduled at item (2p+2) nx + c + 2 + lag: `lag` items after its last dependency. `base` is the 128-byte
// aligned shared space (update tile or blend window), `bar` the CTA's mbarrier. Returns false
// if a bounded wait gave up (the error word is set; the caller stops claiming work).
template <class SV, int MODE, int R>
__device__ __forceinline__ bool fused_item(unsigned char* base, uint64_t* bar, uint32_t& phase, int* s_ok,
                                           const int k, const KParams& kp, const int W, const int H,
                                           const bool reset, const bool stage_ok, const SV& prev, const SV& next,
                                           const StageMaps* maps, const float* __restrict__ rad,
                                           const float* __restrict__ mot, float* __restrict__ out, int* err,
                                           int* flags, const int epoch, const int lag) {
  constexpr int PIX = BlendGeom<kFusedTH>::kPix;
  UpdateSmem<SV>& us = *reinterpret_cast<UpdateSmem<SV>*>(base);
  float4* bw = reinterpret_cast<float4*>(base);  // the blend window reuses the update space
  const int nx = (W + kTW - 1) / kTW;
  const int nbu = (H + kTH - 1) / kTH;
  const int nbb = (H + kFusedTH - 1) / kFusedTH;
  const int n_u = nx * nbu;
  if (k < n_u) {
    if (!update_tile(us, bar, phase, err, kp, W, H, reset, stage_ok, prev, next, maps, rad, mot, (k % nx) * kTW,
                     (k / nx) * kTH))
      return false;
    __syncthreads();  // every thread's state stores precede the flag
    if (threadIdx.x == 0) {
      __threadfence();
      st_release_gpu(flags + k, epoch);
    }
  }
  const int kk = k - 2 - lag;
  if (kk < 0) return true;
  const int bu = kk / nx;
  if (bu < 2 || (bu & 1)) return true;
  const int p = bu / 2 - 1;
  if (p >= nbb) return true;
  const int c = kk % nx;
  if (threadIdx.x == 0) {
    int ok = 1;
    const long long t0 = clock64();
    for (int b = max(2 * p - 1, 0); ok && b <= min(2 * p + 2, nbu - 1); ++b)
      for (int cc = max(c - 1, 0); ok && cc <= min(c + 1, nx - 1); ++cc)
        while (ld_acquire_gpu(flags + b * nx + cc) != epoch) {
          if (clock64() - t0 > kWaitLimit) {
            ok = 0;
            break;
          }
        }
    if (!ok) atomicExch(err, (int)WRLS_ERR_TIMEOUT);
    *s_ok = ok;
  }
  __syncthreads();
  if (!*s_ok) return false;
  blend_fill<SV, kFusedTH, kTileThreads, true, 2>(bw, bw + 3 * PIX, kp, W, H, next, c * kTW, p * kFusedTH);
  __syncthreads();
  if (threadIdx.x < kTW * kFusedTH / R)
    blend_compute<kFusedTH, R, MODE>(bw, bw + 3 * PIX, kp, W, H, out, c * kTW, p * kFusedTH);
  return true;
}

// The last CTA of a launch to leave resets the two work counters for the next launch.
__device__ __forceinline__ void fused_exit(int* work) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const int done = atomicAdd(work + 1, 1);
    if (done == (int)gridDim.x - 1) {
      atomicExch(work, 0);
      atomicExch(work + 1, 0);
    }
  }
}

}  // namespace wrls
