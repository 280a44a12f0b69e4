// Persistent, prefetching temporal update (the update half of the two-kernel pipeline).
//
// Same per-pixel arithmetic as update_tile (reprojection, Eq. 12-14/9/11), hence bitwise
// identical states. Each CTA walks the 32 x 8 tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// and keeps two buffers (staged state window + radiance tile). While it updates tile i from
// one buffer, the other is being filled for tile i+1: the footprint of tile i+1's bilinear
// taps (from motion vectors loaded one tile earlier still) is reduced over the CTA, one thread
// issues the TMA bulk tensor copy of that window of all state planes, and every thread issues
// 4-byte cp.async copies of tile i+1's radiance tile with its 1-pixel halo. So the motion,
// radiance and state loads of a tile all overlap the arithmetic of the tile before it.
// Waits for the bulk copies are bounded (kWaitLimit clocks; WRLS_ERR_TIMEOUT, then a bounded
// wait for the copies in flight and return).
#include "wrls_internal.h"
#include "wrls_tiles.cuh"

namespace wrls {

template <class SV>
struct UpdatePipeSmem {
  static constexpr int kStage = (int)((SV::kStageBytes + 127) / 128 * 128);
  alignas(128) unsigned char stage[2][kStage];
  float rad[2][3][kTH + 2][kTW + 2];
  int red[kTileThreads / 32][4];
  int box[2][4];
};

__device__ __forceinline__ void cpa4(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem_dst)), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Reprojection of this thread's pixel of the tile at (bx0, by0) given its motion (mx, my).
__device__ __forceinline__ bool reproject(int x, int y, int W, int H, bool reset, float mx, float my, float& qx,
                                          float& qy) {
  qx = (float)x + mx;
  qy = (float)y + my;
  return x < W && y < H && !reset && qx >= 0.0f && qx <= (float)(W - 1) && qy >= 0.0f && qy <= (float)(H - 1);
}

// Reduce the tile's tap footprint, issue its state-window copy into buffer `b` (thread 0) and
// the radiance tile copies (all threads). Contains one CTA barrier.
template <class SV>
__device__ __forceinline__ void prefetch_tile(UpdatePipeSmem<SV>& sm, uint64_t* bar, const int b, const int W,
                                              const int H, const bool stage_ok, const StageMaps* maps,
                                              const float* __restrict__ rad, const int bx0, const int by0,
                                              const bool valid, const float qx, const float qy) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int lo_x = 0x7fffffff, hi_x = -1, lo_y = 0x7fffffff, hi_y = -1;
  if (valid) {
    const int x0 = (int)floorf(qx), y0 = (int)floorf(qy);
    lo_x = x0; hi_x = min(x0 + 1, W - 1);
    lo_y = y0; hi_y = min(y0 + 1, H - 1);
  }
  lo_x = __reduce_min_sync(0xffffffffu, lo_x);
  hi_x = __reduce_max_sync(0xffffffffu, hi_x);
  lo_y = __reduce_min_sync(0xffffffffu, lo_y);
  hi_y = __reduce_max_sync(0xffffffffu, hi_y);
  if (lane == 0) {
    sm.red[warp][0] = lo_x; sm.red[warp][1] = hi_x; sm.red[warp][2] = lo_y; sm.red[warp][3] = hi_y;
  }
  // radiance tile with halo: in-image samples by cp.async, the rest NaN (fixed up after landing)
  const size_t npix = (size_t)W * H;
  for (int i = threadIdx.x; i < (kTH + 2) * (kTW + 2); i += kTileThreads) {
    const int ly = i / (kTW + 2), lx = i % (kTW + 2);
    const int gx = bx0 - 1 + lx, gy = by0 - 1 + ly;
    if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
      const size_t jj = (size_t)gy * W + gx;
      cpa4(&sm.rad[b][0][ly][lx], rad + jj);
      cpa4(&sm.rad[b][1][ly][lx], rad + npix + jj);
      cpa4(&sm.rad[b][2][ly][lx], rad + 2 * npix + jj);
    } else {
      const float nan = __int_as_float(0x7fc00000);
      sm.rad[b][0][ly][lx] = nan;
      sm.rad[b][1][ly][lx] = nan;
      sm.rad[b][2][ly][lx] = nan;
    }
  }
  cpa_commit();
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 1; w < kTileThreads / 32; ++w) {
      lo_x = min(lo_x, sm.red[w][0]); hi_x = max(hi_x, sm.red[w][1]);
      lo_y = min(lo_y, sm.red[w][2]); hi_y = max(hi_y, sm.red[w][3]);
    }
    int fits = 0, X0 = 0, Y0 = 0;
    if (stage_ok && hi_x >= 0) {
      X0 = lo_x - lo_x % SV::kAlignX;
      Y0 = lo_y;
      fits = (hi_x - X0 < kStageW) && (hi_y - Y0 < kStageH);
    }
    sm.box[b][0] = X0; sm.box[b][1] = Y0; sm.box[b][2] = fits;
    if (fits) {
      fence_proxy_async();
      mbar_expect_tx(&bar[b], SV::kTxBytes);
      tma_load_3d(sm.stage[b], &maps->planes, X0, Y0, 0, &bar[b]);
      if constexpr (SV::kHasScale) tma_load_2d(sm.stage[b] + SV::kScaleOffset, &maps->scale, X0, Y0, &bar[b]);
    }
  }
}

template <class SV>
__global__ void __launch_bounds__(kTileThreads)
    k_update_pipe(const KParams kp, const int W, const int H, const int reset, const int stage_ok, const SV prev,
                  const SV next, const __grid_constant__ StageMaps maps, const float* __restrict__ rad,
                  const float* __restrict__ mot, int* err) {
  extern __shared__ unsigned char dsmem[];
  UpdatePipeSmem<SV>& sm = *reinterpret_cast<UpdatePipeSmem<SV>*>(align128(dsmem));
  __shared__ alignas(8) uint64_t bar[2];
  const int tiles_x = (W + kTW - 1) / kTW;
  const int n_tiles = tiles_x * ((H + kTH - 1) / kTH);
  const int G = gridDim.x;
  int tile = blockIdx.x;
  if (tile >= n_tiles) return;
  const int tx = threadIdx.x % kTW, ty = threadIdx.x / kTW;
  const size_t npix = (size_t)W * H;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  __syncthreads();
  uint32_t ph0 = 0u, ph1 = 0u;
  auto load_motion = [&](int t, float& mx, float& my) {
    const int x = (t % tiles_x) * kTW + tx, y = (t / tiles_x) * kTH + ty;
    mx = 0.0f;
    my = 0.0f;
    if (x < W && y < H) {
      const size_t j = (size_t)y * W + x;
      mx = __ldg(mot + j);
      my = __ldg(mot + npix + j);
    }
  };
  // prologue: tile `tile` into buffer 0, motion of the following tile in flight
  float mx, my, q0x, q0y, q1x = 0.0f, q1y = 0.0f, m1x = 0.0f, m1y = 0.0f;
  load_motion(tile, mx, my);
  bool v0 = reproject((tile % tiles_x) * kTW + tx, (tile / tiles_x) * kTH + ty, W, H, reset != 0, mx, my, q0x, q0y);
  bool v1 = false;
  prefetch_tile(sm, bar, 0, W, H, stage_ok != 0, &maps, rad, (tile % tiles_x) * kTW, (tile / tiles_x) * kTH, v0,
                q0x, q0y);
  if (tile + G < n_tiles) load_motion(tile + G, m1x, m1y);
  for (int it = 0;; ++it) {
    const int b = it & 1;
    const int nxt = tile + G;
    if (nxt < n_tiles) {
      v1 = reproject((nxt % tiles_x) * kTW + tx, (nxt / tiles_x) * kTH + ty, W, H, reset != 0, m1x, m1y, q1x, q1y);
      prefetch_tile(sm, bar, b ^ 1, W, H, stage_ok != 0, &maps, rad, (nxt % tiles_x) * kTW, (nxt / tiles_x) * kTH,
                    v1, q1x, q1y);
      if (nxt + G < n_tiles) load_motion(nxt + G, m1x, m1y);
      cpa_wait<1>();  // this tile's radiance copies have landed
    } else {
      cpa_wait<0>();
    }
    const bool fits = sm.box[b][2] != 0;
    const uint32_t ph = b ? ph1 : ph0;
    bool ok = true;
    if (fits) ok = mbar_wait_bounded(&bar[b], ph);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(err, (int)WRLS_ERR_TIMEOUT);
      mbar_wait_bounded(&bar[b], ph);  // copies may still be in flight
      if (nxt < n_tiles && sm.box[b ^ 1][2]) mbar_wait_bounded(&bar[b ^ 1], b ? ph0 : ph1);
      cpa_wait<0>();
      return;
    }
    if (fits) {
      if (b) ph1 ^= 1u; else ph0 ^= 1u;
    }
    // a missing sample (a non-finite channel) becomes (NaN, NaN, NaN), skipped by the clamp
    for (int i = threadIdx.x; i < (kTH + 2) * (kTW + 2); i += kTileThreads) {
      float* p = &sm.rad[b][0][0][0] + i;
      constexpr int PL = (kTH + 2) * (kTW + 2);
      if (!(isfinite(p[0]) && isfinite(p[PL]) && isfinite(p[2 * PL]))) {
        const float nan = __int_as_float(0x7fc00000);
        p[0] = nan; p[PL] = nan; p[2 * PL] = nan;
      }
    }
    __syncthreads();
    const int x = (tile % tiles_x) * kTW + tx, y = (tile / tiles_x) * kTH + ty;
    if (x < W && y < H) {
      float I[3] = {sm.rad[b][0][ty + 1][tx + 1], sm.rad[b][1][ty + 1][tx + 1], sm.rad[b][2][ty + 1][tx + 1]};
      const bool missing = I[0] != I[0];
      float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float v = sm.rad[b][c][ty + dy][tx + dx];
            lo[c] = fminf(lo[c], v);
            hi[c] = fmaxf(hi[c], v);
          }
      const bool have_box = lo[0] <= hi[0];
      float st[kNState];
      if (v0) {
        if (fits) gather_bilinear_staged<SV>(sm.stage[b], sm.box[b][0], sm.box[b][1], W, H, q0x, q0y, st);
        else gather_bilinear(prev, W, H, q0x, q0y, st);
      }
      update_pixel(kp, v0, st, I, missing, lo, hi, have_box);
      next.store((size_t)y * next.pitch + x, st);
    }
    if (nxt >= n_tiles) break;
    __syncthreads();  // buffer b is refilled by the next iteration's prefetch
    tile = nxt;
    q0x = q1x; q0y = q1y; v0 = v1;
  }
}

template <class SV>
static cudaError_t launch_update_pipe_t(const KParams& kp, const StateDesc& prev, const SV& pv, const SV& nx,
                                       bool reset, const float* rad, const float* mot, int* err, cudaStream_t cs) {
  constexpr int bytes = (int)sizeof(UpdatePipeSmem<SV>) + 128;
  static int per_sm = 0;  // per instantiation
  if (!per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_update_pipe<SV>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_update_pipe<SV>, kTileThreads, bytes);
    if (e != cudaSuccess) return e;
    per_sm = occ > 0 ? occ : 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int n_tiles = ((prev.W + kTW - 1) / kTW) * ((prev.H + kTH - 1) / kTH);
  int grid = sms * per_sm;
  if (grid > n_tiles) grid = n_tiles;
  k_update_pipe<SV><<<grid, kTileThreads, bytes, cs>>>(kp, prev.W, prev.H, reset ? 1 : 0, prev.stage_ok ? 1 : 0, pv,
                                                       nx, prev.maps, rad, mot, err);
  return cudaGetLastError();
}

cudaError_t launch_update_pipelined(const KParams& kp, const StateDesc& prev, const StateDesc& next, bool reset,
                                    const float* rad, const float* mot, int* err, cudaStream_t cs) {
  switch (prev.precision) {
    case 0: return launch_update_pipe_t(kp, prev, prev.f32(), next.f32(), reset, rad, mot, err, cs);
    case 1: return launch_update_pipe_t(kp, prev, prev.bf16(), next.bf16(), reset, rad, mot, err, cs);
    case 2: return launch_update_pipe_t(kp, prev, prev.f16(), next.f16(), reset, rad, mot, err, cs);
  }
  return cudaErrorInvalidValue;
}

}  // namespace wrls
