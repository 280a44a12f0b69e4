// Persistent, software-pipelined blend for the binary32 state.
//
// Same arithmetic and neighbour order as k_blend (wrls_tiles.cuh: blend_compute), hence
// bitwise identical outputs. Each CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// and keeps two shared windows: while it blends tile i from one window, the 4-byte cp.async
// copies of tile i+1's window (12 beta and 3 z planes, written straight into the per-pixel
// records) are in flight into the other. The copies hold no registers, so the fill latency
// hides behind the blend arithmetic. When a window has landed, one pass computes each
// record's 1/(|z|+eps). Window pixels outside the image are written directly as far records
// (beta = 0, z = kFarZ), whose weights are exactly 0.
#include "wrls_internal.h"
#include "wrls_tiles.cuh"

namespace wrls {

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem_dst)), "l"(gmem_src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int TH, int NT>
__device__ __forceinline__ void pipe_fill_issue(float4* __restrict__ sb, float4* __restrict__ szr,
                                                const StateF32& cur, const int W, const int H,
                                                const int bx0, const int by0) {
  constexpr int R0 = kMaxRadius;
  for (int i = threadIdx.x; i < BlendGeom<TH>::kPix; i += NT) {
    const int ly = i / kBlendSW, lx = i % kBlendSW;
    const int gx = bx0 - R0 + lx, gy = by0 - R0 + ly;
    if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
      const float* src = cur.base + (size_t)gy * cur.pitch + gx;
      float* b = (float*)(sb + 3 * i);
#pragma unroll
      for (int p = 0; p < 12; ++p) cp_async4(b + p, src + p * cur.plane_stride);
      float* z = (float*)(szr + i);
#pragma unroll
      for (int c = 0; c < 3; ++c) cp_async4(z + c, src + (kZ + c) * cur.plane_stride);
    } else {
      const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      sb[3 * i + 0] = zero;
      sb[3 * i + 1] = zero;
      sb[3 * i + 2] = zero;
      szr[i] = make_float4(kFarZ, kFarZ, kFarZ, 0.0f);
    }
  }
  cp_async_commit();
}

// 1/(|z|+eps) of every record (far records get a value ~6e-19, below any pixel's own r).
template <int TH, int NT>
__device__ __forceinline__ void pipe_recip_pass(float4* __restrict__ szr, const float eps) {
  for (int i = threadIdx.x; i < BlendGeom<TH>::kPix; i += NT) {
    float4 q = szr[i];
    q.w = 1.0f / (sqrtf(q.x * q.x + q.y * q.y + q.z * q.z) + eps);
    szr[i] = q;
  }
}

template <int TH, int R, int MODE>
__global__ void __launch_bounds__(kTW * TH / R)
    k_blend_pipe(const KParams kp, const int W, const int H, const StateF32 cur, float* __restrict__ out) {
  constexpr int NT = kTW * TH / R;
  constexpr int PIX = BlendGeom<TH>::kPix;
  extern __shared__ float4 smem[];  // two windows, each [3 * PIX beta records][PIX z records]
  const int tiles_x = (W + kTW - 1) / kTW;
  const int n_tiles = tiles_x * ((H + TH - 1) / TH);
  int tile = blockIdx.x;
  if (tile >= n_tiles) return;
  pipe_fill_issue<TH, NT>(smem, smem + 3 * PIX, cur, W, H, (tile % tiles_x) * kTW, (tile / tiles_x) * TH);
  for (int it = 0;; ++it) {
    float4* sb = smem + (it & 1) * 4 * PIX;
    float4* sz = sb + 3 * PIX;
    const int next = tile + gridDim.x;
    if (next < n_tiles) {
      float4* nb = smem + ((it & 1) ^ 1) * 4 * PIX;
      pipe_fill_issue<TH, NT>(nb, nb + 3 * PIX, cur, W, H, (next % tiles_x) * kTW, (next / tiles_x) * TH);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    pipe_recip_pass<TH, NT>(sz, kp.eps);
    __syncthreads();
    blend_compute<TH, R, MODE>(sb, sz, kp, W, H, out, (tile % tiles_x) * kTW, (tile / tiles_x) * TH);
    if (next >= n_tiles) break;
    __syncthreads();  // buf is refilled by the next iteration's copies
    tile = next;
  }
}

template <int TH, int R, int MODE>
static cudaError_t launch_pipe_cfg(const KParams& kp, const StateF32& cur, int W, int H, float* out,
                                   cudaStream_t cs) {
  constexpr int bytes = 2 * BlendGeom<TH>::kSmemBytes;
  constexpr int nt = kTW * TH / R;
  static int grid_per_sm = 0;  // per instantiation
  if (!grid_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_blend_pipe<TH, R, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         bytes);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_blend_pipe<TH, R, MODE>, nt, bytes);
    if (e != cudaSuccess) return e;
    grid_per_sm = occ > 0 ? occ : 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int n_tiles = ((W + kTW - 1) / kTW) * ((H + TH - 1) / TH);
  int grid = sms * grid_per_sm;
  if (grid > n_tiles) grid = n_tiles;
  k_blend_pipe<TH, R, MODE><<<grid, nt, bytes, cs>>>(kp, W, H, cur, out);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_pipe_mode(const KParams& kp, int cfg, const StateF32& cur, int W, int H, float* out,
                                    cudaStream_t cs) {
  switch (cfg) {
    case 0: return launch_pipe_cfg<16, 4, MODE>(kp, cur, W, H, out, cs);
    case 1: return launch_pipe_cfg<8, 4, MODE>(kp, cur, W, H, out, cs);
    case 2: return launch_pipe_cfg<16, 2, MODE>(kp, cur, W, H, out, cs);
    case 3: return launch_pipe_cfg<8, 2, MODE>(kp, cur, W, H, out, cs);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_blend_pipelined(const KParams& kp, int cfg, const StateDesc& cur, float* out, cudaStream_t cs) {
  if (cur.precision != 0) return cudaErrorInvalidValue;
  return kp.blend_mode == 0 ? launch_pipe_mode<0>(kp, cfg, cur.f32(), cur.W, cur.H, out, cs)
                            : launch_pipe_mode<1>(kp, cfg, cur.f32(), cur.W, cur.H, out, cs);
}

}  // namespace wrls
