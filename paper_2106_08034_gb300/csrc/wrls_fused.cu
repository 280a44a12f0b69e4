// Fused wavefront kernel: the temporal update and the spatial blend of one frame in a single
// persistent launch, overlapping the memory-bound update of some tiles with the arithmetic-
// bound blend of others.
//
// Work items are claimed in raster order from a counter. Item k
//   1. updates 32 x 8 tile k (reprojection, Eq. 12-14/9/11; update_tile), writes its new state
//      and publishes the tile's done flag (release, stamped with the frame's epoch);
//   2. blends one 32 x 16 tile whose 5x5 windows touch update tiles that all have smaller item
//      indices: blend tile (c, p) (rows 16p .. 16p+15) reads update bands 2p-1 .. 2p+2 and columns
//      c-1 .. c+1, the largest of which is item (2p+2) nx + c + 1, so it is scheduled at item
//      (2p+2) nx + c + 2 + lag, with lag about twice the number of resident CTAs, so its
//      dependencies have normally finished when it starts. Its state comes from L2 (written
//      shortly before), not from DRAM.
// A CTA waits for a dependency only after that dependency's item was claimed by a running CTA,
// which finishes its update without waiting on anything: the waits cannot form a cycle.
// Every wait is bounded (kWaitLimit clocks): on expiry the CTA records WRLS_ERR_TIMEOUT in the
// stream's error word and stops claiming work. The last CTA to leave resets the counters, so
// no per-frame memset is needed. Results are bitwise identical to the two-kernel path (same
// tile bodies, same arithmetic order).
#include "wrls_internal.h"
#include "wrls_fused.cuh"

namespace wrls {

template <class SV, int MODE, int R, int MIN_CTAS>
__global__ void __launch_bounds__(kTileThreads, MIN_CTAS)
    k_fused(const KParams kp, const int W, const int H, const int reset, const int stage_ok, const SV prev,
            const SV next, const __grid_constant__ StageMaps maps, const float* __restrict__ rad,
            const float* __restrict__ mot, float* __restrict__ out, int* err, int* work, int* flags,
            const int epoch, const int lag) {
  extern __shared__ unsigned char dsmem[];
  unsigned char* base = align128(dsmem);
  __shared__ alignas(8) uint64_t bar;
  __shared__ int s_item, s_ok;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  uint32_t phase = 0;
  const int n_items = fused_items(W, H, lag);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(work, 1);
    __syncthreads();
    const int k = s_item;
    if (k >= n_items) break;
    if (!fused_item<SV, MODE, R>(base, &bar, phase, &s_ok, k, kp, W, H, reset != 0, stage_ok != 0, prev, next,
                                 &maps, rad, mot, out, err, flags, epoch, lag))
      break;
  }
  fused_exit(work);
}
template <class SV, int MODE, int R, int MIN_CTAS>
static cudaError_t launch_fused_t(const KParams& kp, const StateDesc& prev, const SV& pv, const SV& nx_,
                                  bool reset, const float* rad, const float* mot, float* out, int* err,
                                  int* work, int* flags, int epoch, cudaStream_t cs) {
  constexpr int bytes = fused_smem_bytes<SV>();
  static int per_sm = 0;  // per instantiation
  if (!per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_fused<SV, MODE, R, MIN_CTAS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         bytes);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused<SV, MODE, R, MIN_CTAS>, kTileThreads, bytes);
    if (e != cudaSuccess) return e;
    per_sm = occ > 0 ? occ : 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int grid = sms * per_sm;
  const int lag = fused_lag(prev.W, prev.H, grid);
  const int items = fused_items(prev.W, prev.H, lag);
  if (grid > items) grid = items;
  k_fused<SV, MODE, R, MIN_CTAS><<<grid, kTileThreads, bytes, cs>>>(kp, prev.W, prev.H, reset ? 1 : 0, prev.stage_ok ? 1 : 0, pv,
                                                       nx_, prev.maps, rad, mot, out, err, work, flags, epoch, lag);
  return cudaGetLastError();
}

template <class SV, int R, int MIN_CTAS>
static cudaError_t launch_fused_r(const KParams& kp, const StateDesc& prev, const SV& pv, const SV& nx_,
                                  bool reset, const float* rad, const float* mot, float* out, int* err,
                                  int* work, int* flags, int epoch, cudaStream_t cs) {
  return kp.blend_mode == 0
             ? launch_fused_t<SV, 0, R, MIN_CTAS>(kp, prev, pv, nx_, reset, rad, mot, out, err, work, flags, epoch, cs)
             : launch_fused_t<SV, 1, R, MIN_CTAS>(kp, prev, pv, nx_, reset, rad, mot, out, err, work, flags, epoch, cs);
}

template <class SV>
static cudaError_t launch_fused_sv(int variant, const KParams& kp, const StateDesc& prev, const SV& pv,
                                   const SV& nx_, bool reset, const float* rad, const float* mot, float* out,
                                   int* err, int* work, int* flags, int epoch, cudaStream_t cs) {
  return variant == 2 ? launch_fused_r<SV, 4, 2>(kp, prev, pv, nx_, reset, rad, mot, out, err, work, flags, epoch, cs)
                      : launch_fused_r<SV, 2, 3>(kp, prev, pv, nx_, reset, rad, mot, out, err, work, flags, epoch, cs);
}

size_t fused_scratch_bytes(int W, int H) {
  const size_t n_u = (size_t)((W + kTW - 1) / kTW) * ((H + kTH - 1) / kTH);
  return 256 + n_u * sizeof(int);
}

cudaError_t launch_fused(int variant, const KParams& kp, const StateDesc& prev, const StateDesc& next, bool reset,
                         const float* rad, const float* mot, float* out, int* err, int* work, int* flags,
                         int epoch, cudaStream_t cs) {
  switch (prev.precision) {
    case 0: return launch_fused_sv(variant, kp, prev, prev.f32(), next.f32(), reset, rad, mot, out, err, work, flags, epoch, cs);
    case 1: return launch_fused_sv(variant, kp, prev, prev.bf16(), next.bf16(), reset, rad, mot, out, err, work, flags, epoch, cs);
    case 2: return launch_fused_sv(variant, kp, prev, prev.f16(), next.f16(), reset, rad, mot, out, err, work, flags, epoch, cs);
  }
  return cudaErrorInvalidValue;
}

}  // namespace wrls
