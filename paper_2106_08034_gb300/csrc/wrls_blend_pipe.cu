// Persistent blend with TMA double-buffered windows (binary32 state).
//
// Same arithmetic and neighbour order as k_blend (wrls_tiles.cuh: blend_compute), hence
// bitwise identical outputs. Each CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// and keeps two shared windows. While it blends tile i from one window, two bulk tensor
// copies (cp.async.bulk.tensor.3d: the 12 beta planes and the 3 z planes of the 40 x (TH+4)
// box around tile i+1) fill the other, completion tracked by that window's mbarrier; no
// thread spends an instruction or a register per loaded value. When a window has landed, one
// pass computes every pixel's rk = K / (|z|+eps)^2 (K = log2(e) / h_s^2) and turns pixels outside
// the image (zero-filled by the copy, or pitch padding) into far records (beta = 0,
// z = kFarZ, rk = 0), whose blend weights are exactly 0. The blend then reads the window's
// planes directly (structure of arrays: a warp's loads are 32 consecutive floats).
// Waits are bounded (kWaitLimit clocks); on expiry the CTA records WRLS_ERR_TIMEOUT, waits
// (bounded) for its copies in flight and returns.
#include <string.h>

#include "wrls_internal.h"
#include "wrls_tiles.cuh"

namespace wrls {

template <int TH>
struct TmaBlendGeom {
  static constexpr int SH = TH + 2 * kMaxRadius;
  static constexpr int PLANE = SH * kBlendBoxW;   // floats per plane of a window
  static constexpr int BUF = 16 * PLANE;          // 12 beta + 3 z + rk planes
  static constexpr uint32_t kTx = 15u * PLANE * 4u;
  static constexpr int smem_bytes(int nbuf) { return nbuf * BUF * 4 + 128; }
};

// Blend from a structure-of-arrays window whose origin is (bx0 - 4, by0 - 2).
template <int TH, int R, int MODE>
__device__ __forceinline__ void blend_compute_soa(const float* __restrict__ w, const KParams& kp, const int W,
                                                  const int H, float* __restrict__ out, const int bx0,
                                                  const int by0) {
  constexpr int R0 = kMaxRadius;
  constexpr int RW = 2 * R0 + 1;
  constexpr int SW = kBlendBoxW;
  constexpr int P = TmaBlendGeom<TH>::PLANE;
  const int tx = threadIdx.x % kTW, ty = threadIdx.x / kTW;
  const int x = bx0 + tx, y0 = by0 + ty * R;
  const bool feat = kp.feature_mode == 0;
  float zi[R][3], pf[R][3], ri[R], den[R], acc[R][3];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int idx = (ty * R + i + R0) * SW + tx + 4;
    zi[i][0] = w[12 * P + idx]; zi[i][1] = w[13 * P + idx]; zi[i][2] = w[14 * P + idx];
    ri[i] = w[15 * P + idx];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pf[i][c] = feat ? zi[i][c] : 0.0f;
      acc[i][c] = 0.0f;
    }
    den[i] = 0.0f;
  }
#pragma unroll
  for (int kr = 0; kr < R + 2 * R0; ++kr) {
#pragma unroll
    for (int dx = -R0; dx <= R0; ++dx) {
      const int idx = (ty * R + kr) * SW + tx + 4 + dx;
      const float zk0 = w[12 * P + idx], zk1 = w[13 * P + idx], zk2 = w[14 * P + idx], rkk = w[15 * P + idx];
      float bk[12];
#pragma unroll
      for (int p = 0; p < 12; ++p) bk[p] = w[p * P + idx];
      float pk0 = 0.0f, pk1 = 0.0f, pk2 = 0.0f;
      if (MODE == 1) {
        const float a1 = feat ? zk0 : 0.0f, a2 = feat ? zk1 : 0.0f, a3 = feat ? zk2 : 0.0f;
        pk0 = cross_pred(bk[0], bk[1], bk[2], bk[3], a1, a2, a3);
        pk1 = cross_pred(bk[4], bk[5], bk[6], bk[7], a1, a2, a3);
        pk2 = cross_pred(bk[8], bk[9], bk[10], bk[11], a1, a2, a3);
      }
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int dy = kr - R0 - i;
        if (dy < -R0 || dy > R0) continue;  // compile-time
        const float e0 = zi[i][0] - zk0, e1 = zi[i][1] - zk1, e2 = zi[i][2] - zk2;
        const float rk = fmaxf(ri[i], rkk);
        const float b = ex2_approx(blend_exponent(kp.spatial[(dy + R0) * RW + (dx + R0)], e0, e1, e2, rk));
        den[i] += b;
        if (MODE == 0) {
          pk0 = cross_pred(bk[0], bk[1], bk[2], bk[3], pf[i][0], pf[i][1], pf[i][2]);
          pk1 = cross_pred(bk[4], bk[5], bk[6], bk[7], pf[i][0], pf[i][1], pf[i][2]);
          pk2 = cross_pred(bk[8], bk[9], bk[10], bk[11], pf[i][0], pf[i][1], pf[i][2]);
        }
        acc[i][0] = fmaf(b, pk0, acc[i][0]);
        acc[i][1] = fmaf(b, pk1, acc[i][1]);
        acc[i][2] = fmaf(b, pk2, acc[i][2]);
      }
    }
  }
  if (x >= W) return;
  const size_t npix = (size_t)W * H;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int y = y0 + i;
    if (y >= H) break;
    const float inv = 1.0f / den[i];
    const size_t j = (size_t)y * W + x;
    out[j] = acc[i][0] * inv;
    out[npix + j] = acc[i][1] * inv;
    out[2 * npix + j] = acc[i][2] * inv;
  }
}

// NBUF = 2: the next tile's window is copied while the current one is blended. NBUF = 1: one
// window (half the shared memory, twice the CTAs per SM): the next copy starts once the
// current tile is blended, and other CTAs of the SM compute meanwhile.
template <int TH, int R, int MODE, int NBUF>
__global__ void __launch_bounds__(kTW * TH / R)
    k_blend_tma(const KParams kp, const int W, const int H, const __grid_constant__ BlendMaps maps,
                float* __restrict__ out, int* err) {
  using G = TmaBlendGeom<TH>;
  constexpr int NT = kTW * TH / R;
  constexpr int P = G::PLANE;
  extern __shared__ unsigned char dsmem[];
  float* sm = reinterpret_cast<float*>(align128(dsmem));
  __shared__ alignas(8) uint64_t bar[2];
  const CUtensorMap* mb = TH == 16 ? &maps.beta16 : &maps.beta8;
  const CUtensorMap* mz = TH == 16 ? &maps.z16 : &maps.z8;
  const int tiles_x = (W + kTW - 1) / kTW;
  const int n_tiles = tiles_x * ((H + TH - 1) / TH);
  int tile = blockIdx.x;
  if (tile >= n_tiles) return;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  __syncthreads();
  uint32_t ph0 = 0u, ph1 = 0u;  // phases of the two windows' mbarriers
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar[0], G::kTx);
    tma_load_3d(sm, mb, (tile % tiles_x) * kTW - 4, (tile / tiles_x) * TH - 2, 0, &bar[0]);
    tma_load_3d(sm + 12 * P, mz, (tile % tiles_x) * kTW - 4, (tile / tiles_x) * TH - 2, kZ, &bar[0]);
  }
  for (int it = 0;; ++it) {
    const int b = NBUF == 2 ? (it & 1) : 0;
    float* wcur = sm + b * G::BUF;
    const int next = tile + gridDim.x;
    if (NBUF == 2 && next < n_tiles && threadIdx.x == 0) {  // the other window was released by the last barrier
      float* wn = sm + (b ^ 1) * G::BUF;
      fence_proxy_async();
      mbar_expect_tx(&bar[b ^ 1], G::kTx);
      tma_load_3d(wn, mb, (next % tiles_x) * kTW - 4, (next / tiles_x) * TH - 2, 0, &bar[b ^ 1]);
      tma_load_3d(wn + 12 * P, mz, (next % tiles_x) * kTW - 4, (next / tiles_x) * TH - 2, kZ, &bar[b ^ 1]);
    }
    const uint32_t ph = b ? ph1 : ph0;
    const bool ok = mbar_wait_bounded(&bar[b], ph);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(err, (int)WRLS_ERR_TIMEOUT);
      mbar_wait_bounded(&bar[b], ph);  // copies may still be in flight
      if (NBUF == 2 && next < n_tiles) mbar_wait_bounded(&bar[b ^ 1], b ? ph0 : ph1);
      return;
    }
    if (b) ph1 ^= 1u; else ph0 ^= 1u;
    const int bx0 = (tile % tiles_x) * kTW, by0 = (tile / tiles_x) * TH;
    for (int i = threadIdx.x; i < P; i += NT) {
      const int gx = bx0 - 4 + i % kBlendBoxW, gy = by0 - 2 + i / kBlendBoxW;
      if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
        wcur[15 * P + i] = blend_rk(wcur[12 * P + i], wcur[13 * P + i], wcur[14 * P + i], kp.eps, kp.range_k);
      } else {
#pragma unroll
        for (int p = 0; p < 12; ++p) wcur[p * P + i] = 0.0f;
        wcur[12 * P + i] = kFarZ;
        wcur[13 * P + i] = kFarZ;
        wcur[14 * P + i] = kFarZ;
        wcur[15 * P + i] = 0.0f;
      }
    }
    __syncthreads();
    blend_compute_soa<TH, R, MODE>(wcur, kp, W, H, out, bx0, by0);
    if (next >= n_tiles) break;
    __syncthreads();  // this window is refilled by a later copy
    if (NBUF == 1 && threadIdx.x == 0) {
      fence_proxy_async();
      mbar_expect_tx(&bar[0], G::kTx);
      tma_load_3d(sm, mb, (next % tiles_x) * kTW - 4, (next / tiles_x) * TH - 2, 0, &bar[0]);
      tma_load_3d(sm + 12 * P, mz, (next % tiles_x) * kTW - 4, (next / tiles_x) * TH - 2, kZ, &bar[0]);
    }
    tile = next;
  }
}

template <int TH, int R, int MODE, int NBUF>
static cudaError_t launch_tma_cfg(const KParams& kp, const StateDesc& cur, float* out, int* err, cudaStream_t cs) {
  constexpr int bytes = TmaBlendGeom<TH>::smem_bytes(NBUF);
  constexpr int nt = kTW * TH / R;
  static int per_sm = 0;  // per instantiation
  if (!per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_blend_tma<TH, R, MODE, NBUF>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_blend_tma<TH, R, MODE, NBUF>, nt, bytes);
    if (e != cudaSuccess) return e;
    per_sm = occ > 0 ? occ : 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int n_tiles = ((cur.W + kTW - 1) / kTW) * ((cur.H + TH - 1) / TH);
  const int use = (kp.blend_ctas_cap > 0 && kp.blend_ctas_cap < per_sm) ? kp.blend_ctas_cap : per_sm;
  int grid = sms * use;
  if (grid > n_tiles) grid = n_tiles;
  k_blend_tma<TH, R, MODE, NBUF><<<grid, nt, bytes, cs>>>(kp, cur.W, cur.H, cur.bmaps, out, err);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_tma_mode(const KParams& kp, int cfg, const StateDesc& cur, float* out, int* err,
                                   cudaStream_t cs) {
  switch (cfg) {
    case 0: return launch_tma_cfg<16, 2, MODE, 2>(kp, cur, out, err, cs);
    case 1: return launch_tma_cfg<16, 2, MODE, 1>(kp, cur, out, err, cs);
    case 2: return launch_tma_cfg<8, 2, MODE, 2>(kp, cur, out, err, cs);
    case 3: return launch_tma_cfg<16, 4, MODE, 1>(kp, cur, out, err, cs);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_blend_pipelined(const KParams& kp, int cfg, const StateDesc& cur, float* out, int* err,
                                   cudaStream_t cs) {
  if (cur.precision != 0 || !cur.blend_tma_ok) return cudaErrorInvalidValue;
  return kp.blend_mode == 0 ? launch_tma_mode<0>(kp, cfg, cur, out, err, cs)
                            : launch_tma_mode<1>(kp, cfg, cur, out, err, cs);
}

}  // namespace wrls

// ---- two-wide variant: each thread blends 2 adjacent columns x R rows -----------------------
//
// Tiles are 64 x TH; the window is kBlendBoxW2 = 72 columns (64 + 2 x 4) x (TH + 4) rows of the
// 12 beta and 3 z planes (one TMA box each) plus a plane of -rk. A thread's two output columns
// 2tx and 2tx+1 have neighbour columns 2tx-2 .. 2tx+3: three aligned column pairs, each
// fetched with one 64-bit shared load per plane, so each neighbour value is loaded once for up
// to two output columns and R rows. Same arithmetic and neighbour order per output as
// blend_compute, hence bitwise identical outputs.
namespace wrls {

template <int TH>
struct TmaBlend2Geom {
  static constexpr int SH = TH + 2 * kMaxRadius;
  static constexpr int PLANE = SH * kBlendBoxW2;
  static constexpr int BUF = 16 * PLANE;
  static constexpr uint32_t kTx = 15u * PLANE * 4u;
  static constexpr int kSmemBytes = BUF * 4 + 128;
};

template <int TH, int R, int MODE>
__device__ __forceinline__ void blend_compute_soa2(const float* __restrict__ w, const KParams& kp, const int W,
                                                   const int H, float* __restrict__ out, const int bx0,
                                                   const int by0) {
  constexpr int R0 = kMaxRadius;
  constexpr int RW = 2 * R0 + 1;
  constexpr int SW = kBlendBoxW2;
  constexpr int P = TmaBlend2Geom<TH>::PLANE;
  constexpr int NO = 2 * R;  // outputs per thread: (column o, row i) -> o * R + i
  const int tx = threadIdx.x % kTW, ty = threadIdx.x / kTW;
  const int x = bx0 + 2 * tx, y0 = by0 + ty * R;
  const bool feat = kp.feature_mode == 0;
  float zi[NO][3], pf[NO][3], ri[NO], den[NO], acc[NO][3];
#pragma unroll
  for (int o = 0; o < 2; ++o)
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int idx = (ty * R + i + R0) * SW + 2 * tx + 4 + o;
      const int q = o * R + i;
      zi[q][0] = w[12 * P + idx]; zi[q][1] = w[13 * P + idx]; zi[q][2] = w[14 * P + idx];
      ri[q] = w[15 * P + idx];  // -rk
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pf[q][c] = feat ? zi[q][c] : 0.0f;
        acc[q][c] = 0.0f;
      }
      den[q] = 0.0f;
    }
#pragma unroll
  for (int kr = 0; kr < R + 2 * R0; ++kr) {
#pragma unroll
    for (int pair = 0; pair < 3; ++pair) {
      // neighbour columns 2tx-2+2pair and 2tx-1+2pair (window columns 2tx+2+2pair, +1)
      const int idx = (ty * R + kr) * SW + 2 * tx + 2 + 2 * pair;
      float2 bk2[12];
#pragma unroll
      for (int p = 0; p < 12; ++p) bk2[p] = *reinterpret_cast<const float2*>(w + p * P + idx);
      const float2 z0 = *reinterpret_cast<const float2*>(w + 12 * P + idx);
      const float2 z1 = *reinterpret_cast<const float2*>(w + 13 * P + idx);
      const float2 z2 = *reinterpret_cast<const float2*>(w + 14 * P + idx);
      const float2 rr = *reinterpret_cast<const float2*>(w + 15 * P + idx);
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int n = 2 * pair + e;  // neighbour column offset from 2tx - 2
        const float zk0 = e ? z0.y : z0.x, zk1 = e ? z1.y : z1.x, zk2 = e ? z2.y : z2.x;
        const float rkk = e ? rr.y : rr.x;
        float bk[12];
#pragma unroll
        for (int p = 0; p < 12; ++p) bk[p] = e ? bk2[p].y : bk2[p].x;
        float pk0 = 0.0f, pk1 = 0.0f, pk2 = 0.0f;
        if (MODE == 1) {
          const float a1 = feat ? zk0 : 0.0f, a2 = feat ? zk1 : 0.0f, a3 = feat ? zk2 : 0.0f;
          pk0 = cross_pred(bk[0], bk[1], bk[2], bk[3], a1, a2, a3);
          pk1 = cross_pred(bk[4], bk[5], bk[6], bk[7], a1, a2, a3);
          pk2 = cross_pred(bk[8], bk[9], bk[10], bk[11], a1, a2, a3);
        }
#pragma unroll
        for (int o = 0; o < 2; ++o) {
          const int dx = n - 2 - o;
          if (dx < -R0 || dx > R0) continue;  // compile-time
#pragma unroll
          for (int i = 0; i < R; ++i) {
            const int dy = kr - R0 - i;
            if (dy < -R0 || dy > R0) continue;  // compile-time
            const int q = o * R + i;
            const float e0 = zi[q][0] - zk0, e1 = zi[q][1] - zk1, e2 = zi[q][2] - zk2;
            const float rk = -fminf(ri[q], rkk);  // both hold -rk: max of the positive values
            const float b = ex2_approx(blend_exponent(kp.spatial[(dy + R0) * RW + (dx + R0)], e0, e1, e2, rk));
            den[q] += b;
            if (MODE == 0) {
              pk0 = cross_pred(bk[0], bk[1], bk[2], bk[3], pf[q][0], pf[q][1], pf[q][2]);
              pk1 = cross_pred(bk[4], bk[5], bk[6], bk[7], pf[q][0], pf[q][1], pf[q][2]);
              pk2 = cross_pred(bk[8], bk[9], bk[10], bk[11], pf[q][0], pf[q][1], pf[q][2]);
            }
            acc[q][0] = fmaf(b, pk0, acc[q][0]);
            acc[q][1] = fmaf(b, pk1, acc[q][1]);
            acc[q][2] = fmaf(b, pk2, acc[q][2]);
          }
        }
      }
    }
  }
  const size_t npix = (size_t)W * H;
#pragma unroll
  for (int o = 0; o < 2; ++o) {
    if (x + o >= W) break;
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int y = y0 + i;
      if (y >= H) break;
      const int q = o * R + i;
      const float inv = 1.0f / den[q];
      const size_t j = (size_t)y * W + x + o;
      out[j] = acc[q][0] * inv;
      out[npix + j] = acc[q][1] * inv;
      out[2 * npix + j] = acc[q][2] * inv;
    }
  }
}

// MODE 0 with packed binary32 pairs. The thread's two columns 2tx and 2tx+1 at the same
// neighbour offset (dx, dy) read neighbour columns c and c+1, which for even dx are the two
// halves of one aligned 64-bit load: the feature differences, the range exponent, the weight
// sum, the cross predictions and the accumulations of both outputs then take one packed
// instruction per pair of values (sub/mul/fma .f32x2). Odd dx (the halves of two different
// loads) stays scalar. Per output the neighbours are still visited row by row, dx ascending,
// with the operations of blend_exponent and cross_pred, so the results are bitwise those of
// the scalar blends.
template <int TH, int R>
__device__ __forceinline__ void blend_compute_soa2_packed(const float* __restrict__ w, const KParams& kp,
                                                          const int W, const int H, float* __restrict__ out,
                                                          const int bx0, const int by0) {
  constexpr int R0 = kMaxRadius;
  static_assert(R0 == 2, "the pairing below assumes a 5 x 5 window");
  constexpr int RW = 2 * R0 + 1;
  constexpr int SW = kBlendBoxW2;
  constexpr int P = TmaBlend2Geom<TH>::PLANE;
  const int tx = threadIdx.x % kTW, ty = threadIdx.x / kTW;
  const int x = bx0 + 2 * tx, y0 = by0 + ty * R;
  const bool feat = kp.feature_mode == 0;
  // .x: output column 2tx, .y: output column 2tx + 1
  float2 zi[R][3], pf[R][3], nri[R], den[R], acc[R][3];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int idx = (ty * R + i + R0) * SW + 2 * tx + 4;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      zi[i][c] = *reinterpret_cast<const float2*>(w + (12 + c) * P + idx);
      pf[i][c] = feat ? zi[i][c] : make_float2(0.0f, 0.0f);
      acc[i][c] = make_float2(0.0f, 0.0f);
    }
    nri[i] = *reinterpret_cast<const float2*>(w + 15 * P + idx);
    den[i] = make_float2(0.0f, 0.0f);
  }
#pragma unroll
  for (int kr = 0; kr < R + 2 * R0; ++kr) {
#pragma unroll
    for (int pair = 0; pair < 3; ++pair) {
      // neighbour columns 2tx-2+2pair (.x) and 2tx-1+2pair (.y)
      const int idx = (ty * R + kr) * SW + 2 * tx + 2 + 2 * pair;
      float2 bk[12];
#pragma unroll
      for (int p = 0; p < 12; ++p) bk[p] = *reinterpret_cast<const float2*>(w + p * P + idx);
      const float2 z0 = *reinterpret_cast<const float2*>(w + 12 * P + idx);
      const float2 z1 = *reinterpret_cast<const float2*>(w + 13 * P + idx);
      const float2 z2 = *reinterpret_cast<const float2*>(w + 14 * P + idx);
      const float2 nr = *reinterpret_cast<const float2*>(w + 15 * P + idx);
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int dy = kr - R0 - i;
        if (dy < -R0 || dy > R0) continue;  // compile-time
        // (a) column 2tx+1 against neighbour .x: dx = 2 pair - 3
        if (pair >= 1) {
          const int dx = 2 * pair - 3;
          const float e0 = zi[i][0].y - z0.x, e1 = zi[i][1].y - z1.x, e2 = zi[i][2].y - z2.x;
          const float rk = -fminf(nri[i].y, nr.x);
          const float b = ex2_approx(blend_exponent(kp.spatial[(dy + R0) * RW + (dx + R0)], e0, e1, e2, rk));
          den[i].y += b;
#pragma unroll
          for (int c = 0; c < 3; ++c)
            acc[i][c].y = fmaf(b, cross_pred(bk[4 * c].x, bk[4 * c + 1].x, bk[4 * c + 2].x, bk[4 * c + 3].x,
                                             pf[i][0].y, pf[i][1].y, pf[i][2].y), acc[i][c].y);
        }
        // (b) both columns at dx = 2 pair - 2: column 2tx against .x, column 2tx+1 against .y
        {
          const int dx = 2 * pair - 2;
          const float sp = kp.spatial[(dy + R0) * RW + (dx + R0)];
          const float2 e0 = f2sub(zi[i][0], z0), e1 = f2sub(zi[i][1], z1), e2 = f2sub(zi[i][2], z2);
          const float2 nrk = make_float2(fminf(nri[i].x, nr.x), fminf(nri[i].y, nr.y));
          const float2 t = blend_exponent2(make_float2(sp, sp), e0, e1, e2, nrk);
          const float2 b = make_float2(ex2_approx(t.x), ex2_approx(t.y));
          den[i] = f2add(den[i], b);
#pragma unroll
          for (int c = 0; c < 3; ++c)
            acc[i][c] = f2fma(b, cross_pred2(bk[4 * c], bk[4 * c + 1], bk[4 * c + 2], bk[4 * c + 3],
                                             pf[i][0], pf[i][1], pf[i][2]), acc[i][c]);
        }
        // (c) column 2tx against neighbour .y: dx = 2 pair - 1
        if (pair <= 1) {
          const int dx = 2 * pair - 1;
          const float e0 = zi[i][0].x - z0.y, e1 = zi[i][1].x - z1.y, e2 = zi[i][2].x - z2.y;
          const float rk = -fminf(nri[i].x, nr.y);
          const float b = ex2_approx(blend_exponent(kp.spatial[(dy + R0) * RW + (dx + R0)], e0, e1, e2, rk));
          den[i].x += b;
#pragma unroll
          for (int c = 0; c < 3; ++c)
            acc[i][c].x = fmaf(b, cross_pred(bk[4 * c].y, bk[4 * c + 1].y, bk[4 * c + 2].y, bk[4 * c + 3].y,
                                             pf[i][0].x, pf[i][1].x, pf[i][2].x), acc[i][c].x);
        }
      }
    }
  }
  const size_t npix = (size_t)W * H;
#pragma unroll
  for (int o = 0; o < 2; ++o) {
    if (x + o >= W) break;
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int y = y0 + i;
      if (y >= H) break;
      const float inv = 1.0f / (o ? den[i].y : den[i].x);
      const size_t j = (size_t)y * W + x + o;
      out[j] = (o ? acc[i][0].y : acc[i][0].x) * inv;
      out[npix + j] = (o ? acc[i][1].y : acc[i][1].x) * inv;
      out[2 * npix + j] = (o ? acc[i][2].y : acc[i][2].x) * inv;
    }
  }
}

// At most 128 registers a thread, so that two 256-thread CTAs (the shared-memory limit) fit an SM.
template <int TH, int R, int MODE>
__global__ void __launch_bounds__(kTW * TH / R, 65536 / 128 / (kTW * TH / R))
    k_blend_tma2(const KParams kp, const int W, const int H, const __grid_constant__ BlendMaps maps,
                 float* __restrict__ out, int* err) {
  using G = TmaBlend2Geom<TH>;
  constexpr int NT = kTW * TH / R;
  constexpr int P = G::PLANE;
  constexpr int TW2 = 2 * kTW;
  extern __shared__ unsigned char dsmem[];
  float* sm = reinterpret_cast<float*>(align128(dsmem));
  __shared__ alignas(8) uint64_t bar;
  const CUtensorMap* mb = TH == 16 ? &maps.beta16w : &maps.beta8w;
  const CUtensorMap* mz = TH == 16 ? &maps.z16w : &maps.z8w;
  const int tiles_x = (W + TW2 - 1) / TW2;
  const int n_tiles = tiles_x * ((H + TH - 1) / TH);
  int tile = blockIdx.x;
  if (tile >= n_tiles) return;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t ph = 0u;
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, G::kTx);
    tma_load_3d(sm, mb, (tile % tiles_x) * TW2 - 4, (tile / tiles_x) * TH - 2, 0, &bar);
    tma_load_3d(sm + 12 * P, mz, (tile % tiles_x) * TW2 - 4, (tile / tiles_x) * TH - 2, kZ, &bar);
  }
  for (;;) {
    const int next = tile + gridDim.x;
    const bool ok = mbar_wait_bounded(&bar, ph);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(err, (int)WRLS_ERR_TIMEOUT);
      mbar_wait_bounded(&bar, ph);  // the copies may still be in flight
      return;
    }
    ph ^= 1u;
    const int bx0 = (tile % tiles_x) * TW2, by0 = (tile / tiles_x) * TH;
    if (bx0 - 4 >= 0 && bx0 - 4 + kBlendBoxW2 <= W && by0 - 2 >= 0 && by0 - 2 + G::SH <= H) {
      // the whole window inside the image (most tiles): -rk of column pairs, no per-pixel tests
      const float2* z0 = reinterpret_cast<const float2*>(sm + 12 * P);
      const float2* z1 = reinterpret_cast<const float2*>(sm + 13 * P);
      const float2* z2 = reinterpret_cast<const float2*>(sm + 14 * P);
      float2* nrk = reinterpret_cast<float2*>(sm + 15 * P);
      for (int j = threadIdx.x; j < P / 2; j += NT) {
        const float2 r = blend_rk2(z0[j], z1[j], z2[j], kp.eps, kp.range_k);
        nrk[j] = make_float2(-r.x, -r.y);
      }
    } else for (int i = threadIdx.x; i < P; i += NT) {
      const int gx = bx0 - 4 + i % kBlendBoxW2, gy = by0 - 2 + i / kBlendBoxW2;
      if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
        sm[15 * P + i] = -blend_rk(sm[12 * P + i], sm[13 * P + i], sm[14 * P + i], kp.eps, kp.range_k);
      } else {
#pragma unroll
        for (int p = 0; p < 12; ++p) sm[p * P + i] = 0.0f;
        sm[12 * P + i] = kFarZ;
        sm[13 * P + i] = kFarZ;
        sm[14 * P + i] = kFarZ;
        sm[15 * P + i] = -0.0f;
      }
    }
    __syncthreads();
    if constexpr (MODE == 0) blend_compute_soa2_packed<TH, R>(sm, kp, W, H, out, bx0, by0);
    else blend_compute_soa2<TH, R, MODE>(sm, kp, W, H, out, bx0, by0);
    if (next >= n_tiles) break;
    __syncthreads();  // the window is refilled for the next tile
    if (threadIdx.x == 0) {
      fence_proxy_async();
      mbar_expect_tx(&bar, G::kTx);
      tma_load_3d(sm, mb, (next % tiles_x) * TW2 - 4, (next / tiles_x) * TH - 2, 0, &bar);
      tma_load_3d(sm + 12 * P, mz, (next % tiles_x) * TW2 - 4, (next / tiles_x) * TH - 2, kZ, &bar);
    }
    tile = next;
  }
}

template <int TH, int R, int MODE>
static cudaError_t launch_tma2_cfg(const KParams& kp, const StateDesc& cur, float* out, int* err, cudaStream_t cs) {
  constexpr int bytes = TmaBlend2Geom<TH>::kSmemBytes;
  constexpr int nt = kTW * TH / R;
  static int per_sm = 0;  // per instantiation
  if (!per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_blend_tma2<TH, R, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_blend_tma2<TH, R, MODE>, nt, bytes);
    if (e != cudaSuccess) return e;
    per_sm = occ > 0 ? occ : 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int n_tiles = ((cur.W + 2 * kTW - 1) / (2 * kTW)) * ((cur.H + TH - 1) / TH);
  const int use = (kp.blend_ctas_cap > 0 && kp.blend_ctas_cap < per_sm) ? kp.blend_ctas_cap : per_sm;
  int grid = sms * use;
  if (grid > n_tiles) grid = n_tiles;
  k_blend_tma2<TH, R, MODE><<<grid, nt, bytes, cs>>>(kp, cur.W, cur.H, cur.bmaps, out, err);
  return cudaGetLastError();
}

// ---- two-wide variant for the 16-bit state formats ---------------------------------------
//
// The 16-bit state stores two planes per 32-bit word (State16: word k = planes 2k, 2k + 1), so
// the blend's inputs are 8 word planes (beta: words 0-5; z: words 11-12) with the geometry of
// the binary32 planes: the same 72-column boxes from tile x - 4 (one TMA box for the 6 beta
// words, one for the 2 z words). They land in the upper half of the binary32 window buffer
// (raw word plane k in binary32 plane slot 8 + k) and are decoded in place, in three phases
// separated by barriers: raw words 0-3 into binary32 planes 0-7 (slots 8-11 are read, 0-7
// written); raw words 4-5 into planes 8-11 (slots 12-13 read, 8-11 written: raw words 0-3 are
// consumed); raw words 6-7 into z planes 12-14 and the -rk plane 15, read into registers before
// a barrier since they are overwritten. The blend is blend_compute_soa2_packed /
// blend_compute_soa2 on the decoded values, so the outputs equal those of the other blend
// configurations for the same state, and the kernel keeps the binary32 kernel's shared memory
// and occupancy.
template <int TH>
struct TmaBlend2hGeom {
  static constexpr int SH = TH + 2 * kMaxRadius;
  static constexpr int PLANE = TmaBlend2Geom<TH>::PLANE;  // one plane: SH x 72 32-bit values
  static constexpr int RAW = 8 * PLANE;                    // first raw word plane (in values)
  static constexpr uint32_t kTx = 8u * PLANE * 4u;
  static constexpr int kSmemBytes = TmaBlend2Geom<TH>::kSmemBytes;
  static constexpr int kPairs = SH * (kBlendBoxW2 / 2);   // column pairs of a window plane
  static_assert((6 * PLANE * 4) % 128 == 0, "z box destination not 128-byte aligned");
};

template <int TH, int R, int MODE, typename T>
__global__ void __launch_bounds__(kTW * TH / R, 65536 / 128 / (kTW * TH / R))
    k_blend_tma2h(const KParams kp, const int W, const int H, const __grid_constant__ BlendMaps maps,
                  float* __restrict__ out, int* err) {
  using G = TmaBlend2hGeom<TH>;
  using SV = State16<T>;
  constexpr int NT = kTW * TH / R;
  constexpr int P = G::PLANE;
  constexpr int TW2 = 2 * kTW;
  constexpr int NJ = (G::kPairs + NT - 1) / NT;  // column pairs a thread decodes per plane
  constexpr int HW = kBlendBoxW2 / 2;             // column pairs a row
  extern __shared__ unsigned char dsmem[];
  float* sm = reinterpret_cast<float*>(align128(dsmem));
  const uint2* raw = reinterpret_cast<const uint2*>(sm + G::RAW);  // (column 2cp, 2cp + 1) words
  __shared__ alignas(8) uint64_t bar;
  const CUtensorMap* mb = TH == 16 ? &maps.beta16w : &maps.beta8w;
  const CUtensorMap* mz = TH == 16 ? &maps.z16w : &maps.z8w;
  const int tiles_x = (W + TW2 - 1) / TW2;
  const int n_tiles = tiles_x * ((H + TH - 1) / TH);
  int tile = blockIdx.x;
  if (tile >= n_tiles) return;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t ph = 0u;
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, G::kTx);
    tma_load_3d(sm + G::RAW, mb, (tile % tiles_x) * TW2 - 4, (tile / tiles_x) * TH - 2, 0, &bar);
    tma_load_3d(sm + G::RAW + 6 * P, mz, (tile % tiles_x) * TW2 - 4, (tile / tiles_x) * TH - 2, 11, &bar);
  }
  for (;;) {
    const int next = tile + gridDim.x;
    const bool ok = mbar_wait_bounded(&bar, ph);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(err, (int)WRLS_ERR_TIMEOUT);
      mbar_wait_bounded(&bar, ph);  // the copies may still be in flight
      return;
    }
    ph ^= 1u;
    const int bx0 = (tile % tiles_x) * TW2, by0 = (tile / tiles_x) * TH;
    // in-image flags of a column pair (window pixels outside the image become far records)
    auto inside = [&](int j, bool& in0, bool& in1) {
      const int row = j / HW, cp = j % HW;
      const int gx = bx0 - 4 + 2 * cp, gy = by0 - 2 + row;
      const bool rin = gy >= 0 && gy < H;
      in0 = rin && gx >= 0 && gx < W;
      in1 = rin && gx + 1 >= 0 && gx + 1 < W;
    };
    // beta words 0-5 -> binary32 planes 0-11 (phase 1: words 0-3, phase 2: words 4-5)
#pragma unroll
    for (int ph2 = 0; ph2 < 2; ++ph2) {
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) {
        const int j = threadIdx.x + jj * NT;
        if (j < G::kPairs) {
          bool in0, in1;
          inside(j, in0, in1);
#pragma unroll
          for (int k = ph2 * 4; k < (ph2 ? 6 : 4); ++k) {
            const uint2 w = raw[(k * P) / 2 + j];
            const float2 a = SV::unpack(w.x), b = SV::unpack(w.y);  // (plane 2k, 2k+1) of columns 0, 1
            const float2 lo = make_float2(in0 ? a.x : 0.0f, in1 ? b.x : 0.0f);
            const float2 hi = make_float2(in0 ? a.y : 0.0f, in1 ? b.y : 0.0f);
            reinterpret_cast<float2*>(sm + (2 * k) * P)[j] = lo;
            reinterpret_cast<float2*>(sm + (2 * k + 1) * P)[j] = hi;
          }
        }
      }
      __syncthreads();  // raw words of this phase read before the next phase overwrites them
    }
    // z words 6-7 (z0 z1 | z2 e) -> planes 12-14 and -rk (plane 15): read first, they are overwritten
    {
      uint2 zw[NJ][2];
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) {
        const int j = threadIdx.x + jj * NT;
        if (j < G::kPairs) {
          zw[jj][0] = raw[(6 * P) / 2 + j];
          zw[jj][1] = raw[(7 * P) / 2 + j];
        }
      }
      __syncthreads();
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) {
        const int j = threadIdx.x + jj * NT;
        if (j < G::kPairs) {
          bool in0, in1;
          inside(j, in0, in1);
          const float2 a01 = SV::unpack(zw[jj][0].x), b01 = SV::unpack(zw[jj][0].y);
          const float a2 = SV::unpack(zw[jj][1].x).x, b2 = SV::unpack(zw[jj][1].y).x;
          const float2 z0 = make_float2(in0 ? a01.x : kFarZ, in1 ? b01.x : kFarZ);
          const float2 z1 = make_float2(in0 ? a01.y : kFarZ, in1 ? b01.y : kFarZ);
          const float2 z2 = make_float2(in0 ? a2 : kFarZ, in1 ? b2 : kFarZ);
          reinterpret_cast<float2*>(sm + 12 * P)[j] = z0;
          reinterpret_cast<float2*>(sm + 13 * P)[j] = z1;
          reinterpret_cast<float2*>(sm + 14 * P)[j] = z2;
          reinterpret_cast<float2*>(sm + 15 * P)[j] =
              make_float2(in0 ? -blend_rk(z0.x, z1.x, z2.x, kp.eps, kp.range_k) : -0.0f,
                          in1 ? -blend_rk(z0.y, z1.y, z2.y, kp.eps, kp.range_k) : -0.0f);
        }
      }
    }
    __syncthreads();
    if constexpr (MODE == 0) blend_compute_soa2_packed<TH, R>(sm, kp, W, H, out, bx0, by0);
    else blend_compute_soa2<TH, R, MODE>(sm, kp, W, H, out, bx0, by0);
    if (next >= n_tiles) break;
    __syncthreads();  // the buffer is refilled for the next tile
    if (threadIdx.x == 0) {
      fence_proxy_async();
      mbar_expect_tx(&bar, G::kTx);
      tma_load_3d(sm + G::RAW, mb, (next % tiles_x) * TW2 - 4, (next / tiles_x) * TH - 2, 0, &bar);
      tma_load_3d(sm + G::RAW + 6 * P, mz, (next % tiles_x) * TW2 - 4, (next / tiles_x) * TH - 2, 11, &bar);
    }
    tile = next;
  }
}

template <int TH, int R, int MODE, typename T>
static cudaError_t launch_tma2h_cfg(const KParams& kp, const StateDesc& cur, float* out, int* err, cudaStream_t cs) {
  constexpr int bytes = TmaBlend2hGeom<TH>::kSmemBytes;
  constexpr int nt = kTW * TH / R;
  static int per_sm = 0;  // per instantiation
  if (!per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_blend_tma2h<TH, R, MODE, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_blend_tma2h<TH, R, MODE, T>, nt, bytes);
    if (e != cudaSuccess) return e;
    per_sm = occ > 0 ? occ : 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int n_tiles = ((cur.W + 2 * kTW - 1) / (2 * kTW)) * ((cur.H + TH - 1) / TH);
  const int use = (kp.blend_ctas_cap > 0 && kp.blend_ctas_cap < per_sm) ? kp.blend_ctas_cap : per_sm;
  int grid = sms * use;
  if (grid > n_tiles) grid = n_tiles;
  k_blend_tma2h<TH, R, MODE, T><<<grid, nt, bytes, cs>>>(kp, cur.W, cur.H, cur.bmaps, out, err);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_two_wide_16(const KParams& kp, int cfg, const StateDesc& cur, float* out, int* err,
                                      cudaStream_t cs) {
  if (kp.blend_mode == 0)
    return cfg == 0 ? launch_tma2h_cfg<16, 2, 0, T>(kp, cur, out, err, cs) : launch_tma2h_cfg<8, 2, 0, T>(kp, cur, out, err, cs);
  return cfg == 0 ? launch_tma2h_cfg<16, 2, 1, T>(kp, cur, out, err, cs) : launch_tma2h_cfg<8, 2, 1, T>(kp, cur, out, err, cs);
}

cudaError_t launch_blend_two_wide(const KParams& kp, int cfg, const StateDesc& cur, float* out, int* err,
                                  cudaStream_t cs) {
  if (!cur.blend_tma2_ok) return cudaErrorInvalidValue;
  if (cur.precision == 1) return launch_two_wide_16<__nv_bfloat16>(kp, cfg, cur, out, err, cs);
  if (cur.precision == 2) return launch_two_wide_16<__half>(kp, cfg, cur, out, err, cs);
  if (cur.precision != 0) return cudaErrorInvalidValue;
  if (kp.blend_mode == 0)
    return cfg == 0 ? launch_tma2_cfg<16, 2, 0>(kp, cur, out, err, cs) : launch_tma2_cfg<8, 2, 0>(kp, cur, out, err, cs);
  return cfg == 0 ? launch_tma2_cfg<16, 2, 1>(kp, cur, out, err, cs) : launch_tma2_cfg<8, 2, 1>(kp, cur, out, err, cs);
}

}  // namespace wrls
