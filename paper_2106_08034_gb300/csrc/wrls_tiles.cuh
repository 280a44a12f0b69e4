// Tile bodies of the wRLS denoiser, shared by the single-frame kernels (one CTA per
// tile) and the persistent batched kernel (each CTA loops over work items).
//
//  update_tile : per pixel, reprojection + Eq. 12 + Eq. 13 + Eq. 8/14/9/11 (Sec. 5.2-5.3);
//                reads the previous state copy, writes the new one.
//  blend_tile  : per pixel, the spatio-temporal blend of Sec. 5.3 over the (2r+1)^2 window
//                of models after the update; writes the denoised colour.
//
// Update tiles are 32 x 8 pixels (one warp per tile row: each plane access of a warp is one
// 128-byte row segment). The 3x3 neighbourhood of the radiance (clamp of Eq. 12) and the
// 5x5 neighbourhood of beta/z (blend) are staged in shared memory with their halos;
// out-of-image halo pixels are marked (NaN radiance, negative 1/|z|) and skipped.
// Both bodies start with a CTA barrier so a CTA may run tiles back to back.
#pragma once
#include "../../include/wrls.h"
#include "wrls_device.cuh"

namespace wrls {

constexpr int kTW = 32;
constexpr int kTH = 8;
constexpr int kTileThreads = kTW * kTH;

// Shared memory of an update tile: the staged previous-state window, the radiance tile with a
// 1-pixel halo and the tap-footprint reduction. (The copy's mbarrier lives outside, so that a
// persistent kernel keeps it, and its phase, across the tiles it runs.)
template <class SV>
struct UpdateSmem {
  alignas(128) unsigned char stage[SV::kStageBytes];
  float rad[3][kTH + 2][kTW + 2];
  int red[kTileThreads / 32][4];
  int box[4];
};
template <class SV>
constexpr int update_smem_bytes() { return (int)sizeof(UpdateSmem<SV>) + 128; }  // + alignment slack

// Update tile at (bx0, by0): the footprint of the bilinear taps of the tile's valid pixels is
// reduced over the CTA; when it fits the kStageW x kStageH box, one thread copies that window
// of every state plane into shared memory with a TMA bulk tensor copy (completion on the
// mbarrier) while all threads stage the radiance tile; the taps are then read from shared
// memory. Otherwise (large motion spread) the taps are read from global memory.
// `bar` is the CTA's mbarrier (count 1) and `phase` its current phase. Returns false if the
// bounded wait for the copy gave up (the error word is set; the caller must return).
template <class SV>
__device__ __forceinline__ bool update_tile(UpdateSmem<SV>& sm, uint64_t* bar, uint32_t& phase, int* err,
                                           const KParams& kp, const int W, const int H,
                                           const bool reset, const bool stage_ok, const SV& prev,
                                           const SV& next, const StageMaps* maps,
                                           const float* __restrict__ rad,
                                           const float* __restrict__ mot, const int bx0,
                                           const int by0) {
  const int tx = threadIdx.x % kTW, ty = threadIdx.x / kTW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t npix = (size_t)W * H;
  const int x = bx0 + tx, y = by0 + ty;
  const bool inside = x < W && y < H;
  const size_t j = (size_t)y * W + x;
  __syncthreads();  // the previous tile is done with shared memory

  // reprojection q = pi(v_j) = j + v_j (Table 2), in binary32
  float qx = 0.0f, qy = 0.0f;
  bool valid = false;
  if (inside) {
    qx = (float)x + __ldg(mot + j);
    qy = (float)y + __ldg(mot + npix + j);
    valid = !reset && qx >= 0.0f && qx <= (float)(W - 1) && qy >= 0.0f && qy <= (float)(H - 1);
  }
  int lo_x = 0x7fffffff, hi_x = -1, lo_y = 0x7fffffff, hi_y = -1;
  if (valid) {
    const int x0 = (int)floorf(qx), y0 = (int)floorf(qy);
    lo_x = x0; hi_x = min(x0 + 1, W - 1);
    lo_y = y0; hi_y = min(y0 + 1, H - 1);
  }
  // taps of weight exactly 0, decided per warp (one tile row) so that each branch stays
  // straight-line code: a warp whose valid pixels all have an integral motion component in y
  // (and x), as under a static camera or an axis-aligned pan, reads 2 (1) taps instead of 4
  const bool fy0 = __all_sync(0xffffffffu, !valid || qy == floorf(qy));
  const bool fx0 = __all_sync(0xffffffffu, !valid || qx == floorf(qx));
  lo_x = __reduce_min_sync(0xffffffffu, lo_x);
  hi_x = __reduce_max_sync(0xffffffffu, hi_x);
  lo_y = __reduce_min_sync(0xffffffffu, lo_y);
  hi_y = __reduce_max_sync(0xffffffffu, hi_y);
  if (lane == 0) {
    sm.red[warp][0] = lo_x; sm.red[warp][1] = hi_x; sm.red[warp][2] = lo_y; sm.red[warp][3] = hi_y;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 1; w < kTileThreads / 32; ++w) {
      lo_x = min(lo_x, sm.red[w][0]); hi_x = max(hi_x, sm.red[w][1]);
      lo_y = min(lo_y, sm.red[w][2]); hi_y = max(hi_y, sm.red[w][3]);
    }
    int fits = 0, X0 = 0, Y0 = 0;
    if (stage_ok && hi_x >= 0) {
      X0 = lo_x - lo_x % SV::kAlignX;  // TMA box origin: 16-byte aligned column
      Y0 = lo_y;
      fits = (hi_x - X0 < kStageW) && (hi_y - Y0 < kStageH);
    }
    sm.box[0] = X0; sm.box[1] = Y0; sm.box[2] = fits;
    if (fits) {
      fence_proxy_async();
      mbar_expect_tx(bar, SV::kTxBytes);
      if (!kp.debug_withhold_copy) tma_load_3d(sm.stage, &maps->planes, X0, Y0, 0, bar);
    }
  }
  // radiance tile with a 1-pixel halo; a missing sample (a non-finite channel) and a pixel
  // outside the image are stored as (NaN, NaN, NaN): fminf/fmaxf ignore NaN operands, so the
  // clamp box below skips them without a test per neighbour
  for (int i = threadIdx.x; i < (kTH + 2) * (kTW + 2); i += kTileThreads) {
    const int ly = i / (kTW + 2), lx = i % (kTW + 2);
    const int gx = bx0 - 1 + lx, gy = by0 - 1 + ly;
    const float nan = __int_as_float(0x7fc00000);
    float r = nan, g = nan, b = nan;
    if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
      const size_t jj = (size_t)gy * W + gx;
      r = __ldg(rad + jj);
      g = __ldg(rad + npix + jj);
      b = __ldg(rad + 2 * npix + jj);
      if (!(isfinite(r) && isfinite(g) && isfinite(b))) r = g = b = nan;
    }
    sm.rad[0][ly][lx] = r;
    sm.rad[1][ly][lx] = g;
    sm.rad[2][ly][lx] = b;
  }
  __syncthreads();
  const int X0 = sm.box[0], Y0 = sm.box[1];
  const bool fits = sm.box[2] != 0;
  bool ok = true;
  if (fits) ok = mbar_wait_bounded(bar, phase);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicExch(err, (int)WRLS_ERR_TIMEOUT);
    mbar_wait_bounded(bar, phase);  // the copy may still be in flight
    return false;
  }
  if (fits) phase ^= 1u;
  if (!inside) return true;

  float I[3] = {sm.rad[0][ty + 1][tx + 1], sm.rad[1][ty + 1][tx + 1], sm.rad[2][ty + 1][tx + 1]};
  const bool missing = I[0] != I[0];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
  for (int dy = 0; dy < 3; ++dy)
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float v = sm.rad[c][ty + dy][tx + dx];
        lo[c] = fminf(lo[c], v);
        hi[c] = fmaxf(hi[c], v);
      }
    }
  const bool have_box = lo[0] <= hi[0];  // some neighbour (possibly the pixel itself) was present
  float st[kNState];
  if (valid) {
    if (fits) {
      if (fy0 && fx0) gather_bilinear_staged<SV, 1>(sm.stage, X0, Y0, W, H, qx, qy, st);
      else if (fy0) gather_bilinear_staged<SV, 2>(sm.stage, X0, Y0, W, H, qx, qy, st);
      else gather_bilinear_staged<SV, 4>(sm.stage, X0, Y0, W, H, qx, qy, st);
    }
    else gather_bilinear(prev, W, H, qx, qy, st);
  }
  update_pixel(kp, valid, st, I, missing, lo, hi, have_box);
  next.store((size_t)y * next.pitch + x, st);
  return true;
}

// 128-byte aligned view of a dynamic shared-memory buffer.
__device__ __forceinline__ unsigned char* align128(unsigned char* p) {
  return p + ((128u - (smem_u32(p) & 127u)) & 127u);
}

// ---- spatio-temporal blend (Sec. 5.3) -------------------------------------------------------
//
// A blend tile is 32 x TH output pixels; each thread produces R vertically adjacent outputs of
// one column, so a neighbour read from shared memory serves up to 5 of the thread's outputs.
// Shared memory holds the (32+4) x (TH+4) window of the models after the update as two record
// arrays: beta[12] per pixel (48-byte stride) and {z[3], rk} per pixel (16 bytes), with
// rk = K / (|z|+eps)^2 and K = log2(e) / h_s^2; both strides make a warp's 128-bit loads
// conflict-free. With r = 1/(|z|+eps), the range exponent of a pair is
// |z_i - z_k|^2 max(r_i, r_k)^2 K = |z_i - z_k|^2 max(rk_i, rk_k).
//
// No neighbour is tested in the inner loop. A window pixel outside the image gets beta = 0,
// z = kFarZ and rk = 0, so its feature distance to any pixel of the image is huge and its
// weight exp2(-huge) is exactly 0; offsets beyond the window radius (radius < 2) get a
// spatial exponent of -inf, weight exactly 0. Adding exact zeros leaves every sum unchanged,
// so the result equals skipping those neighbours.
constexpr int kBlendSW = kTW + 2 * kMaxRadius;
constexpr float kFarZ = 1.0e18f;

template <int TH>
struct BlendGeom {
  static constexpr int SH = TH + 2 * kMaxRadius;
  static constexpr int kPix = SH * kBlendSW;
  static constexpr int kSmemBytes = kPix * (48 + 16);
};

// Fill the shared window of the blend tile at (bx0, by0) from the state copy `cur`.
template <class SV, int TH, int NT, int UNROLL = 4>
__device__ __forceinline__ void blend_fill(float4* __restrict__ sb, float4* __restrict__ szr,
                                           const KParams& kp, const int W, const int H, const SV& cur,
                                           const int bx0, const int by0) {
  constexpr int R0 = kMaxRadius;
#pragma unroll UNROLL
  for (int i = threadIdx.x; i < BlendGeom<TH>::kPix; i += NT) {
    const int ly = i / kBlendSW, lx = i % kBlendSW;
    const int gx = bx0 - R0 + lx, gy = by0 - R0 + ly;
    if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
      float b[12], z[3];
      cur.load_beta_z((size_t)gy * cur.pitch + gx, b, z);
      sb[3 * i + 0] = make_float4(b[0], b[1], b[2], b[3]);
      sb[3 * i + 1] = make_float4(b[4], b[5], b[6], b[7]);
      sb[3 * i + 2] = make_float4(b[8], b[9], b[10], b[11]);
      szr[i] = make_float4(z[0], z[1], z[2], blend_rk(z[0], z[1], z[2], kp.eps, kp.range_k));
    } else {
      const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      sb[3 * i + 0] = zero;
      sb[3 * i + 1] = zero;
      sb[3 * i + 2] = zero;
      szr[i] = make_float4(kFarZ, kFarZ, kFarZ, 0.0f);
    }
  }
}

// Blend the outputs of the tile whose window is in shared memory. MODE 0: out_i = sum_k b_ik
// (p_i . beta_k) / sum_k b_ik (neighbours' models predict pixel i; cross_pred per pair, three
// accumulators per output); MODE 1: sum_k b_ik (p_k . beta_k) / sum_k b_ik. b_ik = exp(-|dxy|^2 / (2 sigma_s^2)) exp(-d_z(i,k)^2 / h_s^2) with d_z the
// Eq. 13 distance of the features; 1 / (min(|z_i|, |z_k|) + eps) = max(r_i, r_k), computed in
// base 2 as exp2(spatial - |z_i - z_k|^2 max(rk_i, rk_k)).
template <int TH, int R, int MODE>
__device__ __forceinline__ void blend_compute(const float4* __restrict__ sb,
                                              const float4* __restrict__ szr, const KParams& kp,
                                              const int W, const int H, float* __restrict__ out,
                                              const int bx0, const int by0) {
  constexpr int R0 = kMaxRadius;
  constexpr int RW = 2 * R0 + 1;
  const int tx = threadIdx.x % kTW, ty = threadIdx.x / kTW;
  const int x = bx0 + tx, y0 = by0 + ty * R;
  const bool feat = kp.feature_mode == 0;
  float zi[R][3], pf[R][3], ri[R], den[R], acc[R][3];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const float4 q = szr[(ty * R + i + R0) * kBlendSW + tx + R0];
    zi[i][0] = q.x; zi[i][1] = q.y; zi[i][2] = q.z; ri[i] = q.w;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pf[i][c] = feat ? zi[i][c] : 0.0f;  // feature entries of p_i
      acc[i][c] = 0.0f;
    }
    den[i] = 0.0f;
  }
#pragma unroll
  for (int kr = 0; kr < R + 2 * R0; ++kr) {
#pragma unroll
    for (int dx = -R0; dx <= R0; ++dx) {
      const int k = (ty * R + kr) * kBlendSW + tx + R0 + dx;
      const float4 q3 = szr[k];
      const float4 q0 = sb[3 * k + 0], q1 = sb[3 * k + 1], q2 = sb[3 * k + 2];
      float pk0 = 0.0f, pk1 = 0.0f, pk2 = 0.0f;
      if (MODE == 1) {
        const float a1 = feat ? q3.x : 0.0f, a2 = feat ? q3.y : 0.0f, a3 = feat ? q3.z : 0.0f;
        pk0 = cross_pred(q0.x, q0.y, q0.z, q0.w, a1, a2, a3);
        pk1 = cross_pred(q1.x, q1.y, q1.z, q1.w, a1, a2, a3);
        pk2 = cross_pred(q2.x, q2.y, q2.z, q2.w, a1, a2, a3);
      }
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int dy = kr - R0 - i;
        if (dy < -R0 || dy > R0) continue;  // compile-time
        const float e0 = zi[i][0] - q3.x, e1 = zi[i][1] - q3.y, e2 = zi[i][2] - q3.z;
        const float rk = fmaxf(ri[i], q3.w);  // K / (min(|z_i|, |z_k|) + eps)^2
        const float b = ex2_approx(blend_exponent(kp.spatial[(dy + R0) * RW + (dx + R0)], e0, e1, e2, rk));
        den[i] += b;
        if (MODE == 0) {
          pk0 = cross_pred(q0.x, q0.y, q0.z, q0.w, pf[i][0], pf[i][1], pf[i][2]);
          pk1 = cross_pred(q1.x, q1.y, q1.z, q1.w, pf[i][0], pf[i][1], pf[i][2]);
          pk2 = cross_pred(q2.x, q2.y, q2.z, q2.w, pf[i][0], pf[i][1], pf[i][2]);
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

// Whole blend tile: barrier, fill, barrier, compute (a CTA may run tiles back to back).
// `smem` is 16-byte aligned and holds BlendGeom<TH>::kSmemBytes.
template <class SV, int TH, int R, int MODE>
__device__ __forceinline__ void blend_tile(float4* __restrict__ smem, const KParams& kp, const int W,
                                           const int H, const SV& cur, float* __restrict__ out,
                                           const int bx0, const int by0) {
  float4* sb = smem;
  float4* szr = smem + 3 * BlendGeom<TH>::kPix;
  __syncthreads();
  blend_fill<SV, TH, kTW * TH / R>(sb, szr, kp, W, H, cur, bx0, by0);
  __syncthreads();
  blend_compute<TH, R, MODE>(sb, szr, kp, W, H, out, bx0, by0);
}

}  // namespace wrls
