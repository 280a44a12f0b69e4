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
#include "wrls_device.cuh"

namespace wrls {

constexpr int kTW = 32;
constexpr int kTH = 8;
constexpr int kTileThreads = kTW * kTH;

struct UpdateSmem {
  float rad[3][kTH + 2][kTW + 2];
};

template <class SV>
__device__ __forceinline__ void update_tile(UpdateSmem& sm, const KParams& kp, const int W,
                                            const int H, const bool reset, const SV& prev,
                                            const SV& next, const float* __restrict__ rad,
                                            const float* __restrict__ mot, const int bx0,
                                            const int by0) {
  const int tx = threadIdx.x % kTW, ty = threadIdx.x / kTW;
  const size_t npix = (size_t)W * H;
  __syncthreads();
  for (int i = threadIdx.x; i < (kTH + 2) * (kTW + 2); i += kTileThreads) {
    const int ly = i / (kTW + 2), lx = i % (kTW + 2);
    const int gx = bx0 - 1 + lx, gy = by0 - 1 + ly;
    float r = __int_as_float(0x7fc00000), g = r, b = r;
    if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
      const size_t j = (size_t)gy * W + gx;
      r = __ldg(rad + j);
      g = __ldg(rad + npix + j);
      b = __ldg(rad + 2 * npix + j);
    }
    sm.rad[0][ly][lx] = r;
    sm.rad[1][ly][lx] = g;
    sm.rad[2][ly][lx] = b;
  }
  __syncthreads();
  const int x = bx0 + tx, y = by0 + ty;
  if (x < W && y < H) {
    const size_t j = (size_t)y * W + x;
    float I[3] = {sm.rad[0][ty + 1][tx + 1], sm.rad[1][ty + 1][tx + 1], sm.rad[2][ty + 1][tx + 1]};
    const bool missing = !(isfinite(I[0]) && isfinite(I[1]) && isfinite(I[2]));
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool have_box = false;
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const float a = sm.rad[0][ty + dy][tx + dx], b = sm.rad[1][ty + dy][tx + dx],
                    c = sm.rad[2][ty + dy][tx + dx];
        if (isfinite(a) && isfinite(b) && isfinite(c)) {
          have_box = true;
          lo[0] = fminf(lo[0], a); hi[0] = fmaxf(hi[0], a);
          lo[1] = fminf(lo[1], b); hi[1] = fmaxf(hi[1], b);
          lo[2] = fminf(lo[2], c); hi[2] = fmaxf(hi[2], c);
        }
      }
    // reprojection q = pi(v_j) = j + v_j (Table 2), in binary32
    const float qx = (float)x + __ldg(mot + j);
    const float qy = (float)y + __ldg(mot + npix + j);
    const bool valid = !reset && qx >= 0.0f && qx <= (float)(W - 1) && qy >= 0.0f &&
                       qy <= (float)(H - 1);
    float st[kNState];
    if (valid) gather_bilinear(prev, W, H, qx, qy, st);
    update_pixel(kp, valid, st, I, missing, lo, hi, have_box);
    next.store((size_t)y * next.pitch + x, st);
  }
}

// ---- spatio-temporal blend (Sec. 5.3) -------------------------------------------------------
//
// A blend tile is 32 x TH output pixels; each thread produces R vertically adjacent outputs of
// one column, so a neighbour read from shared memory serves up to 5 of the thread's outputs.
// Shared memory holds the (32+4) x (TH+4) window of the models after the update, one 20-float
// record per pixel: beta[12], z[3], 1/(|z|+eps) (negative = outside the image), 4 pad floats.
// The 80-byte record stride makes the four 128-bit loads of a warp conflict-free.
constexpr int kBlendRec = 20;
constexpr int kBlendSW = kTW + 2 * kMaxRadius;

template <int TH>
struct BlendGeom {
  static constexpr int SH = TH + 2 * kMaxRadius;
  static constexpr int kSmemBytes = SH * kBlendSW * kBlendRec * 4;
};

// Fill the shared window of the blend tile at (bx0, by0) from the state copy `cur`.
template <class SV, int TH, int NT>
__device__ __forceinline__ void blend_fill(float4* __restrict__ sm, const KParams& kp, const int W,
                                           const int H, const SV& cur, const int bx0, const int by0) {
  constexpr int R0 = kMaxRadius, SH = BlendGeom<TH>::SH;
#pragma unroll 2
  for (int i = threadIdx.x; i < SH * kBlendSW; i += NT) {
    const int ly = i / kBlendSW, lx = i % kBlendSW;
    const int gx = bx0 - R0 + lx, gy = by0 - R0 + ly;
    float4* rec = sm + i * (kBlendRec / 4);
    if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
      float b[12], z[3];
      cur.load_beta_z((size_t)gy * cur.pitch + gx, b, z);
      const float r = 1.0f / (sqrtf(z[0] * z[0] + z[1] * z[1] + z[2] * z[2]) + kp.eps);
      rec[0] = make_float4(b[0], b[1], b[2], b[3]);
      rec[1] = make_float4(b[4], b[5], b[6], b[7]);
      rec[2] = make_float4(b[8], b[9], b[10], b[11]);
      rec[3] = make_float4(z[0], z[1], z[2], r);
    } else {
      rec[3] = make_float4(0.0f, 0.0f, 0.0f, -1.0f);
    }
  }
}

// Blend the outputs of the tile whose window is in `sm`. MODE 0: out_i = sum_k b_ik (p_i .
// beta_k) / sum_k b_ik (neighbours' models predict pixel i); MODE 1: sum_k b_ik (p_k . beta_k)
// / sum_k b_ik. b_ik = exp(-|dxy|^2 / (2 sigma_s^2)) exp(-d_z(i,k)^2 / h_s^2) with d_z the
// Eq. 13 distance of the features; 1 / (min(|z_i|, |z_k|) + eps) = max(r_i, r_k).
template <int TH, int R, int MODE>
__device__ __forceinline__ void blend_compute(const float4* __restrict__ sm, const KParams& kp,
                                              const int W, const int H, float* __restrict__ out,
                                              const int bx0, const int by0) {
  constexpr int R0 = kMaxRadius;
  constexpr int RW = 2 * R0 + 1;
  const int tx = threadIdx.x % kTW, ty = threadIdx.x / kTW;
  const int x = bx0 + tx, y0 = by0 + ty * R;
  const int rad = kp.radius;
  const bool feat = kp.feature_mode == 0;
  float zi[R][3], ri[R], den[R];
  float acc[R][MODE == 0 ? 12 : 3];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const float4 q = sm[((ty * R + i + R0) * kBlendSW + tx + R0) * (kBlendRec / 4) + 3];
    zi[i][0] = q.x; zi[i][1] = q.y; zi[i][2] = q.z; ri[i] = q.w;
    den[i] = 0.0f;
#pragma unroll
    for (int p = 0; p < (MODE == 0 ? 12 : 3); ++p) acc[i][p] = 0.0f;
  }
#pragma unroll
  for (int kr = 0; kr < R + 2 * R0; ++kr) {
#pragma unroll
    for (int dx = -R0; dx <= R0; ++dx) {
      if (dx < -rad || dx > rad) continue;
      const float4* rec = sm + ((ty * R + kr) * kBlendSW + tx + R0 + dx) * (kBlendRec / 4);
      const float4 q3 = rec[3];
      if (q3.w < 0.0f) continue;
      const float4 q0 = rec[0], q1 = rec[1], q2 = rec[2];
      float pk0 = 0.0f, pk1 = 0.0f, pk2 = 0.0f;
      if (MODE == 1) {
        const float a1 = feat ? q3.x : 0.0f, a2 = feat ? q3.y : 0.0f, a3 = feat ? q3.z : 0.0f;
        pk0 = q0.x + q0.y * a1 + q0.z * a2 + q0.w * a3;
        pk1 = q1.x + q1.y * a1 + q1.z * a2 + q1.w * a3;
        pk2 = q2.x + q2.y * a1 + q2.z * a2 + q2.w * a3;
      }
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int dy = kr - R0 - i;
        if (dy < -R0 || dy > R0) continue;
        if (dy < -rad || dy > rad) continue;
        const float e0 = zi[i][0] - q3.x, e1 = zi[i][1] - q3.y, e2 = zi[i][2] - q3.z;
        const float rm = fmaxf(ri[i], q3.w);
        const float d2 = (e0 * e0 + e1 * e1 + e2 * e2) * (rm * rm);
        const float b = ex2_approx(kp.spatial[(dy + R0) * RW + (dx + R0)] - d2 * kp.range_k);
        den[i] += b;
        if (MODE == 0) {
          acc[i][0] += b * q0.x; acc[i][1] += b * q0.y; acc[i][2] += b * q0.z; acc[i][3] += b * q0.w;
          acc[i][4] += b * q1.x; acc[i][5] += b * q1.y; acc[i][6] += b * q1.z; acc[i][7] += b * q1.w;
          acc[i][8] += b * q2.x; acc[i][9] += b * q2.y; acc[i][10] += b * q2.z; acc[i][11] += b * q2.w;
        } else {
          acc[i][0] += b * pk0; acc[i][1] += b * pk1; acc[i][2] += b * pk2;
        }
      }
    }
  }
  if (x >= W) return;
  const size_t npix = (size_t)W * H;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int y = y0 + i;
    if (y >= H) break;
    float o0, o1, o2;
    if (MODE == 0) {
      // sum_k b_k (p_i . beta_k) = p_i . sum_k b_k beta_k, p_i = [1, z_i]
      const float p1 = feat ? zi[i][0] : 0.0f, p2 = feat ? zi[i][1] : 0.0f, p3 = feat ? zi[i][2] : 0.0f;
      o0 = acc[i][0] + acc[i][1] * p1 + acc[i][2] * p2 + acc[i][3] * p3;
      o1 = acc[i][4] + acc[i][5] * p1 + acc[i][6] * p2 + acc[i][7] * p3;
      o2 = acc[i][8] + acc[i][9] * p1 + acc[i][10] * p2 + acc[i][11] * p3;
    } else {
      o0 = acc[i][0]; o1 = acc[i][1]; o2 = acc[i][2];
    }
    const float inv = 1.0f / den[i];
    const size_t j = (size_t)y * W + x;
    out[j] = o0 * inv;
    out[npix + j] = o1 * inv;
    out[2 * npix + j] = o2 * inv;
  }
}

// Whole blend tile: barrier, fill, barrier, compute (a CTA may run tiles back to back).
template <class SV, int TH, int R, int MODE>
__device__ __forceinline__ void blend_tile(float4* __restrict__ sm, const KParams& kp, const int W,
                                           const int H, const SV& cur, float* __restrict__ out,
                                           const int bx0, const int by0) {
  __syncthreads();
  blend_fill<SV, TH, kTW * TH / R>(sm, kp, W, H, cur, bx0, by0);
  __syncthreads();
  blend_compute<TH, R, MODE>(sm, kp, W, H, out, bx0, by0);
}

}  // namespace wrls
