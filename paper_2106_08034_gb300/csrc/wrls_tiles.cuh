// Tile bodies of the wRLS denoiser, shared by the single-frame kernels (one CTA per
// tile) and the persistent batched kernel (each CTA loops over work items).
//
//  update_tile : per pixel, reprojection + Eq. 12 + Eq. 13 + Eq. 8/14/9/11 (Sec. 5.2-5.3);
//                reads the previous state copy, writes the new one.
//  blend_tile  : per pixel, the spatio-temporal blend of Sec. 5.3 over the (2r+1)^2 window
//                of models after the update; writes the denoised colour.
//
// Tiles are 32 x 8 pixels (one warp per tile row: each plane access of a warp is one
// 128-byte row segment). The 3x3 neighbourhood of the radiance (clamp of Eq. 12) and the
// 5x5 neighbourhood of beta/z (blend) are staged in shared memory with their halos;
// out-of-image halo pixels are marked (NaN radiance, negative 1/|z|) and skipped.
// Both bodies start and end with a CTA barrier so a CTA may run them back to back.
#pragma once
#include "wrls_device.cuh"

namespace wrls {

constexpr int kTW = 32;
constexpr int kTH = 8;
constexpr int kTileThreads = kTW * kTH;

struct UpdateSmem {
  float rad[3][kTH + 2][kTW + 2];
};

struct BlendSmem {
  static constexpr int SW = kTW + 2 * kMaxRadius, SH = kTH + 2 * kMaxRadius;
  float b[12][SH][SW];
  float z[3][SH][SW];
  float r[SH][SW];
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

template <class SV>
__device__ __forceinline__ void blend_tile(BlendSmem& sm, const KParams& kp, const int W,
                                           const int H, const SV& cur, float* __restrict__ out,
                                           const int bx0, const int by0) {
  constexpr int R = kMaxRadius;
  constexpr int SW = BlendSmem::SW, SH = BlendSmem::SH;
  const int tx = threadIdx.x % kTW, ty = threadIdx.x / kTW;
  __syncthreads();
  for (int i = threadIdx.x; i < SH * SW; i += kTileThreads) {
    const int ly = i / SW, lx = i % SW;
    const int gx = bx0 - R + lx, gy = by0 - R + ly;
    if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
      float b[12], z[3];
      cur.load_beta_z((size_t)gy * cur.pitch + gx, b, z);
#pragma unroll
      for (int p = 0; p < 12; ++p) sm.b[p][ly][lx] = b[p];
#pragma unroll
      for (int c = 0; c < 3; ++c) sm.z[c][ly][lx] = z[c];
      sm.r[ly][lx] = 1.0f / (sqrtf(z[0] * z[0] + z[1] * z[1] + z[2] * z[2]) + kp.eps);
    } else {
      sm.r[ly][lx] = -1.0f;
    }
  }
  __syncthreads();
  const int x = bx0 + tx, y = by0 + ty;
  if (x < W && y < H) {
    const int cy = ty + R, cx = tx + R;
    const float zi0 = sm.z[0][cy][cx], zi1 = sm.z[1][cy][cx], zi2 = sm.z[2][cy][cx];
    const float ri = sm.r[cy][cx];
    const bool feat = kp.feature_mode == 0;
    const float p1 = feat ? zi0 : 0.0f, p2 = feat ? zi1 : 0.0f, p3 = feat ? zi2 : 0.0f;
    const int r = kp.radius;
    float acc[12];
#pragma unroll
    for (int p = 0; p < 12; ++p) acc[p] = 0.0f;
    float num0 = 0.0f, num1 = 0.0f, num2 = 0.0f, den = 0.0f;
    for (int dy = -r; dy <= r; ++dy) {
      for (int dx = -r; dx <= r; ++dx) {
        const int ky = cy + dy, kx = cx + dx;
        const float rk = sm.r[ky][kx];
        if (rk < 0.0f) continue;
        const float e0 = zi0 - sm.z[0][ky][kx], e1 = zi1 - sm.z[1][ky][kx], e2 = zi2 - sm.z[2][ky][kx];
        const float rm = fmaxf(ri, rk);  // = 1 / (min(|z_i|, |z_k|) + eps)
        const float d2 = (e0 * e0 + e1 * e1 + e2 * e2) * (rm * rm);
        const float b = ex2_approx(kp.spatial[(dy + R) * (2 * R + 1) + (dx + R)] - d2 * kp.range_k);
        den += b;
        if (kp.blend_mode == 0) {
#pragma unroll
          for (int p = 0; p < 12; ++p) acc[p] += b * sm.b[p][ky][kx];
        } else {
          const float q1 = feat ? sm.z[0][ky][kx] : 0.0f, q2 = feat ? sm.z[1][ky][kx] : 0.0f,
                      q3 = feat ? sm.z[2][ky][kx] : 0.0f;
          num0 += b * (sm.b[0][ky][kx] + sm.b[1][ky][kx] * q1 + sm.b[2][ky][kx] * q2 + sm.b[3][ky][kx] * q3);
          num1 += b * (sm.b[4][ky][kx] + sm.b[5][ky][kx] * q1 + sm.b[6][ky][kx] * q2 + sm.b[7][ky][kx] * q3);
          num2 += b * (sm.b[8][ky][kx] + sm.b[9][ky][kx] * q1 + sm.b[10][ky][kx] * q2 + sm.b[11][ky][kx] * q3);
        }
      }
    }
    if (kp.blend_mode == 0) {
      // sum_k b_k (p_i . beta_k) = p_i . sum_k b_k beta_k
      num0 = acc[0] + acc[1] * p1 + acc[2] * p2 + acc[3] * p3;
      num1 = acc[4] + acc[5] * p1 + acc[6] * p2 + acc[7] * p3;
      num2 = acc[8] + acc[9] * p1 + acc[10] * p2 + acc[11] * p3;
    }
    const float inv = 1.0f / den;
    const size_t npix = (size_t)W * H, j = (size_t)y * W + x;
    out[j] = num0 * inv;
    out[npix + j] = num1 * inv;
    out[2 * npix + j] = num2 * inv;
  }
}

}  // namespace wrls
