// The denoiser's per-frame inputs from the renderer's raw data:
//   k_reconstruct : pixel reconstruction filter (Sec. 4, Table 2: the samples f_j of a pixel
//                   are filtered into I~_j; Sec. 6: separable Gaussian kernel), plus the
//                   variance of each pixel's sample mean;
//   k_velocity    : per-pixel backward motion from the first-collision world position
//                   (Sec. 5.3; Sec. 6 "Optical flow estimation"), projected with the previous
//                   frame's view-projection matrix.
#include <math.h>
#include <string.h>

#include "wrls_internal.h"

namespace wrls {

constexpr int kRecTW = 32, kRecTH = 8;
constexpr int kRecSW = kRecTW + 2, kRecSH = kRecTH + 2, kRecSP = kRecSW * kRecSH;

struct ReconArgs {
  float k2;      // log2(e) / (2 sigma^2): g(dx) g(dy) = 2^(-(dx^2 + dy^2) k2)
  float radius;  // support: |dx|, |dy| <= radius (binary32)
};

// I~_j = sum_k g(x_k - x_j) g(y_k - y_j) f_k / sum_k g g over the samples of the 3x3 pixels
// around j. Samples: ((s * 5 + k) * H + y) * W + x, k = r, g, b, ox, oy. One CTA per 32 x 8
// tile; the 34 x 10 windows of up to kRecChunk sample indices at a time are staged in shared
// memory (one barrier pair per chunk). A sample with a non-finite colour or offset, or
// outside the image, is staged with an infinite offset, which no support contains.
constexpr int kRecChunk = 4;

__global__ void __launch_bounds__(kRecTW * kRecTH)
    k_reconstruct(const ReconArgs a, const int W, const int H, const int spp, const float* __restrict__ smp,
                  float* __restrict__ out, float* __restrict__ var) {
  __shared__ float sm[kRecChunk][5][kRecSP];
  const int bx0 = blockIdx.x * kRecTW, by0 = blockIdx.y * kRecTH;
  const int tid = threadIdx.y * kRecTW + threadIdx.x;
  const int x = bx0 + threadIdx.x, y = by0 + threadIdx.y;
  const size_t np = (size_t)W * H;
  const bool inside = x < W && y < H;
  float n0 = 0.0f, n1 = 0.0f, n2 = 0.0f, den = 0.0f;
  // own samples, shifted by the first valid one (k): sums and sum of squares
  float k0 = 0.0f, k1 = 0.0f, k2 = 0.0f, m0 = 0.0f, m1 = 0.0f, m2 = 0.0f, q = 0.0f;
  int cnt = 0;
  for (int s0 = 0; s0 < spp; s0 += kRecChunk) {
    const int ns = min(kRecChunk, spp - s0);
    for (int e = tid; e < kRecSP * ns; e += kRecTW * kRecTH) {
      const int c = e / kRecSP, ew = e - c * kRecSP;
      const int gx = bx0 - 1 + ew % kRecSW, gy = by0 - 1 + ew / kRecSW;
      float r = 0.0f, g = 0.0f, b = 0.0f, ox = INFINITY, oy = INFINITY;
      if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
        const float* base = smp + (size_t)(s0 + c) * 5 * np + (size_t)gy * W + gx;
        r = __ldg(base);
        g = __ldg(base + np);
        b = __ldg(base + 2 * np);
        ox = __ldg(base + 3 * np);
        oy = __ldg(base + 4 * np);
        if (!(isfinite(r) && isfinite(g) && isfinite(b) && isfinite(ox) && isfinite(oy))) {
          r = g = b = 0.0f;
          ox = oy = INFINITY;
        }
      }
      sm[c][0][ew] = r;
      sm[c][1][ew] = g;
      sm[c][2][ew] = b;
      sm[c][3][ew] = ox;
      sm[c][4][ew] = oy;
    }
    __syncthreads();
    if (inside) {
      const int ec = (threadIdx.y + 1) * kRecSW + threadIdx.x + 1;
      for (int c = 0; c < ns; ++c) {
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) {
            const int e = ec + dy * kRecSW + dx;
            const float ux = (float)dx + sm[c][3][e], uy = (float)dy + sm[c][4][e];
            const float w = (fabsf(ux) <= a.radius && fabsf(uy) <= a.radius)
                                ? ex2_approx(-(ux * ux + uy * uy) * a.k2) : 0.0f;
            n0 = fmaf(w, sm[c][0][e], n0);
            n1 = fmaf(w, sm[c][1][e], n1);
            n2 = fmaf(w, sm[c][2][e], n2);
            den += w;
          }
        if (var && isfinite(sm[c][3][ec])) {  // own sample is valid
          if (cnt == 0) {
            k0 = sm[c][0][ec];
            k1 = sm[c][1][ec];
            k2 = sm[c][2][ec];
          }
          const float r = sm[c][0][ec] - k0, g = sm[c][1][ec] - k1, b = sm[c][2][ec] - k2;
          m0 += r;
          m1 += g;
          m2 += b;
          q = fmaf(r, r, fmaf(g, g, fmaf(b, b, q)));
          ++cnt;
        }
      }
    }
    __syncthreads();
  }
  if (!inside) return;
  const size_t j = (size_t)y * W + x;
  const float inv = den > 0.0f ? 1.0f / den : __int_as_float(0x7fc00000);
  out[j] = n0 * inv;
  out[np + j] = n1 * inv;
  out[2 * np + j] = n2 * inv;
  if (var) {
    if (cnt < 2) {
      var[j] = __int_as_float(0x7fc00000);
    } else {
      // sum over channels of sum_s (f - mean)^2 = sum u^2 - (sum u)^2 / n, u = f - k
      const float fn = (float)cnt;
      const float ss = q - (m0 * m0 + m1 * m1 + m2 * m2) / fn;
      var[j] = fmaxf(ss, 0.0f) / (3.0f * (fn - 1.0f)) / fn;
    }
  }
}

struct Mat4 {
  float m[16];
};

__global__ void k_velocity(const Mat4 M, const int W, const int H, const int miss_policy,
                           const float* __restrict__ world, float* __restrict__ mot) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W || y >= H) return;
  const size_t np = (size_t)W * H, j = (size_t)y * W + x;
  const float X = __ldg(world + j), Y = __ldg(world + np + j), Z = __ldg(world + 2 * np + j);
  const float nan = __int_as_float(0x7fc00000);
  float vx, vy;
  if (!(isfinite(X) && isfinite(Y) && isfinite(Z))) {
    vx = vy = miss_policy == 0 ? 0.0f : nan;
  } else {
    const float cw = fmaf(M.m[12], X, fmaf(M.m[13], Y, fmaf(M.m[14], Z, M.m[15])));
    if (!(cw > 0.0f)) {
      vx = vy = nan;
    } else {
      const float cx = fmaf(M.m[0], X, fmaf(M.m[1], Y, fmaf(M.m[2], Z, M.m[3])));
      const float cy = fmaf(M.m[4], X, fmaf(M.m[5], Y, fmaf(M.m[6], Z, M.m[7])));
      const float iw = 1.0f / cw;
      vx = fmaf(cx * iw + 1.0f, 0.5f * (float)W, -0.5f) - (float)x;
      vy = fmaf(1.0f - cy * iw, 0.5f * (float)H, -0.5f) - (float)y;
    }
  }
  mot[j] = vx;
  mot[np + j] = vy;
}

}  // namespace wrls

using namespace wrls;

static bool in_range(int w, int h) { return w >= 1 && h >= 1 && w <= 16384 && h <= 16384; }

static bool overlap_bytes(const void* a, size_t an, const void* b, size_t bn) {
  if (!a || !b) return false;
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x < y + bn && y < x + an;
}

extern "C" {

void wrls_recon_params_default(wrls_recon_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->struct_size = sizeof(wrls_recon_params);
  p->sigma = 0.5f;
  p->radius = 1.5f;
}

wrls_status wrls_reconstruct(int width, int height, int spp, const float* samples, const wrls_recon_params* p,
                             float* radiance, float* variance, void* cuda_stream) {
  NvtxRange nvtx("wrls_reconstruct");
  if (!p || p->struct_size != sizeof(wrls_recon_params)) {
    set_error("wrls_reconstruct: params NULL or struct_size != sizeof(wrls_recon_params)");
    return WRLS_ERR_INVALID_ARG;
  }
  if (!in_range(width, height) || spp < 1 || spp > 1024 || !samples || !radiance) {
    set_error("wrls_reconstruct: bad size (%d x %d, spp %d) or NULL samples/radiance", width, height, spp);
    return WRLS_ERR_INVALID_ARG;
  }
  if (!(p->sigma > 0.0f) || !(p->radius > 0.0f && p->radius <= 1.5f)) {
    set_error("wrls_reconstruct: sigma must be > 0 and radius in (0, 1.5]");
    return WRLS_ERR_INVALID_ARG;
  }
  if (((uintptr_t)samples | (uintptr_t)radiance | (uintptr_t)variance) & 3u) {
    set_error("wrls_reconstruct: buffers must be 4-byte aligned");
    return WRLS_ERR_INVALID_ARG;
  }
  const size_t np = (size_t)width * height;
  if (overlap_bytes(radiance, 12 * np, samples, 20 * np * spp) || overlap_bytes(variance, 4 * np, samples, 20 * np * spp) ||
      overlap_bytes(radiance, 12 * np, variance, 4 * np)) {
    set_error("wrls_reconstruct: outputs overlap each other or the samples");
    return WRLS_ERR_INVALID_ARG;
  }
  ReconArgs a;
  a.k2 = (float)(1.4426950408889634 / (2.0 * (double)p->sigma * (double)p->sigma));
  a.radius = p->radius;
  const dim3 grid((width + kRecTW - 1) / kRecTW, (height + kRecTH - 1) / kRecTH), block(kRecTW, kRecTH);
  k_reconstruct<<<grid, block, 0, (cudaStream_t)cuda_stream>>>(a, width, height, spp, samples, radiance, variance);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("wrls_reconstruct: launch: %s", cudaGetErrorString(e));
    return WRLS_ERR_CUDA;
  }
  return WRLS_OK;
}

wrls_status wrls_velocity_from_world(int width, int height, const float* world, const float* prev_view_proj,
                                     int miss_policy, float* motion, void* cuda_stream) {
  NvtxRange nvtx("wrls_velocity_from_world");
  if (!in_range(width, height) || !world || !prev_view_proj || !motion || miss_policy < 0 || miss_policy > 1) {
    set_error("wrls_velocity_from_world: bad size (%d x %d), NULL pointer or miss_policy %d", width, height,
              miss_policy);
    return WRLS_ERR_INVALID_ARG;
  }
  if (((uintptr_t)world | (uintptr_t)motion) & 3u) {
    set_error("wrls_velocity_from_world: buffers must be 4-byte aligned");
    return WRLS_ERR_INVALID_ARG;
  }
  const size_t np = (size_t)width * height;
  if (overlap_bytes(motion, 8 * np, world, 12 * np)) {
    set_error("wrls_velocity_from_world: motion overlaps world");
    return WRLS_ERR_INVALID_ARG;
  }
  Mat4 M;
  for (int i = 0; i < 16; ++i) {
    if (!isfinite(prev_view_proj[i])) {
      set_error("wrls_velocity_from_world: prev_view_proj[%d] is not finite", i);
      return WRLS_ERR_INVALID_ARG;
    }
    M.m[i] = prev_view_proj[i];
  }
  const dim3 grid((width + 127) / 128, height);
  k_velocity<<<grid, 128, 0, (cudaStream_t)cuda_stream>>>(M, width, height, miss_policy, world, motion);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("wrls_velocity_from_world: launch: %s", cudaGetErrorString(e));
    return WRLS_ERR_CUDA;
  }
  return WRLS_OK;
}

}  // extern "C"
