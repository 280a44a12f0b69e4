// Volumetric path tracer that produces the denoiser's inputs (Sec. 3 and Sec. 6): progressive
// path tracing of a heterogeneous medium, free paths by delta tracking (Eq. 4) with the
// majorant mu_t^max, the collision estimator of Eq. 3 (throughput times mu_s / mu_t at every
// real collision), next-event estimation to a directional light with delta-tracked
// visibility and the isotropic phase function 1 / (4 pi), background radiance for paths that
// leave the volume (Eq. 1), and the first real collision closest to the viewer kept for the
// velocity estimate (Sec. 6). The volume is procedural: Gaussian density blobs in [-1, 1]^3
// behind an opacity ramp and a colour ramp (the transfer function).
//
// One thread per pixel, looping over its samples. Random numbers: Philox4x32-10 (Salmon et
// al., SC 2011), counter (pixel, sample, frame, block), key = the scene seed; each block's four
// words are used in order. Every tracking loop counts toward a cap of 2^20 tentative
// collisions per path.
#include <math.h>
#include <string.h>

#include "wrls_internal.h"

namespace wrls {

constexpr int kVptMaxSteps = 1 << 20;
constexpr float kVptPi = 3.14159265358979f;

struct VptBlob {
  float cx, cy, cz, inv2r2, a;  // density term a exp(-|x - c|^2 inv2r2), inv2r2 = 1 / (2 r^2)
};

struct VptArgs {
  uint32_t key0, key1;
  float eye[3];
  float ivp[16];
  int n_blobs;
  VptBlob blob[16];
  float mu_max, inv_mu_max, tf_lo, inv_tf_span, albedo;
  float col_lo[3], col_span[3];
  float light_dir[3], light_rgb[3], env_rgb[3];
  int max_bounces;
};

struct Philox {
  uint32_t c0, c1, c2, c3, k0, k1;
  uint32_t buf[4];
  int used;
  int steps;

  __device__ __forceinline__ void block() {
    uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = c3, a = k0, b = k1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      if (r > 0) {
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
      }
      const uint32_t hi0 = __umulhi(0xD2511F53u, x0), lo0 = 0xD2511F53u * x0;
      const uint32_t hi1 = __umulhi(0xCD9E8D57u, x2), lo1 = 0xCD9E8D57u * x2;
      const uint32_t n0 = hi1 ^ x1 ^ a, n2 = hi0 ^ x3 ^ b;
      x0 = n0;
      x1 = lo1;
      x2 = n2;
      x3 = lo0;
    }
    buf[0] = x0;
    buf[1] = x1;
    buf[2] = x2;
    buf[3] = x3;
    c3 += 1u;
    used = 0;
  }
  // u in [0, 1): the top 24 bits times 2^-24 (exact in binary32)
  __device__ __forceinline__ float u() {
    if (used == 4) block();
    const uint32_t v = buf[used];
    ++used;
    return (float)(v >> 8) * (1.0f / 16777216.0f);
  }
};

__device__ __forceinline__ float vpt_density(const VptArgs& s, float x, float y, float z) {
  if (fabsf(x) > 1.0f || fabsf(y) > 1.0f || fabsf(z) > 1.0f) return 0.0f;
  float acc = 0.0f;
  for (int i = 0; i < s.n_blobs; ++i) {
    const float dx = x - s.blob[i].cx, dy = y - s.blob[i].cy, dz = z - s.blob[i].cz;
    acc = fmaf(s.blob[i].a, expf(-(dx * dx + dy * dy + dz * dz) * s.blob[i].inv2r2), acc);
  }
  return fminf(acc, 1.0f);
}

__device__ __forceinline__ float vpt_opacity(const VptArgs& s, float rho) {
  return fminf(fmaxf((rho - s.tf_lo) * s.inv_tf_span, 0.0f), 1.0f);
}

// [t0, t1] of the ray o + t d inside [-1, 1]^3 with t >= 0; false if empty.
__device__ __forceinline__ bool vpt_box(const float o[3], const float d[3], float& t0, float& t1) {
  float lo = 0.0f, hi = INFINITY;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float inv = 1.0f / d[a];
    float ta = (-1.0f - o[a]) * inv, tb = (1.0f - o[a]) * inv;
    if (ta > tb) {
      const float t = ta;
      ta = tb;
      tb = t;
    }
    lo = fmaxf(lo, ta);
    hi = fminf(hi, tb);
  }
  t0 = lo;
  t1 = hi;
  return lo < hi;
}

__device__ bool vpt_visible(const VptArgs& s, Philox& g, const float p[3], const float w[3]) {
  float t0, t1;
  if (!vpt_box(p, w, t0, t1)) return true;
  float t = t0;
  for (;;) {
    if (++g.steps > kVptMaxSteps) return false;
    t += -logf(1.0f - g.u()) * s.inv_mu_max;
    if (t >= t1) return true;
    const float mu = s.mu_max * vpt_opacity(s, vpt_density(s, p[0] + t * w[0], p[1] + t * w[1], p[2] + t * w[2]));
    if (g.u() < mu * s.inv_mu_max) return false;
  }
}

__global__ void __launch_bounds__(128)
    k_render_vpt(const __grid_constant__ VptArgs s, const int W, const int H, const int spp, const uint32_t frame,
                 float* __restrict__ samples, float* __restrict__ world, float* __restrict__ features) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W || y >= H) return;
  const size_t np = (size_t)W * H, j = (size_t)y * W + x;
  float best_t = INFINITY, by0 = 0.0f, by1 = 0.0f, by2 = 0.0f;
  for (int smp = 0; smp < spp; ++smp) {
    Philox g;
    g.c0 = (uint32_t)j;
    g.c1 = (uint32_t)smp;
    g.c2 = frame;
    g.c3 = 0u;
    g.k0 = s.key0;
    g.k1 = s.key1;
    g.used = 4;
    g.steps = 0;
    const float ox = g.u() - 0.5f, oy = g.u() - 0.5f;
    const float nx = ((float)x + 0.5f + ox) / (float)W * 2.0f - 1.0f;
    const float ny = 1.0f - ((float)y + 0.5f + oy) / (float)H * 2.0f;
    float P[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) P[r] = s.ivp[r * 4 + 0] * nx + s.ivp[r * 4 + 1] * ny + s.ivp[r * 4 + 2] + s.ivp[r * 4 + 3];
    float w[3] = {P[0] / P[3] - s.eye[0], P[1] / P[3] - s.eye[1], P[2] / P[3] - s.eye[2]};
    const float inv_n = 1.0f / sqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    w[0] *= inv_n;
    w[1] *= inv_n;
    w[2] *= inv_n;
    float o[3] = {s.eye[0], s.eye[1], s.eye[2]};
    float L0 = 0.0f, L1 = 0.0f, L2 = 0.0f, b0 = 1.0f, b1 = 1.0f, b2 = 1.0f;
    bool hit = false;
    float t0, t1;
    if (!vpt_box(o, w, t0, t1)) {
      L0 = s.env_rgb[0];
      L1 = s.env_rgb[1];
      L2 = s.env_rgb[2];
    } else {
      float t = t0;
      int bounces = 0;
      for (;;) {
        if (++g.steps > kVptMaxSteps) break;
        t += -logf(1.0f - g.u()) * s.inv_mu_max;
        if (t >= t1) {  // leaves the volume: background
          L0 = fmaf(b0, s.env_rgb[0], L0);
          L1 = fmaf(b1, s.env_rgb[1], L1);
          L2 = fmaf(b2, s.env_rgb[2], L2);
          break;
        }
        const float p[3] = {o[0] + t * w[0], o[1] + t * w[1], o[2] + t * w[2]};
        const float rho = vpt_density(s, p[0], p[1], p[2]);
        const float mu = s.mu_max * vpt_opacity(s, rho);
        if (!(g.u() < mu * s.inv_mu_max)) continue;  // null collision
        if (!hit) {
          hit = true;
          if (t < best_t) {
            best_t = t;
            by0 = p[0];
            by1 = p[1];
            by2 = p[2];
          }
        }
        b0 *= s.albedo * fmaf(rho, s.col_span[0], s.col_lo[0]);
        b1 *= s.albedo * fmaf(rho, s.col_span[1], s.col_lo[1]);
        b2 *= s.albedo * fmaf(rho, s.col_span[2], s.col_lo[2]);
        if (vpt_visible(s, g, p, s.light_dir)) {
          L0 = fmaf(b0, s.light_rgb[0] * (1.0f / (4.0f * kVptPi)), L0);
          L1 = fmaf(b1, s.light_rgb[1] * (1.0f / (4.0f * kVptPi)), L1);
          L2 = fmaf(b2, s.light_rgb[2] * (1.0f / (4.0f * kVptPi)), L2);
        }
        if (++bounces >= s.max_bounces) break;
        const float z = 1.0f - 2.0f * g.u(), phi = 2.0f * kVptPi * g.u();
        const float r = sqrtf(fmaxf(1.0f - z * z, 0.0f));
        float sn, cs;
        sincosf(phi, &sn, &cs);
        w[0] = r * cs;
        w[1] = r * sn;
        w[2] = z;
        o[0] = p[0];
        o[1] = p[1];
        o[2] = p[2];
        if (!vpt_box(o, w, t0, t1)) t1 = 0.0f;
        t = 0.0f;
      }
    }
    float* out = samples + (size_t)smp * 5 * np + j;
    out[0] = L0;
    out[np] = L1;
    out[2 * np] = L2;
    out[3 * np] = ox;
    out[4 * np] = oy;
  }
  const bool any = best_t < INFINITY;
  const float nan = __int_as_float(0x7fc00000);
  world[j] = any ? by0 : nan;
  world[np + j] = any ? by1 : nan;
  world[2 * np + j] = any ? by2 : nan;
  if (features) {
    float f[7] = {0, 0, 0, 0, 0, 0, 0};
    if (any) {
      float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
      for (int i = 0; i < s.n_blobs; ++i) {
        const float dx = by0 - s.blob[i].cx, dy = by1 - s.blob[i].cy, dz = by2 - s.blob[i].cz;
        const float e = s.blob[i].a * expf(-(dx * dx + dy * dy + dz * dz) * s.blob[i].inv2r2);
        const float k = -2.0f * s.blob[i].inv2r2 * e;  // d/dx of e = -(x - c) / r^2 e
        g0 = fmaf(k, dx, g0);
        g1 = fmaf(k, dy, g1);
        g2 = fmaf(k, dz, g2);
      }
      const float gn = sqrtf(g0 * g0 + g1 * g1 + g2 * g2);
      const float rho = vpt_density(s, by0, by1, by2);
      f[0] = best_t;
      if (gn > 0.0f) {
        f[1] = -g0 / gn;
        f[2] = -g1 / gn;
        f[3] = -g2 / gn;
      }
      f[4] = fmaf(rho, s.col_span[0], s.col_lo[0]);
      f[5] = fmaf(rho, s.col_span[1], s.col_lo[1]);
      f[6] = fmaf(rho, s.col_span[2], s.col_lo[2]);
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) features[k * np + j] = f[k];
  }
}

}  // namespace wrls

using namespace wrls;

extern "C" {

wrls_status wrls_render_vpt(const wrls_vpt_scene* sc, int width, int height, int spp, uint32_t frame,
                            float* samples, float* world, float* features, void* cuda_stream) {
  NvtxRange nvtx("wrls_render_vpt");
  if (!sc || sc->struct_size != sizeof(wrls_vpt_scene)) {
    set_error("wrls_render_vpt: scene NULL or struct_size != sizeof(wrls_vpt_scene)");
    return WRLS_ERR_INVALID_ARG;
  }
  if (width < 1 || height < 1 || width > 16384 || height > 16384 || spp < 1 || spp > 1024 || !samples || !world) {
    set_error("wrls_render_vpt: bad size (%d x %d, spp %d) or NULL samples/world", width, height, spp);
    return WRLS_ERR_INVALID_ARG;
  }
  if (sc->n_blobs < 0 || sc->n_blobs > 16 || !(sc->mu_max > 0.0f) || !(sc->tf_hi > sc->tf_lo) ||
      sc->max_bounces < 1 || !(sc->albedo >= 0.0f)) {
    set_error("wrls_render_vpt: n_blobs in [0, 16], mu_max > 0, tf_hi > tf_lo, max_bounces >= 1, albedo >= 0");
    return WRLS_ERR_INVALID_ARG;
  }
  if (((uintptr_t)samples | (uintptr_t)world | (uintptr_t)features) & 3u) {
    set_error("wrls_render_vpt: buffers must be 4-byte aligned");
    return WRLS_ERR_INVALID_ARG;
  }
  const size_t np = (size_t)width * height;
  const char* sm = (const char*)samples;
  const char* wd = (const char*)world;
  const char* ft = (const char*)features;
  if ((sm < wd + 12 * np && wd < sm + 20 * np * spp) ||
      (ft && ((ft < sm + 20 * np * spp && sm < ft + 28 * np) || (ft < wd + 12 * np && wd < ft + 28 * np)))) {
    set_error("wrls_render_vpt: output buffers overlap");
    return WRLS_ERR_INVALID_ARG;
  }
  VptArgs a;
  memset(&a, 0, sizeof(a));
  a.key0 = sc->seed[0];
  a.key1 = sc->seed[1];
  for (int i = 0; i < 3; ++i) {
    a.eye[i] = sc->eye[i];
    a.col_lo[i] = sc->color_lo[i];
    a.col_span[i] = sc->color_hi[i] - sc->color_lo[i];
    a.light_dir[i] = sc->light_dir[i];
    a.light_rgb[i] = sc->light_rgb[i];
    a.env_rgb[i] = sc->env_rgb[i];
  }
  for (int i = 0; i < 16; ++i) a.ivp[i] = sc->inv_view_proj[i];
  a.n_blobs = sc->n_blobs;
  for (int i = 0; i < sc->n_blobs; ++i) {
    const float r = sc->blobs[i][3];
    if (!(r > 0.0f)) {
      set_error("wrls_render_vpt: blob %d has a non-positive radius", i);
      return WRLS_ERR_INVALID_ARG;
    }
    a.blob[i] = VptBlob{sc->blobs[i][0], sc->blobs[i][1], sc->blobs[i][2], (float)(1.0 / (2.0 * (double)r * r)),
                        sc->blobs[i][4]};
  }
  a.mu_max = sc->mu_max;
  a.inv_mu_max = (float)(1.0 / (double)sc->mu_max);
  a.tf_lo = sc->tf_lo;
  a.inv_tf_span = (float)(1.0 / ((double)sc->tf_hi - (double)sc->tf_lo));
  a.albedo = sc->albedo;
  a.max_bounces = sc->max_bounces;
  const dim3 grid((width + 127) / 128, height);
  k_render_vpt<<<grid, 128, 0, (cudaStream_t)cuda_stream>>>(a, width, height, spp, frame, samples, world, features);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("wrls_render_vpt: launch: %s", cudaGetErrorString(e));
    return WRLS_ERR_CUDA;
  }
  return WRLS_OK;
}

}  // extern "C"
