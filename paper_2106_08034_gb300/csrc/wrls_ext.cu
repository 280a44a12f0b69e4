// Extended predictor and weights (streams whose parameters select them):
//   - G-buffer entries in the predictor, p = [1, z, g_1..g_n] (or [1, g_1..g_n] without the
//     temporal feature), d up to 8: the regression on auxiliary G-buffer features of RLS
//     denoisers that Sec. 2.1 and Sec. 5.2-5.3 discuss (and argue against for noisy
//     path-traced G-buffers);
//   - the sample-variance weight that Sec. 5.3 sets aside: Eq. 13 with the squared colour
//     distance replaced by its expectation 3 sigma^2 under the per-pixel variance;
//   - nearest-pixel reprojection (floor(q + 0.5) per axis, binary32).
// Everything else is the paper's step for step: reprojection, Eq. 12 feature with the 3x3
// clamp, Eq. 13 / Eq. 14 / Eq. 8 / Eq. 9 / Eq. 11, restarts, missing samples, the wind-up
// guard and the 5x5 bilateral cross-prediction blend (Sec. 5.3).
//
// State: binary32 planes, d = predictor dimension: beta[c][a] (plane c*d + a), the upper
// triangle of P row by row (d(d+1)/2 planes), z (3 planes). With d = 4 and the temporal
// feature this is the paper layout of the fast kernels.
//
// The update is one thread per pixel with plain cached loads (32 x 8 tiles); the blend
// stages the 36 x 12 window of beta, z and the per-pixel range factor in shared memory and
// gives each thread two vertically adjacent outputs of the 32 x 8 tile.
#include "wrls_internal.h"

namespace wrls {

template <int D, bool F>
struct ExtDim {
  static constexpr int kG = D - (F ? 4 : 1);  // G-buffer entries of p
  static constexpr int kNP = D * (D + 1) / 2;
  static constexpr int kBeta = 0;
  static constexpr int kP = 3 * D;
  static constexpr int kZ = 3 * D + kNP;
  static constexpr int kNS = kZ + 3;
  static constexpr int kG0 = F ? 4 : 1;  // index of the first G-buffer entry in p
};

// Index of P(a, b), a <= b, in the packed upper triangle (row by row).
__host__ __device__ constexpr int sym_index(int d, int a, int b) { return a * d - a * (a - 1) / 2 + (b - a); }

__device__ __forceinline__ bool finite3(const float v[3]) {
  return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]);
}

constexpr int kExtTW = 32, kExtTH = 8;

template <int D, bool F>
__global__ void __launch_bounds__(kExtTW * kExtTH)
    k_update_ext(const ExtParams ep, const int W, const int H, const int reset, const float* __restrict__ prev,
                 float* __restrict__ next, const int pitch, const size_t ps, const float* __restrict__ rad,
                 const float* __restrict__ mot, const float* __restrict__ var, const float* __restrict__ gbuf) {
  using L = ExtDim<D, F>;
  const KParams& kp = ep.kp;
  const int x = blockIdx.x * kExtTW + threadIdx.x, y = blockIdx.y * kExtTH + threadIdx.y;
  const bool inside = x < W && y < H;
  const size_t npix = (size_t)W * H, j = (size_t)y * W + x;

  // reprojection q = j + v_j (Table 2), binary32; NaN motion fails every comparison
  float qx = 0.0f, qy = 0.0f;
  bool valid = false;
  if (inside) {
    qx = (float)x + __ldg(mot + j);
    qy = (float)y + __ldg(mot + npix + j);
    valid = !reset && qx >= 0.0f && qx <= (float)(W - 1) && qy >= 0.0f && qy <= (float)(H - 1);
  }
  // a warp (one tile row) whose valid pixels all have an integral vertical motion component
  // reads only the upper two taps
  const bool fy0 = __all_sync(0xffffffffu, !valid || qy == floorf(qy));
  if (!inside) return;
  const float I[3] = {__ldg(rad + j), __ldg(rad + npix + j), __ldg(rad + 2 * npix + j)};
  const bool missing = !finite3(I);

  float st[L::kNS];
  if (valid) {
    if (ep.reproj_filter == 1) {
      const int xn = (int)floorf(qx + 0.5f), yn = (int)floorf(qy + 0.5f);
      const float* src = prev + (size_t)yn * pitch + xn;
#pragma unroll
      for (int p = 0; p < L::kNS; ++p) st[p] = __ldg(src + p * ps);
    } else {
      const int x0 = (int)floorf(qx), y0 = (int)floorf(qy);
      const float fx = qx - (float)x0, fy = qy - (float)y0;
      const int x1 = min(x0 + 1, W - 1), y1 = min(y0 + 1, H - 1);
      const float w00 = (1.0f - fx) * (1.0f - fy), w10 = fx * (1.0f - fy);
      const float w01 = (1.0f - fx) * fy, w11 = fx * fy;
      const float* s00 = prev + (size_t)y0 * pitch + x0;
      const float* s10 = prev + (size_t)y0 * pitch + x1;
      const float* s01 = prev + (size_t)y1 * pitch + x0;
      const float* s11 = prev + (size_t)y1 * pitch + x1;
      if (fy0) {  // the lower taps have weight exactly 0 (adding 0 * v leaves the sum as it is)
#pragma unroll
        for (int p = 0; p < L::kNS; ++p) {
          const size_t o = p * ps;
          st[p] = w00 * __ldg(s00 + o) + w10 * __ldg(s10 + o);
        }
      } else {
#pragma unroll
        for (int p = 0; p < L::kNS; ++p) {
          const size_t o = p * ps;
          st[p] = w00 * __ldg(s00 + o) + w10 * __ldg(s10 + o) + (w01 * __ldg(s01 + o) + w11 * __ldg(s11 + o));
        }
      }
    }
  }

  // Eq. 12 temporal feature (Psi = clamp to the 3x3 min/max of the finite samples)
  float z[3];
  if (valid) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool any = false;
    if (kp.clamp_mode == 0) {
      for (int dy = -1; dy <= 1; ++dy) {
        const int yy = y + dy;
        if (yy < 0 || yy >= H) continue;
        for (int dx = -1; dx <= 1; ++dx) {
          const int xx = x + dx;
          if (xx < 0 || xx >= W) continue;
          const size_t jj = (size_t)yy * W + xx;
          const float In[3] = {__ldg(rad + jj), __ldg(rad + npix + jj), __ldg(rad + 2 * npix + jj)};
          if (!finite3(In)) continue;
          any = true;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            lo[c] = fminf(lo[c], In[c]);
            hi[c] = fmaxf(hi[c], In[c]);
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float zc = st[L::kZ + c];
      if (any) zc = fminf(fmaxf(zc, lo[c]), hi[c]);
      z[c] = missing ? zc : fmaf(kp.alpha, zc, kp.one_m_alpha * I[c]);
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) z[c] = missing ? 0.0f : I[c];
#pragma unroll
    for (int p = 0; p < L::kZ; ++p) st[p] = 0.0f;
    if (kp.init_mode == 1) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (F) st[L::kBeta + c * D + c + 1] = 1.0f;
        else st[L::kBeta + c * D] = z[c];
      }
    }
#pragma unroll
    for (int a = 0; a < D; ++a) st[L::kP + sym_index(D, a, a)] = kp.p0_delta;
  }

  // predictor p = [1, z, g] of frame t; a non-finite G-buffer value enters as 0, weight 0
  float p[D];
  p[0] = 1.0f;
  if (F) {
    p[1] = z[0];
    p[2] = z[1];
    p[3] = z[2];
  }
  bool g_ok = true;
#pragma unroll
  for (int i = 0; i < L::kG; ++i) {
    const float g = __ldg(gbuf + (size_t)i * npix + j);
    const bool f = isfinite(g);
    p[L::kG0 + i] = f ? g : 0.0f;
    g_ok = g_ok && f;
  }

  // weight: Eq. 13, RLS (w = 1) or the sample-variance weight
  float w;
  if (missing || !g_ok) {
    w = 0.0f;
  } else if (kp.weight_mode == 1) {
    w = 1.0f;
  } else {
    const float nI = sqrtf(I[0] * I[0] + I[1] * I[1] + I[2] * I[2]);
    const float nz = sqrtf(z[0] * z[0] + z[1] * z[1] + z[2] * z[2]);
    const float m = fminf(nI, nz) + kp.eps;
    if (kp.weight_mode == 2) {
      const float v = __ldg(var + j);
      w = (isfinite(v) && v >= 0.0f) ? ex2_approx(-(v / (m * m)) * ep.wv_k) : 0.0f;
    } else {
      const float d0 = I[0] - z[0], d1 = I[1] - z[1], d2 = I[2] - z[2];
      w = ex2_approx(-((d0 * d0 + d1 * d1 + d2 * d2) / (m * m)) * kp.w_k);
    }
  }

  // k = P p, s = p^T P p; Eq. 14 gain q^w = (w / (lambda + w s)) k
  float* P = st + L::kP;
  float k[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    float acc = 0.0f;
#pragma unroll
    for (int b = 0; b < D; ++b) acc = fmaf(P[a <= b ? sym_index(D, a, b) : sym_index(D, b, a)], p[b], acc);
    k[a] = acc;
  }
  float s = 0.0f;
#pragma unroll
  for (int a = 0; a < D; ++a) s = fmaf(p[a], k[a], s);
  const float gain = w / (kp.lambda + w * s);
  const bool use = !(missing || !g_ok);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float* beta = st + L::kBeta + c * D;
    float pred = 0.0f;
#pragma unroll
    for (int a = 0; a < D; ++a) pred = fmaf(p[a], beta[a], pred);
    const float ge = gain * (use ? I[c] - pred : 0.0f);  // Eq. 8, Eq. 9
#pragma unroll
    for (int a = 0; a < D; ++a) beta[a] = fmaf(ge, k[a], beta[a]);
  }
  // Eq. 11: P <- (P - q^w p^T P) / lambda, p^T P = k^T
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = a; b < D; ++b) {
      const int e = sym_index(D, a, b);
      P[e] = (P[e] - gain * k[a] * k[b]) * kp.inv_lambda;
    }
  if (kp.p_trace_max > 0.0f) {
    float tr = 0.0f;
    bool bad = false;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const float v = P[sym_index(D, a, a)];
      tr += v;
      bad = bad || !(v > 0.0f);
    }
    if (bad || tr > kp.p_trace_max) {
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b) P[sym_index(D, a, b)] = a == b ? kp.p0_delta : 0.0f;
    }
  }
  st[L::kZ + 0] = z[0];
  st[L::kZ + 1] = z[1];
  st[L::kZ + 2] = z[2];
  float* dst = next + (size_t)y * pitch + x;
#pragma unroll
  for (int q = 0; q < L::kNS; ++q) dst[q * ps] = st[q];
}

constexpr int kExtSW = kExtTW + 4, kExtSH = kExtTH + 4, kExtSP = kExtSW * kExtSH;
constexpr float kExtFarZ = 1e18f;  // feature of an out-of-image neighbour: its blend weight is 0

// 5x5 blend: out_i = sum_k b_ik (p_i beta_k) / sum_k b_ik (blend_mode 1: p_k beta_k), with
// b_ik = 2^(spatial_ik - |z_i - z_k|^2 max(r_i, r_k)), r = log2(e) / (h_s^2 (|z| + eps)^2):
// the Eq. 13 distance of the two features, min(|z_i|, |z_k|) taken through max(r_i, r_k).
// A CTA of 32 x 4 threads blends a 32 x 8 tile; each thread produces two vertically adjacent
// outputs, so that every neighbour read from shared memory serves both (6 x 5 reads for two
// outputs instead of 2 x 25).
constexpr int kExtBlendRows = 2;

template <int D, bool F>
__device__ __forceinline__ void ext_predictor_g(const float* __restrict__ gbuf, size_t npix, size_t j, float p[D]) {
  using L = ExtDim<D, F>;
#pragma unroll
  for (int i = 0; i < L::kG; ++i) {
    const float g = __ldg(gbuf + (size_t)i * npix + j);
    p[L::kG0 + i] = isfinite(g) ? g : 0.0f;
  }
}

template <int D, bool F>
__global__ void __launch_bounds__(kExtTW * kExtTH / kExtBlendRows)
    k_blend_ext(const ExtParams ep, const int W, const int H, const float* __restrict__ cur, const int pitch,
                const size_t ps, const float* __restrict__ gbuf, float* __restrict__ out) {
  using L = ExtDim<D, F>;
  constexpr int NPL = 3 * D + 4;  // beta planes, z (3), range factor
  constexpr int NT = kExtTW * kExtTH / kExtBlendRows;
  static_assert(NPL * kExtSP * 4 <= 48 * 1024, "blend window exceeds static shared memory");
  __shared__ float sm[NPL * kExtSP];
  const KParams& kp = ep.kp;
  const int bx0 = blockIdx.x * kExtTW, by0 = blockIdx.y * kExtTH;
  const int tid = threadIdx.y * kExtTW + threadIdx.x;
  for (int e = tid; e < kExtSP; e += NT) {
    const int gx = bx0 - 2 + e % kExtSW, gy = by0 - 2 + e / kExtSW;
    if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
      const float* src = cur + (size_t)gy * pitch + gx;
#pragma unroll
      for (int a = 0; a < 3 * D; ++a) sm[a * kExtSP + e] = __ldg(src + (L::kBeta + a) * ps);
      const float z0 = __ldg(src + (L::kZ + 0) * ps), z1 = __ldg(src + (L::kZ + 1) * ps),
                  z2 = __ldg(src + (L::kZ + 2) * ps);
      sm[(3 * D + 0) * kExtSP + e] = z0;
      sm[(3 * D + 1) * kExtSP + e] = z1;
      sm[(3 * D + 2) * kExtSP + e] = z2;
      const float nz = sqrtf(z0 * z0 + z1 * z1 + z2 * z2) + kp.eps;
      sm[(3 * D + 3) * kExtSP + e] = kp.range_k / (nz * nz);
    } else {
#pragma unroll
      for (int a = 0; a < 3 * D; ++a) sm[a * kExtSP + e] = 0.0f;
      sm[(3 * D + 0) * kExtSP + e] = kExtFarZ;
      sm[(3 * D + 1) * kExtSP + e] = kExtFarZ;
      sm[(3 * D + 2) * kExtSP + e] = kExtFarZ;
      sm[(3 * D + 3) * kExtSP + e] = 0.0f;
    }
  }
  __syncthreads();
  const int x = bx0 + threadIdx.x;
  const int ty0 = threadIdx.y * kExtBlendRows;  // first of the thread's two rows in the tile
  const size_t npix = (size_t)W * H;
  // the two outputs' features, range factors and predictors
  float zi[kExtBlendRows][3], ri[kExtBlendRows], pi[kExtBlendRows][D];
#pragma unroll
  for (int r = 0; r < kExtBlendRows; ++r) {
    const int ei = (ty0 + r + 2) * kExtSW + threadIdx.x + 2;
    zi[r][0] = sm[(3 * D + 0) * kExtSP + ei];
    zi[r][1] = sm[(3 * D + 1) * kExtSP + ei];
    zi[r][2] = sm[(3 * D + 2) * kExtSP + ei];
    ri[r] = sm[(3 * D + 3) * kExtSP + ei];
    pi[r][0] = 1.0f;
    if (F) {
      pi[r][1] = zi[r][0];
      pi[r][2] = zi[r][1];
      pi[r][3] = zi[r][2];
    }
    const int y = by0 + ty0 + r;
#pragma unroll
    for (int i = 0; i < L::kG; ++i) pi[r][L::kG0 + i] = 0.0f;
    if (x < W && y < H) ext_predictor_g<D, F>(gbuf, npix, (size_t)y * W + x, pi[r]);
  }
  float num[kExtBlendRows][3] = {}, den[kExtBlendRows] = {};
#pragma unroll
  for (int wy = 0; wy < 4 + kExtBlendRows; ++wy)  // window rows ty0 .. ty0 + 5 (relative)
#pragma unroll
    for (int dx = 0; dx < 5; ++dx) {
      const int e = (ty0 + wy) * kExtSW + threadIdx.x + dx;
      const float zk0 = sm[(3 * D + 0) * kExtSP + e], zk1 = sm[(3 * D + 1) * kExtSP + e],
                  zk2 = sm[(3 * D + 2) * kExtSP + e];
      const float rk = sm[(3 * D + 3) * kExtSP + e];
      float bk[3 * D];
#pragma unroll
      for (int a = 0; a < 3 * D; ++a) bk[a] = sm[a * kExtSP + e];
      float own[3] = {0.0f, 0.0f, 0.0f};  // blend_mode 1: neighbour k's own prediction
      if (kp.blend_mode != 0) {
        const int xx = x + dx - 2, yy = by0 + ty0 + wy - 2;
        const bool in = xx >= 0 && xx < W && yy >= 0 && yy < H;
        float pk[D];
        pk[0] = 1.0f;
        if (F) {
          pk[1] = in ? zk0 : 0.0f;
          pk[2] = in ? zk1 : 0.0f;
          pk[3] = in ? zk2 : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < L::kG; ++i) pk[L::kG0 + i] = 0.0f;
        if (in) ext_predictor_g<D, F>(gbuf, npix, (size_t)yy * W + xx, pk);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          own[0] = fmaf(pk[a], bk[0 * D + a], own[0]);
          own[1] = fmaf(pk[a], bk[1 * D + a], own[1]);
          own[2] = fmaf(pk[a], bk[2 * D + a], own[2]);
        }
      }
#pragma unroll
      for (int r = 0; r < kExtBlendRows; ++r) {
        const int dy = wy - r;  // this neighbour's row offset (0..4) for output r
        if (dy < 0 || dy > 4) continue;  // resolved at compile time
        const float a0 = zi[r][0] - zk0, a1 = zi[r][1] - zk1, a2 = zi[r][2] - zk2;
        const float b = ex2_approx(blend_exponent(kp.spatial[dy * 5 + dx], a0, a1, a2, fmaxf(ri[r], rk)));
        float p0 = own[0], p1 = own[1], p2 = own[2];
        if (kp.blend_mode == 0) {
          p0 = p1 = p2 = 0.0f;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            p0 = fmaf(pi[r][a], bk[0 * D + a], p0);
            p1 = fmaf(pi[r][a], bk[1 * D + a], p1);
            p2 = fmaf(pi[r][a], bk[2 * D + a], p2);
          }
        }
        num[r][0] = fmaf(b, p0, num[r][0]);
        num[r][1] = fmaf(b, p1, num[r][1]);
        num[r][2] = fmaf(b, p2, num[r][2]);
        den[r] += b;
      }
    }
#pragma unroll
  for (int r = 0; r < kExtBlendRows; ++r) {
    const int y = by0 + ty0 + r;
    if (x >= W || y >= H) continue;
    const size_t j = (size_t)y * W + x;
    const float inv = 1.0f / den[r];
    out[j] = num[r][0] * inv;
    out[npix + j] = num[r][1] * inv;
    out[2 * npix + j] = num[r][2] * inv;
  }
}

__global__ void k_read_state_ext(const int W, const int H, const float* __restrict__ cur, const int pitch,
                                 const size_t ps, const int nplanes, float* __restrict__ dst) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W || y >= H) return;
  const size_t npix = (size_t)W * H, j = (size_t)y * W + x;
  const float* src = cur + (size_t)y * pitch + x;
  for (int p = 0; p < nplanes; ++p) dst[p * npix + j] = src[p * ps];
}

__global__ void k_write_state_ext(const int W, const int H, float* __restrict__ cur, const int pitch,
                                  const size_t ps, const int nplanes, const float* __restrict__ src) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W || y >= H) return;
  const size_t npix = (size_t)W * H, j = (size_t)y * W + x;
  float* dst = cur + (size_t)y * pitch + x;
  for (int p = 0; p < nplanes; ++p) dst[p * ps] = src[p * npix + j];
}

template <int D, bool F>
static cudaError_t launch_ext_t(const ExtParams& ep, const StateDesc& prev, const StateDesc& next, bool reset,
                                const float* rad, const float* mot, const float* var, const float* gbuf,
                                float* out, cudaStream_t cs) {
  const dim3 grid((prev.W + kExtTW - 1) / kExtTW, (prev.H + kExtTH - 1) / kExtTH), block(kExtTW, kExtTH);
  k_update_ext<D, F><<<grid, block, 0, cs>>>(ep, prev.W, prev.H, reset ? 1 : 0, (const float*)prev.base,
                                             (float*)next.base, prev.pitch, prev.plane_stride, rad, mot, var, gbuf);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !out) return e;
  k_blend_ext<D, F><<<grid, dim3(kExtTW, kExtTH / kExtBlendRows), 0, cs>>>(ep, next.W, next.H, (const float*)next.base, next.pitch,
                                            next.plane_stride, gbuf, out);
  return cudaGetLastError();
}

template <int D, bool F>
static cudaError_t launch_ext_blend_t(const ExtParams& ep, const StateDesc& cur, const float* gbuf, float* out,
                                      cudaStream_t cs) {
  const dim3 grid((cur.W + kExtTW - 1) / kExtTW, (cur.H + kExtTH - 1) / kExtTH), block(kExtTW, kExtTH);
  k_blend_ext<D, F><<<grid, dim3(kExtTW, kExtTH / kExtBlendRows), 0, cs>>>(ep, cur.W, cur.H, (const float*)cur.base, cur.pitch,
                                            cur.plane_stride, gbuf, out);
  return cudaGetLastError();
}

int ext_dim(const wrls_params& p) { return (p.feature_mode == 0 ? 4 : 1) + p.n_gbuf; }

int ext_planes(int d) { return 3 * d + d * (d + 1) / 2 + 3; }

#define WRLS_EXT_DISPATCH(FN, ...)                                 \
  switch ((ep.kp.feature_mode == 0 ? 0 : 16) + d) {                \
    case 4: return FN<4, true>(__VA_ARGS__);                       \
    case 5: return FN<5, true>(__VA_ARGS__);                       \
    case 6: return FN<6, true>(__VA_ARGS__);                       \
    case 7: return FN<7, true>(__VA_ARGS__);                       \
    case 8: return FN<8, true>(__VA_ARGS__);                       \
    case 17: return FN<1, false>(__VA_ARGS__);                     \
    case 18: return FN<2, false>(__VA_ARGS__);                     \
    case 19: return FN<3, false>(__VA_ARGS__);                     \
    case 20: return FN<4, false>(__VA_ARGS__);                     \
    case 21: return FN<5, false>(__VA_ARGS__);                     \
    default: return cudaErrorInvalidValue;                         \
  }

// Update of frame t into `next`, then (out != NULL) the blend of `next` into out.
cudaError_t launch_ext_update(const ExtParams& ep, int d, const StateDesc& prev, const StateDesc& next, bool reset,
                              const float* rad, const float* mot, const float* var, const float* gbuf,
                              cudaStream_t cs) {
  WRLS_EXT_DISPATCH(launch_ext_t, ep, prev, next, reset, rad, mot, var, gbuf, nullptr, cs)
}

cudaError_t launch_ext_blend(const ExtParams& ep, int d, const StateDesc& cur, const float* gbuf, float* out,
                             cudaStream_t cs) {
  WRLS_EXT_DISPATCH(launch_ext_blend_t, ep, cur, gbuf, out, cs)
}

cudaError_t launch_write_state_ext(const StateDesc& cur, int nplanes, const float* src, cudaStream_t cs) {
  const dim3 grid((cur.W + 127) / 128, cur.H);
  k_write_state_ext<<<grid, 128, 0, cs>>>(cur.W, cur.H, (float*)cur.base, cur.pitch, cur.plane_stride, nplanes, src);
  return cudaGetLastError();
}

cudaError_t launch_read_state_ext(const StateDesc& cur, int nplanes, float* dst, cudaStream_t cs) {
  const dim3 grid((cur.W + 127) / 128, cur.H);
  k_read_state_ext<<<grid, 128, 0, cs>>>(cur.W, cur.H, (const float*)cur.base, cur.pitch, cur.plane_stride, nplanes,
                                         dst);
  return cudaGetLastError();
}

}  // namespace wrls
