// Device-side building blocks of the wRLS denoiser (Sec. 5.2-5.3 of Iglesias-Guitian,
// Mane, Moon, IEEE TVCG 2020): kernel parameters, the per-pixel state storage formats,
// and the per-pixel temporal update (reprojection, Eq. 12, Eq. 13, Eq. 8/14/9/11).
//
// State per pixel: beta[3][4] (one linear model per colour channel, Eq. 5), the
// symmetric 4x4 inverse covariance P shared by the three channels (10 values), and the
// temporal feature z[3] (Eq. 12): 25 values. Planes: 0-11 beta[c][a] (c*4+a),
// 12-21 P upper triangle (00,01,02,03,11,12,13,22,23,33), 22-24 z.
#pragma once
#include <cuda.h>  // CUtensorMap (types only; the encoder is looked up at run time)
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace wrls {

constexpr int kNState = 25;
constexpr int kBeta = 0;
constexpr int kP = 12;
constexpr int kZ = 22;
constexpr int kMaxRadius = 2;
constexpr int kMaxTaps = (2 * kMaxRadius + 1) * (2 * kMaxRadius + 1);

// Everything a kernel needs from wrls_params, precomputed on the host.
struct KParams {
  float lambda;       // forgetting factor (Eq. 10-11)
  float inv_lambda;
  float alpha;        // Eq. 12
  float one_m_alpha;
  float eps;          // Eq. 13
  float w_k;          // log2(e) / h^2: Eq. 13 exponent in base 2
  float p0_delta;     // P of a restarted pixel
  float p_trace_max;  // wind-up guard, 0 = off
  float range_k;      // log2(e) / h_s^2: blend range exponent in base 2
  float spatial[kMaxTaps];  // -(dx^2+dy^2) / (2 sigma_s^2) * log2(e), row-major offsets;
                            // -inf beyond the window radius
  int radius;
  int weight_mode;
  int clamp_mode;
  int blend_mode;
  int feature_mode;
  int init_mode;
  int debug_withhold_copy;  // test hook: arm the state-window barrier without issuing the copy
  int blend_ctas_cap;       // host-side launch hint: CTAs per SM of the persistent blends (0 = all that fit)
};

// 2^x on the SFU (PTX ex2.approx, max relative error about 2^-22).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Base-2 exponent of the blend weight of a (pixel i, neighbour k) pair: spatial - |e|^2 rk with
// e = z_i - z_k and rk = K / (min(|z_i|, |z_k|) + eps)^2. The rounding order is fixed here
// (e0^2, then + e1^2, + e2^2 by fused multiply-adds, then one fused multiply-add with -rk) so
// that every blend kernel, scalar or packed (blend_exponent2), gives the same bits.
__device__ __forceinline__ float blend_exponent(float sp, float e0, float e1, float e2, float rk) {
  return fmaf(fmaf(e2, e2, fmaf(e1, e1, e0 * e0)), -rk, sp);
}

// Range factor of a window pixel: rk = K / (|z| + eps)^2 with K = log2(e) / h_s^2, |z|^2 summed
// by fused multiply-adds (one rounding order for every blend kernel).
__device__ __forceinline__ float blend_rk(float z0, float z1, float z2, float eps, float range_k) {
  const float r = 1.0f / (sqrtf(fmaf(z2, z2, fmaf(z1, z1, z0 * z0))) + eps);
  return r * r * range_k;
}

// ---- packed binary32 pairs (sm_100 family: one instruction for two lanes' worth) ----------
// Each component is rounded as the scalar operation would be (round to nearest even, no
// flush), so a packed loop gives bitwise the results of its scalar form.
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
  unsigned long long ra, rb, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }

// blend_rk of two pixels: the same operations in the same order per component (the square
// root and the reciprocal per component), so each component equals blend_rk bit for bit.
__device__ __forceinline__ float2 blend_rk2(float2 z0, float2 z1, float2 z2, float eps, float range_k) {
  const float2 q = f2fma(z2, z2, f2fma(z1, z1, f2mul(z0, z0)));
  const float2 d = f2add(make_float2(sqrtf(q.x), sqrtf(q.y)), make_float2(eps, eps));
  const float2 r = make_float2(1.0f / d.x, 1.0f / d.y);
  return f2mul(f2mul(r, r), make_float2(range_k, range_k));
}

// Cross prediction of one colour channel of pixel i by neighbour k's model (Sec. 5.3):
// p_i . beta_k,c = b0 + a1 b1 + a2 b2 + a3 b3 with p_i = [1, a1, a2, a3], accumulated in this
// order by fused multiply-adds in every blend kernel.
__device__ __forceinline__ float cross_pred(float b0, float b1, float b2, float b3, float a1, float a2, float a3) {
  return fmaf(a3, b3, fmaf(a2, b2, fmaf(a1, b1, b0)));
}
__device__ __forceinline__ float2 cross_pred2(float2 b0, float2 b1, float2 b2, float2 b3, float2 a1, float2 a2,
                                              float2 a3) {
  return f2fma(a3, b3, f2fma(a2, b2, f2fma(a1, b1, b0)));
}

// blend_exponent for two pairs at once; nrk holds -rk.
__device__ __forceinline__ float2 blend_exponent2(float2 sp, float2 e0, float2 e1, float2 e2, float2 nrk) {
  return f2fma(f2fma(e2, e2, f2fma(e1, e1, f2mul(e0, e0))), nrk, sp);
}

// ---- TMA / mbarrier helpers (inline PTX) ------------------------------------------------

// Staged window of the previous state for one 32 x 8 update tile: kStageH rows x kStageW
// columns of every plane. It covers the tile's bilinear taps (33 x 9) with up to 3 columns for
// the 16-byte alignment of the box origin, 4 columns and 1 row of motion spread across the
// tile; a tile whose taps spread further reads them from global memory. 10 rows rather than 12
// leave the binary32 update 44 KB of shared memory a CTA, 5 CTAs per SM.
constexpr int kStageW = 40;
constexpr int kStageH = 10;
constexpr int kStagePix = kStageW * kStageH;
// Bounded waits give up after this many SM clocks (about one second) and report
// WRLS_ERR_TIMEOUT through the stream's error word.
constexpr long long kWaitLimit = 2000000000LL;

// Tensor map of one state copy: all planes as a 3-D tensor (x, y, plane) of 32-bit elements
// (binary32 values, or the packed 16-bit pairs of the 16-bit formats).
struct StageMaps {
  CUtensorMap planes;
};

// Tensor maps of the blend windows of a state copy, boxes of kBlendBoxW (or kBlendBoxW2) columns
// x (TH + 4) rows, for blend tiles of TH = 16 and TH = 8: binary32 state, the 12 beta planes and
// the 3 z planes; 16-bit formats (two-wide boxes only), the 6 beta words and the 2 z words.
constexpr int kBlendBoxW = 40;
constexpr int kBlendBoxW2 = 72;  // two-wide blend tiles: 64 + 2 x 4 columns
struct BlendMaps {
  CUtensorMap beta16, z16, beta8, z8;      // 40-column boxes
  CUtensorMap beta16w, z16w, beta8w, z8w;  // 72-column boxes
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
// Wait for the completion of phase `phase`; false if it did not complete in kWaitLimit clocks.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, phase)) {
    if (clock64() - t0 > kWaitLimit) return false;
  }
  return true;
}
// Order this thread's generic-proxy shared-memory accesses before later async-proxy (TMA) ones.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// ---- state storage formats -------------------------------------------------------------
// A view of one state copy: plane p of pixel (x, y) is at p * plane_stride + y * pitch + x.
// Every format offers
//   load(idx, v)          the 25 values, decoded (P itself)
//   load_raw(idx, v, s)   the 25 values with P divided by a power-of-two scale s (binary32:
//                         s = 1), which the bilinear gather folds into the tap weights
//   load_beta_z(idx, b, z), store(idx, v), and the staged-window geometry of the update.

struct StateF32 {
  float* base;
  size_t plane_stride;
  int pitch;
  __device__ __forceinline__ void load(size_t idx, float v[kNState]) const {
#pragma unroll
    for (int p = 0; p < kNState; ++p) v[p] = __ldg(base + p * plane_stride + idx);
  }
  __device__ __forceinline__ void load_raw(size_t idx, float v[kNState], float& s) const {
    load(idx, v);
    s = 1.0f;
  }
  __device__ __forceinline__ void load_beta_z(size_t idx, float b[12], float z[3]) const {
#pragma unroll
    for (int p = 0; p < 12; ++p) b[p] = __ldg(base + p * plane_stride + idx);
#pragma unroll
    for (int c = 0; c < 3; ++c) z[c] = __ldg(base + (kZ + c) * plane_stride + idx);
  }
  // idx < 2^32: each plane's base is uniform over the warp and the pixel offset 32-bit
  __device__ __forceinline__ void store(size_t idx, const float v[kNState]) const {
    const uint32_t i = (uint32_t)idx;
#pragma unroll
    for (int p = 0; p < kNState; ++p) (base + p * plane_stride)[i] = v[p];
  }
  // Staged window: [plane][kStageH][kStageW] binary32; box origin x multiple of 4 (16 B).
  static constexpr int kPlanes = kNState;  // 32-bit planes of a copy
  static constexpr int kAlignX = 4;
  static constexpr uint32_t kStageBytes = kPlanes * kStagePix * 4;
  static constexpr uint32_t kTxBytes = kStageBytes;  // bytes the bulk copy delivers
  static constexpr bool kScaled = false;
  static __device__ __forceinline__ void load_staged(const unsigned char* stage, int idx, float v[kNState], float& s) {
    const float* f = (const float*)stage;
#pragma unroll
    for (int p = 0; p < kNState; ++p) v[p] = f[p * kStagePix + idx];
    s = 1.0f;
  }
};

// 16-bit storage in packed pairs. Word plane k (k = 0..11) holds the 16-bit values of slots
// 2k (low half) and 2k + 1 (high half) of a pixel; word plane 12 holds z_2 in its low half and,
// in its high half, the exponent e (16-bit two's complement, even) of the pixel's P scale
// s = 2^e. Slots 0-11 are beta and 22-23 z_0, z_1, stored as they are; slots 12-21 hold the
// Cholesky factor of P / s, P / s = L L^T with L lower triangular (l00, l10, l20, l30, l11,
// l21, l31, l22, l32, l33 in the positions of P's upper triangle), so that the decoded P is
// positive semi-definite whatever the rounding (a P rounded entry by entry to 16 bits loses its
// definiteness when its eigenvalues spread more than the format's precision, after which the
// recursion diverges). e = the even number in {f, f + 1} with f = floor(log2 max diag P) + 1,
// clamped to [-126, 126], so |l_ij| <= 1 and scaling by s = 2^e is exact. Each tap's P / s is
// formed from its factor; its s is folded into the tap's bilinear weight, so the reprojection
// interpolates P itself, as with the binary32 state (interpolating the factors instead, with
// one L L^T per pixel, was measured to triple the error against the FP64 oracle under motion:
// near restarts the taps' P differ by orders of magnitude). Round to nearest even on store (one
// cvt for two values), exact decode (BF16: a shift or a mask; FP16: the conversion of a
// half2); all arithmetic binary32. 13 words = 52 bytes per pixel and copy.
template <typename T>
struct State16 {
  uint32_t* base;
  size_t plane_stride;  // in words
  int pitch;
  static constexpr int kPlanes = 13;
  static __device__ __forceinline__ float2 unpack(uint32_t u);          // (low, high) as binary32
  static __device__ __forceinline__ uint32_t pack(float lo, float hi);  // round to nearest even
  static __device__ __forceinline__ float scale_of(uint32_t w12) {  // s = 2^e from word 12
    const int e = (int)(short)(w12 >> 16);
    return __int_as_float((e + 127) << 23);
  }
  // P / s = L L^T from the factor in slots 12-21 (in place).
  static __device__ __forceinline__ void chol_to_p(float v[kNState]) {
    const float l00 = v[kP + 0], l10 = v[kP + 1], l20 = v[kP + 2], l30 = v[kP + 3];
    const float l11 = v[kP + 4], l21 = v[kP + 5], l31 = v[kP + 6];
    const float l22 = v[kP + 7], l32 = v[kP + 8], l33 = v[kP + 9];
    v[kP + 0] = l00 * l00;
    v[kP + 1] = l10 * l00;
    v[kP + 2] = l20 * l00;
    v[kP + 3] = l30 * l00;
    v[kP + 4] = fmaf(l11, l11, l10 * l10);
    v[kP + 5] = fmaf(l21, l11, l20 * l10);
    v[kP + 6] = fmaf(l31, l11, l30 * l10);
    v[kP + 7] = fmaf(l22, l22, fmaf(l21, l21, l20 * l20));
    v[kP + 8] = fmaf(l32, l22, fmaf(l31, l21, l30 * l20));
    v[kP + 9] = fmaf(l33, l33, fmaf(l32, l32, fmaf(l31, l31, l30 * l30)));
  }
  // Cholesky factor of the 4 x 4 P (upper triangle a[0..9]) in place; a pivot <= 0 (P
  // singular in binary32 rounding, or an unused predictor entry) gives a zero column.
  static __device__ __forceinline__ void p_to_chol(float a[10]) {
    auto col = [](float piv, float& l, float& r) {
      if (piv > 0.0f) {
        r = rsqrtf(piv);
        l = piv * r;
      } else {
        l = 0.0f;
        r = 0.0f;
      }
    };
    float l00, r0, l11, r1, l22, r2, l33, r3;
    col(a[0], l00, r0);
    const float l10 = a[1] * r0, l20 = a[2] * r0, l30 = a[3] * r0;
    col(fmaf(-l10, l10, a[4]), l11, r1);
    const float l21 = fmaf(-l20, l10, a[5]) * r1, l31 = fmaf(-l30, l10, a[6]) * r1;
    col(fmaf(-l21, l21, fmaf(-l20, l20, a[7])), l22, r2);
    const float l32 = fmaf(-l31, l21, fmaf(-l30, l20, a[8])) * r2;
    col(fmaf(-l32, l32, fmaf(-l31, l31, fmaf(-l30, l30, a[9]))), l33, r3);
    (void)r3;
    a[0] = l00; a[1] = l10; a[2] = l20; a[3] = l30; a[4] = l11;
    a[5] = l21; a[6] = l31; a[7] = l22; a[8] = l32; a[9] = l33;
  }
  // beta, z and P / s (formed from the stored factor) in v; s.
  static __device__ __forceinline__ void decode(const uint32_t w[kPlanes], float v[kNState], float& s) {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float2 u = unpack(w[k]);
      v[2 * k] = u.x;
      v[2 * k + 1] = u.y;
    }
    v[24] = unpack(w[12]).x;
    s = scale_of(w[12]);
    chol_to_p(v);
  }
  __device__ __forceinline__ void load_raw(size_t idx, float v[kNState], float& s) const {
    uint32_t w[kPlanes];
#pragma unroll
    for (int k = 0; k < kPlanes; ++k) w[k] = __ldg(base + k * plane_stride + idx);
    decode(w, v, s);
  }
  __device__ __forceinline__ void load(size_t idx, float v[kNState]) const {
    float s;
    load_raw(idx, v, s);
#pragma unroll
    for (int p = kP; p < kZ; ++p) v[p] *= s;
  }
  __device__ __forceinline__ void load_beta_z(size_t idx, float b[12], float z[3]) const {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float2 f = unpack(__ldg(base + k * plane_stride + idx));
      b[2 * k] = f.x;
      b[2 * k + 1] = f.y;
    }
    const float2 z01 = unpack(__ldg(base + 11 * plane_stride + idx));
    z[0] = z01.x;
    z[1] = z01.y;
    z[2] = unpack(__ldg(base + 12 * plane_stride + idx)).x;
  }
  __device__ __forceinline__ void store(size_t idx, const float v[kNState]) const {
    const float m = fmaxf(fmaxf(v[kP + 0], v[kP + 4]), fmaxf(v[kP + 7], v[kP + 9]));
    int e = 0;
    if (m > 0.0f && m <= 3.402823466e38f) {
      const int f = ((__float_as_int(m) >> 23) & 0xff) - 126;  // m / 2^f in [0.5, 1) (normal m)
      e = min(max(f + (f & 1), -126), 126);
    }
    const float inv_s = __int_as_float((127 - e) << 23);
    float a[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) a[q] = v[kP + q] * inv_s;
    p_to_chol(a);
    const uint32_t i = (uint32_t)idx;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const int p = 2 * k;
      const float lo = (p >= kP && p < kZ) ? a[p - kP] : v[p];
      const float hi = (p + 1 >= kP && p + 1 < kZ) ? a[p + 1 - kP] : v[p + 1];
      (base + k * plane_stride)[i] = pack(lo, hi);
    }
    (base + 12 * plane_stride)[i] = (pack(v[24], 0.0f) & 0xffffu) | ((uint32_t)e << 16);
  }
  // Staged window: [word plane][kStageH][kStageW] 32-bit words; box origin x multiple of 4.
  static constexpr int kAlignX = 4;
  static constexpr uint32_t kStageBytes = kPlanes * kStagePix * 4;
  static constexpr uint32_t kTxBytes = kStageBytes;
  static constexpr bool kScaled = true;
  static __device__ __forceinline__ void load_staged(const unsigned char* stage, int idx, float v[kNState], float& s) {
    const uint32_t* u = (const uint32_t*)stage;
    uint32_t w[kPlanes];
#pragma unroll
    for (int k = 0; k < kPlanes; ++k) w[k] = u[k * kStagePix + idx];
    decode(w, v, s);
  }
};
template <>
__device__ __forceinline__ float2 State16<__nv_bfloat16>::unpack(uint32_t u) {
  return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));  // exact
}
template <>
__device__ __forceinline__ uint32_t State16<__nv_bfloat16>::pack(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);  // .x (low half) = lo
  return *reinterpret_cast<const uint32_t*>(&h);
}
template <>
__device__ __forceinline__ float2 State16<__half>::unpack(uint32_t u) {
  __half2 h;
  *reinterpret_cast<uint32_t*>(&h) = u;
  return __half22float2(h);
}
template <>
__device__ __forceinline__ uint32_t State16<__half>::pack(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

using StateBF16 = State16<__nv_bfloat16>;
using StateF16 = State16<__half>;

// ---- per-pixel temporal update ----------------------------------------------------------

// Initial model of a restarted pixel: beta = 0 (init_mode 0) or the feature pass-through
// beta_c = e_{c+1} (beta_c = z_c with p = [1]); P = p0_delta * I on the used block.
__device__ __forceinline__ void init_model(const KParams& kp, const float z[3], float st[kNState]) {
#pragma unroll
  for (int p = 0; p < 22; ++p) st[p] = 0.0f;
  if (kp.init_mode == 1) {
    if (kp.feature_mode == 0) {
      st[kBeta + 0 * 4 + 1] = 1.0f;
      st[kBeta + 1 * 4 + 2] = 1.0f;
      st[kBeta + 2 * 4 + 3] = 1.0f;
    } else {
      st[kBeta + 0] = z[0];
      st[kBeta + 4] = z[1];
      st[kBeta + 8] = z[2];
    }
  }
  st[kP + 0] = kp.p0_delta;
  if (kp.feature_mode == 0) {
    st[kP + 4] = kp.p0_delta;
    st[kP + 7] = kp.p0_delta;
    st[kP + 9] = kp.p0_delta;
  }
}

// Bilinear interpolation of every state value from its four taps in a fixed rounding order,
// st = ((w00 a + w10 b) + w01 c) + w11 d by fused multiply-adds; consecutive planes are taken in
// packed pairs (same rounding per component). bilerp_top takes the taps (x0, y0), (x1, y0),
// bilerp_bottom adds (x0, y1), (x1, y1). The P slots take their own weights: the tap weight
// times the tap's scale, a power of two (the products are exact, so this equals scaling the
// decoded values first).
__device__ __forceinline__ void bilerp_top(float w00, float w10, float q00, float q10, const float a[kNState],
                                           const float b[kNState], float st[kNState]) {
#pragma unroll
  for (int p = 0; p + 1 < kNState; p += 2) {
    const bool isP = p >= kP && p < kZ;
    const float2 wa = isP ? make_float2(q00, q00) : make_float2(w00, w00);
    const float2 wb = isP ? make_float2(q10, q10) : make_float2(w10, w10);
    const float2 v = f2fma(wb, make_float2(b[p], b[p + 1]), f2mul(wa, make_float2(a[p], a[p + 1])));
    st[p] = v.x;
    st[p + 1] = v.y;
  }
  if (kNState % 2) st[kNState - 1] = fmaf(w10, b[kNState - 1], w00 * a[kNState - 1]);
}
__device__ __forceinline__ void bilerp_bottom(float w01, float w11, float q01, float q11, const float c[kNState],
                                              const float d[kNState], float st[kNState]) {
#pragma unroll
  for (int p = 0; p + 1 < kNState; p += 2) {
    const bool isP = p >= kP && p < kZ;
    const float2 wc = isP ? make_float2(q01, q01) : make_float2(w01, w01);
    const float2 wd = isP ? make_float2(q11, q11) : make_float2(w11, w11);
    const float2 v = f2fma(wd, make_float2(d[p], d[p + 1]),
                           f2fma(wc, make_float2(c[p], c[p + 1]), make_float2(st[p], st[p + 1])));
    st[p] = v.x;
    st[p + 1] = v.y;
  }
  if (kNState % 2) st[kNState - 1] = fmaf(w11, d[kNState - 1], fmaf(w01, c[kNState - 1], st[kNState - 1]));
}

// One tap alone (the others have weight 0): st = w00 a.
__device__ __forceinline__ void bilerp_top1(float w00, float q00, const float a[kNState], float st[kNState]) {
#pragma unroll
  for (int p = 0; p + 1 < kNState; p += 2) {
    const bool isP = p >= kP && p < kZ;
    const float2 wa = isP ? make_float2(q00, q00) : make_float2(w00, w00);
    const float2 v = f2mul(wa, make_float2(a[p], a[p + 1]));
    st[p] = v.x;
    st[p + 1] = v.y;
  }
  if (kNState % 2) st[kNState - 1] = w00 * a[kNState - 1];
}

// P-slot weight of a tap: w times the tap's scale (binary32: the weight itself).
template <class SV>
__device__ __forceinline__ float scaled_weight(float w, float s) {
  if constexpr (SV::kScaled) return w * s;
  else return w;
}

// Bilinear fetch of the previous state at q = (qx, qy) (Sec. 5.3: models are reprojected,
// not colours). q is valid; taps beyond the last row/column are clamped.
template <class SV>
__device__ __forceinline__ void gather_bilinear(const SV& prev, int W, int H, float qx, float qy,
                                                float st[kNState]) {
  const int x0 = (int)floorf(qx), y0 = (int)floorf(qy);
  const float fx = qx - (float)x0, fy = qy - (float)y0;
  const int x1 = min(x0 + 1, W - 1), y1 = min(y0 + 1, H - 1);
  const float w00 = (1.0f - fx) * (1.0f - fy), w10 = fx * (1.0f - fy);
  const float w01 = (1.0f - fx) * fy, w11 = fx * fy;
  float a[kNState], b[kNState], sa, sb;
  prev.load_raw((size_t)y0 * prev.pitch + x0, a, sa);
  prev.load_raw((size_t)y0 * prev.pitch + x1, b, sb);
  bilerp_top(w00, w10, scaled_weight<SV>(w00, sa), scaled_weight<SV>(w10, sb), a, b, st);
  prev.load_raw((size_t)y1 * prev.pitch + x0, a, sa);
  prev.load_raw((size_t)y1 * prev.pitch + x1, b, sb);
  bilerp_bottom(w01, w11, scaled_weight<SV>(w01, sa), scaled_weight<SV>(w11, sb), a, b, st);
}

// Bilinear fetch from the staged window whose origin is (X0, Y0). TAPS = 4, or 2 (the lower
// row's weights are 0: fy = 0) or 1 (fx = fy = 0): taps of weight exactly 0 are not read. A
// tap of weight 0 adds fma(0, v, s) = s for a finite v, so the result is that of the four-tap
// sum (up to the sign of a zero).
template <class SV, int TAPS = 4>
__device__ __forceinline__ void gather_bilinear_staged(const unsigned char* stage, int X0, int Y0, int W,
                                                       int H, float qx, float qy, float st[kNState]) {
  const int x0 = (int)floorf(qx), y0 = (int)floorf(qy);
  const float fx = qx - (float)x0, fy = qy - (float)y0;
  const int x1 = min(x0 + 1, W - 1), y1 = min(y0 + 1, H - 1);
  const float w00 = (1.0f - fx) * (1.0f - fy), w10 = fx * (1.0f - fy);
  const float w01 = (1.0f - fx) * fy, w11 = fx * fy;
  const int r0 = (y0 - Y0) * kStageW, r1 = (y1 - Y0) * kStageW;
  float a[kNState], b[kNState], sa, sb;
  SV::load_staged(stage, r0 + x0 - X0, a, sa);
  if constexpr (TAPS == 1) {
    bilerp_top1(w00, scaled_weight<SV>(w00, sa), a, st);
    return;
  }
  SV::load_staged(stage, r0 + x1 - X0, b, sb);
  bilerp_top(w00, w10, scaled_weight<SV>(w00, sa), scaled_weight<SV>(w10, sb), a, b, st);
  if constexpr (TAPS == 2) return;
  SV::load_staged(stage, r1 + x0 - X0, a, sa);
  SV::load_staged(stage, r1 + x1 - X0, b, sb);
  bilerp_bottom(w01, w11, scaled_weight<SV>(w01, sa), scaled_weight<SV>(w11, sb), a, b, st);
}

// Eq. 12 feature, Eq. 13 weight and the wRLS update (Eq. 8, 14, 9, 11) of one pixel.
//   st     in: reprojected state (or anything if !valid); out: state of frame t
//   I      noisy sample I~_j(t); missing = a channel is non-finite
//   lo/hi  per-channel min/max of I~ over the 3x3 neighbours (have_box = any finite one)
// Returns w.
__device__ __forceinline__ float update_pixel(const KParams& kp, bool valid, float st[kNState],
                                              const float I[3], bool missing, const float lo[3],
                                              const float hi[3], bool have_box) {
  float z[3];
  if (valid) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float zc = st[kZ + c];
      if (kp.clamp_mode == 0 && have_box) zc = fminf(fmaxf(zc, lo[c]), hi[c]);
      z[c] = missing ? zc : fmaf(kp.alpha, zc, kp.one_m_alpha * I[c]);
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) z[c] = missing ? 0.0f : I[c];
    init_model(kp, z, st);
  }

  // Eq. 13 (one scalar per pixel over RGB); RLS mode: w = 1
  float w;
  if (missing) {
    w = 0.0f;
  } else if (kp.weight_mode == 1) {
    w = 1.0f;
  } else {
    const float d0 = I[0] - z[0], d1 = I[1] - z[1], d2 = I[2] - z[2];
    const float dist2 = d0 * d0 + d1 * d1 + d2 * d2;
    const float nI = sqrtf(I[0] * I[0] + I[1] * I[1] + I[2] * I[2]);
    const float nz = sqrtf(z[0] * z[0] + z[1] * z[1] + z[2] * z[2]);
    const float m = fminf(nI, nz) + kp.eps;
    w = ex2_approx(-(dist2 / (m * m)) * kp.w_k);
  }

  // predictor p = [1, z] (Sec. 5.1), or [1] without feature
  const float z0 = kp.feature_mode == 0 ? z[0] : 0.0f;
  const float z1 = kp.feature_mode == 0 ? z[1] : 0.0f;
  const float z2 = kp.feature_mode == 0 ? z[2] : 0.0f;
  float* P = st + kP;
  // k = P p
  const float k0 = P[0] + P[1] * z0 + P[2] * z1 + P[3] * z2;
  const float k1 = P[1] + P[4] * z0 + P[5] * z1 + P[6] * z2;
  const float k2 = P[2] + P[5] * z0 + P[7] * z1 + P[8] * z2;
  const float k3 = P[3] + P[6] * z0 + P[8] * z1 + P[9] * z2;
  const float s = k0 + k1 * z0 + k2 * z1 + k3 * z2;  // p^T P p
  // Eq. 14: q^w = P p / (lambda / w + p^T P p) = (w / (lambda + w s)) P p
  const float g = w / (kp.lambda + w * s);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float* b = st + kBeta + 4 * c;
    const float e = missing ? 0.0f : I[c] - (b[0] + b[1] * z0 + b[2] * z1 + b[3] * z2);  // Eq. 8
    const float ge = g * e;                                                            // Eq. 9
    b[0] += ge * k0;
    b[1] += ge * k1;
    b[2] += ge * k2;
    b[3] += ge * k3;
  }
  // Eq. 11: P <- (P - q^w p^T P) / lambda, with p^T P = k^T
  const float k[4] = {k0, k1, k2, k3};
  int e = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bb = a; bb < 4; ++bb, ++e) P[e] = (P[e] - g * k[a] * k[bb]) * kp.inv_lambda;
  if (kp.p_trace_max > 0.0f) {
    const bool f = kp.feature_mode == 0;
    const float tr = P[0] + (f ? P[4] + P[7] + P[9] : 0.0f);
    const bool bad = !(P[0] > 0.0f) || (f && (!(P[4] > 0.0f) || !(P[7] > 0.0f) || !(P[9] > 0.0f)));
    if (bad || tr > kp.p_trace_max) {
#pragma unroll
      for (int q = 0; q < 10; ++q) P[q] = 0.0f;
      P[0] = kp.p0_delta;
      if (f) { P[4] = kp.p0_delta; P[7] = kp.p0_delta; P[9] = kp.p0_delta; }
    }
  }
  st[kZ + 0] = z[0];
  st[kZ + 1] = z[1];
  st[kZ + 2] = z[2];
  return w;
}

}  // namespace wrls
