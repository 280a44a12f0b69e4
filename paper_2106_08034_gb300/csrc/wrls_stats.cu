// State health of a stream: the covariance wind-up that the optional reset guard (p_trace_max)
// bounds, positive definiteness of P, and non-finite values anywhere in the state. One pass
// over the current state copy; per-warp reductions, then one atomic per warp and quantity.
#include <string.h>

#include "wrls_internal.h"

namespace wrls {

struct StatsAcc {
  unsigned long long nonfinite;
  double trace_sum;
  unsigned int trace_max;  // order-preserving encodings of binary32 values
  unsigned int diag_min;
};

// Monotone map of binary32 bit patterns to unsigned integers (for atomicMax / atomicMin).
__device__ __forceinline__ unsigned int order_enc(float f) {
  const unsigned int b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// One pixel's contribution: v holds the state values, P its upper triangle of a d x d matrix
// starting at plane p0 (row by row), `used` the leading block that the predictor uses.
__device__ __forceinline__ void stats_pixel(const float* v, int nvals, int p0, int d, int used, bool in,
                                            StatsAcc* acc) {
  unsigned int nf = 0;
  float tr = 0.0f, dmin = INFINITY;
  if (in) {
    for (int p = 0; p < nvals; ++p) nf += isfinite(v[p]) ? 0u : 1u;
    int e = p0;
    for (int a = 0; a < d; ++a) {
      if (a < used) {
        tr += v[e];
        dmin = fminf(dmin, v[e]);
      }
      e += d - a;  // next diagonal entry of the row-by-row upper triangle
    }
  }
  const unsigned int m = 0xffffffffu;
  nf = __reduce_add_sync(m, nf);
  const unsigned int tmax = __reduce_max_sync(m, in ? order_enc(tr) : 0u);
  const unsigned int dm = __reduce_min_sync(m, in ? order_enc(dmin) : 0xffffffffu);
  double s = in ? (double)tr : 0.0;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(m, s, o);
  if ((threadIdx.x & 31) == 0) {
    if (nf) atomicAdd(&acc->nonfinite, (unsigned long long)nf);
    atomicAdd(&acc->trace_sum, s);
    atomicMax(&acc->trace_max, tmax);
    atomicMin(&acc->diag_min, dm);
  }
}

template <class SV>
__global__ void k_state_stats(const int W, const int H, const SV cur, const int used, StatsAcc* acc) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  const bool in = x < W;
  float v[kNState];
  if (in) cur.load((size_t)y * cur.pitch + x, v);
  stats_pixel(v, kNState, kP, 4, used, in, acc);
}

template <int NP>
__global__ void k_state_stats_ext(const int W, const int H, const float* __restrict__ base, const int pitch,
                                  const size_t ps, const int nvals, const int p0, const int d, const int used,
                                  StatsAcc* acc) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  const bool in = x < W;
  float v[NP];
  if (in)
    for (int p = 0; p < nvals; ++p) v[p] = base[p * ps + (size_t)y * pitch + x];
  stats_pixel(v, nvals, p0, d, used, in, acc);
}

}  // namespace wrls

using namespace wrls;

extern "C" wrls_status wrls_stream_state_stats(wrls_stream* s, wrls_state_stats* out) {
  NvtxRange nvtx("wrls_stream_state_stats");
  if (!s || !out) { set_error("wrls_stream_state_stats: NULL argument"); return WRLS_ERR_INVALID_ARG; }
  if (!s->has_frame) { set_error("wrls_stream_state_stats: no frame denoised yet"); return WRLS_ERR_STATE; }
  if (!s->stats) {
    if (cudaMalloc(&s->stats, sizeof(StatsAcc)) != cudaSuccess) {
      cudaGetLastError();
      s->stats = nullptr;
      set_error("wrls_stream_state_stats: device allocation failed");
      return WRLS_ERR_OOM;
    }
  }
  StatsAcc* acc = (StatsAcc*)s->stats;
  StatsAcc init{};
  init.trace_max = 0u;
  init.diag_min = 0xffffffffu;
  const StateDesc& cur = s->state[s->cur];
  const dim3 grid((s->W + 127) / 128, s->H);
  WRLS_CHECK_CUDA(cudaMemcpyAsync(acc, &init, sizeof(init), cudaMemcpyHostToDevice, s->cs),
                  "wrls_stream_state_stats: reset");
  if (s->ext) {
    const int d = s->dim, nvals = cur.nplanes;
    const int used = d;  // every entry of the extended predictor is used
    k_state_stats_ext<64><<<grid, 128, 0, s->cs>>>(s->W, s->H, (const float*)cur.base, cur.pitch, cur.plane_stride,
                                                    nvals, 3 * d, d, used, acc);
  } else {
    const int used = s->prm.feature_mode == 0 ? 4 : 1;
    switch (cur.precision) {
      case 0: k_state_stats<<<grid, 128, 0, s->cs>>>(s->W, s->H, cur.f32(), used, acc); break;
      case 1: k_state_stats<<<grid, 128, 0, s->cs>>>(s->W, s->H, cur.bf16(), used, acc); break;
      default: k_state_stats<<<grid, 128, 0, s->cs>>>(s->W, s->H, cur.f16(), used, acc); break;
    }
  }
  WRLS_CHECK_CUDA(cudaGetLastError(), "wrls_stream_state_stats: launch");
  StatsAcc h{};
  WRLS_CHECK_CUDA(cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, s->cs), "wrls_stream_state_stats: read");
  WRLS_CHECK_CUDA(cudaStreamSynchronize(s->cs), "wrls_stream_state_stats: synchronise");
  auto dec = [](unsigned int u) {
    const unsigned int b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
    memcpy(&f, &b, sizeof(f));
    return (double)f;
  };
  out->frames = s->frames;
  out->p_trace_max = dec(h.trace_max);
  out->p_trace_mean = h.trace_sum / ((double)s->W * s->H);
  out->p_diag_min = dec(h.diag_min);
  out->nonfinite = h.nonfinite;
  return WRLS_OK;
}
