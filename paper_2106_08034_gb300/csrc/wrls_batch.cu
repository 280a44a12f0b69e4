// Batched tick: one frame of each of n streams (of any sizes) in one CUDA graph launch.
//
// wrls_batch_tick: the graph holds each stream's own update and blend
// kernels (those of wrls_denoise_frame, with their parameters in the constant bank and the
// stream's tuned blend tile), the streams' chains spread over kLanes parallel branches, so
// that one stream's arithmetic-bound blend runs while another stream's memory-bound update
// runs. The graph is captured every tick (input pointers and restart flags change) and
// applied to the instantiated graph with cudaGraphExecUpdate.
//
// wrls_batch_tick_static: the host writes a table (header + one FrameWork per frame, with
// each frame's first tile index) and persistent kernels pull (stream, tile) work items from
// it: a CTA takes the next tile with an atomicAdd on a work counter until the counter passes
// the total; no CTA ever waits on another.
//
// The tile bodies are those of the single-frame kernels, so every stream's output and
// state are bitwise identical to denoising it alone.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "wrls_internal.h"
#include "wrls_tiles.cuh"

namespace wrls {

constexpr int kDenoiseBatchMax = 256;  // frames per wrls_denoise_batch call
constexpr int kMaxDevices = 64;         // devices with a wrls_denoise_batch executor

struct alignas(128) FrameWork {
  StageMaps maps;    // TMA tensor maps of the previous state copy
  KParams kp;
  void* prev_base;
  void* next_base;
  size_t plane_stride;
  const float* rad;
  const float* mot;
  float* out;
  int* err;          // the stream's device error word
  int stage_ok;
  int pitch;
  int W, H;
  int reset;
  int tiles_x;       // tiles per row (32 pixels wide, both phases)
  int begin_update;  // first work item of this frame in the update list (32 x 8 tiles)
  int begin_blend;   // first work item of this frame in the blend list (32 x TH tiles)
};

struct alignas(128) BatchHeader {
  int n;
  int total_update;
  int total_blend;
};

template <class SV> __device__ __forceinline__ SV make_view(void* base, size_t ps, int pitch);
template <> __device__ __forceinline__ StateF32 make_view<StateF32>(void* base, size_t ps, int pitch) {
  return StateF32{(float*)base, ps, pitch};
}
template <> __device__ __forceinline__ StateBF16 make_view<StateBF16>(void* base, size_t ps, int pitch) {
  return StateBF16{(uint32_t*)base, ps, pitch};
}
template <> __device__ __forceinline__ StateF16 make_view<StateF16>(void* base, size_t ps, int pitch) {
  return StateF16{(uint32_t*)base, ps, pitch};
}

// Claim the next work item of a list; returns its tile index within its frame (or -1 when
// the list is exhausted) and the frame in *frame.
// Lists: 0 = update tiles, 1 = blend tiles.
template <int LIST>
__device__ __forceinline__ int list_begin(const FrameWork& w) {
  return LIST == 0 ? w.begin_update : w.begin_blend;
}

template <int LIST>
__device__ __forceinline__ int next_item(const BatchHeader* __restrict__ hdr,
                                         const FrameWork* __restrict__ fw, int* counter,
                                         int* s_item, int* s_frame, int* frame) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const int t = atomicAdd(counter, 1);
    const int total = LIST == 0 ? hdr->total_update : hdr->total_blend;
    int f = -1;
    if (t < total) {
      int lo = 0, hi = hdr->n - 1;  // last frame whose list begins at or before t
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (list_begin<LIST>(fw[mid]) <= t) lo = mid; else hi = mid - 1;
      }
      f = lo;
    }
    *s_item = t;
    *s_frame = f;
  }
  __syncthreads();
  *frame = *s_frame;
  if (*frame < 0) return -1;
  return *s_item - list_begin<LIST>(fw[*frame]);
}

// The tensor maps live in the work table (global memory written by a copy before the launch):
// acquire them for the tensormap proxy before the first bulk copy that uses them.
__device__ __forceinline__ void acquire_tensormap(const CUtensorMap* m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)m) : "memory");
}

template <class SV>
__global__ void __launch_bounds__(kTileThreads, SV::kScaled ? 6 : 5)  // as k_update
    k_batch_update(const BatchHeader* __restrict__ hdr, const FrameWork* __restrict__ fw, int* counters) {
  extern __shared__ unsigned char dsmem[];
  UpdateSmem<SV>& sm = *reinterpret_cast<UpdateSmem<SV>*>(align128(dsmem));
  __shared__ int s_item, s_frame;
  __shared__ alignas(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  uint32_t phase = 0;
  for (;;) {
    int f;
    const int lt = next_item<0>(hdr, fw, counters + 0, &s_item, &s_frame, &f);
    if (lt < 0) break;
    const FrameWork& w = fw[f];
    if (threadIdx.x == 0 && w.stage_ok) acquire_tensormap(&w.maps.planes);
    const SV prev = make_view<SV>(w.prev_base, w.plane_stride, w.pitch);
    const SV next = make_view<SV>(w.next_base, w.plane_stride, w.pitch);
    if (!update_tile(sm, &bar, phase, w.err, w.kp, w.W, w.H, w.reset != 0, w.stage_ok != 0, prev, next,
                     &w.maps, w.rad, w.mot, (lt % w.tiles_x) * kTW, (lt / w.tiles_x) * kTH))
      return;
  }
}

template <class SV, int TH, int R, int MODE>
__global__ void __launch_bounds__(kTW * TH / R)
    k_batch_blend(const BatchHeader* __restrict__ hdr, const FrameWork* __restrict__ fw, int* counters) {
  extern __shared__ float4 sm_blend[];
  __shared__ int s_item, s_frame;
  for (;;) {
    int f;
    const int lt = next_item<1>(hdr, fw, counters + 1, &s_item, &s_frame, &f);
    if (lt < 0) break;
    const FrameWork& w = fw[f];
    const SV cur = make_view<SV>(w.next_base, w.plane_stride, w.pitch);
    blend_tile<SV, TH, R, MODE>(sm_blend, w.kp, w.W, w.H, cur, w.out, (lt % w.tiles_x) * kTW,
                                (lt / w.tiles_x) * TH);
  }
}

static int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

static int blend_rows(int cfg) {
  switch (cfg) {
    case 1: return 8;
    case 3: return 32;
    default: return 16;
  }
}

}  // namespace wrls

using namespace wrls;

struct wrls_batch {
  int max_streams = 0;
  cudaStream_t cs = nullptr;
  cudaStream_t cap = nullptr;
  static constexpr int kLanes = 4;          // parallel branches of the per-stream tick graph
  cudaStream_t lane[kLanes] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kLanes] = {};
  cudaGraphExec_t exec_chains = nullptr;    // the per-stream tick graph
  std::vector<int> order;                   // frames by pixel count, largest first
  int device = 0;
};

static void batch_free(wrls_batch* b) {
  if (b->cap) cudaStreamDestroy(b->cap);
  for (int k = 0; k < wrls_batch::kLanes; ++k) {
    if (b->lane[k]) cudaStreamDestroy(b->lane[k]);
    if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->exec_chains) cudaGraphExecDestroy(b->exec_chains);
  cudaGetLastError();
  delete b;
}

// Two-kernel tick: a CUDA graph of each stream's own update and blend kernels, the streams'
// chains spread over kLanes parallel branches. Captured every tick and applied to the
// instantiated graph with cudaGraphExecUpdate (a new instantiation when the shape changed).
static wrls_status tick_chains(wrls_batch* b, const wrls_frame_io* frames, int n) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("wrls_batch_tick: begin capture: %s", cudaGetErrorString(e));
    return WRLS_ERR_CUDA;
  }
  e = cudaEventRecord(b->ev_fork, b->cap);
  const int lanes = n < wrls_batch::kLanes ? n : wrls_batch::kLanes;
  for (int k = 0; k < lanes && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->lane[k], b->ev_fork, 0);
  // Largest frame first, each to the branch with the fewest pixels so far, so that the
  // branches carry similar work and each ends with its smallest kernels.
  std::vector<int>& order = b->order;
  order.resize(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  auto px = [&](int i) { return (long long)frames[i].stream->W * frames[i].stream->H; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return px(a) > px(c); });
  long long load[wrls_batch::kLanes] = {};
  for (int j = 0; j < n && e == cudaSuccess; ++j) {
    const int i = order[j];
    int k = 0;
    for (int m = 1; m < lanes; ++m)
      if (load[m] < load[k]) k = m;
    load[k] += px(i);
    wrls_stream* s = frames[i].stream;
    cudaStream_t ln = b->lane[k];
    const StateDesc& prev = s->state[s->cur];
    const StateDesc& next = s->state[next_copy(s)];
    e = launch_update(s->kp, prev, next, s->need_reset, frames[i].radiance, frames[i].motion, s->err, ln);
    if (e == cudaSuccess) e = launch_blend(s->kp, s->blend_cfg, next, frames[i].out, s->err, ln);
  }
  for (int k = 0; k < lanes && e == cudaSuccess; ++k) {
    e = cudaEventRecord(b->ev_join[k], b->lane[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->ev_join[k], 0);
  }
  const cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
  if (e == cudaSuccess) e = ee;
  if (e == cudaSuccess && b->exec_chains) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(b->exec_chains, g, &info) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(b->exec_chains);
      b->exec_chains = nullptr;
    }
  }
  if (e == cudaSuccess && !b->exec_chains) e = cudaGraphInstantiate(&b->exec_chains, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec_chains, b->cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("wrls_batch_tick: %s", cudaGetErrorString(e));
    return WRLS_ERR_CUDA;
  }
  for (int i = 0; i < n; ++i) {
    wrls_stream* s = frames[i].stream;
    s->cur = next_copy(s);
    s->need_reset = false;
    s->has_frame = true;
    s->frames++;
  }
  return WRLS_OK;
}

extern "C" {

wrls_status wrls_batch_create(int max_streams, wrls_batch** out) {
  if (!out) { set_error("wrls_batch_create: out is NULL"); return WRLS_ERR_INVALID_ARG; }
  *out = nullptr;
  if (max_streams < 1 || max_streams > 4096) {
    set_error("wrls_batch_create: max_streams %d outside [1, 4096]", max_streams);
    return WRLS_ERR_INVALID_ARG;
  }
  wrls_batch* b = new (std::nothrow) wrls_batch();
  if (!b) { set_error("wrls_batch_create: host allocation failed"); return WRLS_ERR_OOM; }
  b->max_streams = max_streams;
  try {
    b->order.reserve(max_streams);  // the ticks resize within this capacity: no allocation
  } catch (...) {
    delete b;
    set_error("wrls_batch_create: host allocation failed");
    return WRLS_ERR_OOM;
  }
  cudaGetDevice(&b->device);
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  for (int k = 0; k < wrls_batch::kLanes && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&b->lane[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    set_error("wrls_batch_create: %s", cudaGetErrorString(e));
    wrls_status st = e == cudaErrorMemoryAllocation ? WRLS_ERR_OOM : WRLS_ERR_CUDA;
    batch_free(b);
    return st;
  }
  *out = b;
  return WRLS_OK;
}

wrls_status wrls_batch_set_cuda_stream(wrls_batch* b, void* cuda_stream) {
  if (!b) { set_error("wrls_batch_set_cuda_stream: batch is NULL"); return WRLS_ERR_INVALID_ARG; }
  b->cs = (cudaStream_t)cuda_stream;
  return WRLS_OK;
}

wrls_status wrls_batch_tick(wrls_batch* b, const wrls_frame_io* frames, int n) {
  NvtxRange nvtx("wrls_batch_tick");
  if (!b || !frames) { set_error("wrls_batch_tick: NULL argument"); return WRLS_ERR_INVALID_ARG; }
  if (n < 1 || n > b->max_streams) {
    set_error("wrls_batch_tick: n = %d outside [1, %d]", n, b->max_streams);
    return WRLS_ERR_INVALID_ARG;
  }
  const int prec = frames[0].stream ? frames[0].stream->prm.state_precision : -1;
  const int mode = frames[0].stream ? frames[0].stream->prm.blend_mode : -1;
  for (int i = 0; i < n; ++i) {
    const wrls_frame_io& io = frames[i];
    if (!io.stream || !io.radiance || !io.motion || !io.out) {
      set_error("wrls_batch_tick: frame %d has a NULL stream, radiance, motion or out", i);
      return WRLS_ERR_INVALID_ARG;
    }
    if (((uintptr_t)io.radiance | (uintptr_t)io.motion | (uintptr_t)io.out) & 3u) {
      set_error("wrls_batch_tick: frame %d buffers must be 4-byte aligned", i);
      return WRLS_ERR_INVALID_ARG;
    }
    if (io.stream->prm.state_precision != prec || io.stream->prm.blend_mode != mode) {
      set_error("wrls_batch_tick: all streams of a tick must share one state precision and blend mode");
      return WRLS_ERR_INVALID_ARG;
    }
    if (io.stream->ext) {
      set_error("wrls_batch_tick: streams on the extended path (G-buffer predictor, variance weight, "
                "nearest reprojection) are not batched");
      return WRLS_ERR_INVALID_ARG;
    }
    for (int k = 0; k < i; ++k)
      if (frames[k].stream == io.stream) {
        set_error("wrls_batch_tick: stream of frame %d appears twice", i);
        return WRLS_ERR_INVALID_ARG;
      }
  }
  return tick_chains(b, frames, n);
}

wrls_status wrls_denoise_batch(wrls_stream* const* streams, const wrls_frame_io* io, int n) {
  NvtxRange nvtx("wrls_denoise_batch");
  if (!streams || !io || n < 1 || n > kDenoiseBatchMax) {
    set_error("wrls_denoise_batch: NULL argument or n = %d outside [1, %d]", n, kDenoiseBatchMax);
    return WRLS_ERR_INVALID_ARG;
  }
  wrls_frame_io* fr = new (std::nothrow) wrls_frame_io[n];
  if (!fr) {
    set_error("wrls_denoise_batch: host allocation failed");
    return WRLS_ERR_OOM;
  }
  for (int i = 0; i < n; ++i) {
    if (!streams[i] || (io[i].stream && io[i].stream != streams[i])) {
      delete[] fr;
      set_error("wrls_denoise_batch: frame %d: NULL stream, or io.stream differs from streams[%d]", i, i);
      return WRLS_ERR_INVALID_ARG;
    }
    fr[i] = io[i];
    fr[i].stream = streams[i];
  }
  // one executor per device, created on first use and kept until the process exits
  static std::mutex mu;
  static wrls_batch* executors[kMaxDevices] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  wrls_status st = WRLS_OK;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= kMaxDevices) {
      set_error("wrls_denoise_batch: device %d beyond the executor table", dev);
      st = WRLS_ERR_INVALID_ARG;
    } else {
      if (!executors[dev]) st = wrls_batch_create(kDenoiseBatchMax, &executors[dev]);
      if (st == WRLS_OK) st = wrls_batch_set_cuda_stream(executors[dev], (void*)streams[0]->cs);
      if (st == WRLS_OK) st = wrls_batch_tick(executors[dev], fr, n);
    }
  }
  delete[] fr;
  return st;
}

void wrls_batch_destroy(wrls_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->cs);
  batch_free(b);
}

}  // extern "C"

// ---- wrls_batch_tick_static: the batched tick without any device allocation -------------
//
// For callers that cannot allocate device memory (see include/wrls.h). The work table and
// the two work counters live in the file-scope array below instead of cudaMalloc'ed memory.
// Host code must not pass the array's name to a kernel (on the host it names a stand-in, not
// device memory): its device address is looked up once per device with
// cudaGetSymbolAddress, on the first call made with that device current, and cached. The host
// builds the table on its stack and hands it to k_static_fill by value (a kernel parameter),
// which writes it into the array and clears the counters: no host buffer is read after the
// call returns and no pageable copy is made.

constexpr int kStaticBatchMax = WRLS_STATIC_BATCH_MAX;  // frames per call
static_assert(kStaticBatchMax == 16, "the documented size of the static array assumes 16 frames");
constexpr size_t kStaticTableBytes = sizeof(BatchHeader) + kStaticBatchMax * sizeof(FrameWork);
constexpr size_t kStaticCountersOffset = (kStaticTableBytes + 255) / 256 * 256;
constexpr size_t kStaticScratchBytes = 10752;  // the size the header states
static_assert(kStaticCountersOffset + 2 * sizeof(int) <= kStaticScratchBytes, "table and counters exceed the array");
static_assert(kStaticTableBytes % 16 == 0, "the fill kernel copies 16-byte words");
static_assert(kStaticTableBytes <= 32000, "the table is passed as one kernel parameter");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct alignas(16) StaticTable {
  unsigned char bytes[kStaticTableBytes];
};

// Copy the host-built table (a kernel parameter) into the static array at `scratch` and clear
// the two work counters; then release the tensor maps in the table to the tensormap proxy
// (the batch kernels acquire them before their first bulk copy).
__global__ void __launch_bounds__(256) k_static_fill(const __grid_constant__ StaticTable tab, const int nbytes,
                                                     unsigned char* __restrict__ scratch) {
  const uint4* src = reinterpret_cast<const uint4*>(tab.bytes);
  uint4* dst = reinterpret_cast<uint4*>(scratch);
  for (int i = threadIdx.x; i < nbytes / 16; i += blockDim.x) dst[i] = src[i];
  if (threadIdx.x == 0) {
    int* counters = reinterpret_cast<int*>(scratch + kStaticCountersOffset);
    counters[0] = 0;
    counters[1] = 0;
  }
  asm volatile("fence.proxy.tensormap::generic.release.gpu;" ::: "memory");
}

static std::mutex g_static_mu;
static void* g_static_addr[256] = {};  // device address of g_static_scratch per device ordinal

static wrls_status static_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256) {
    set_error("wrls_batch_tick_static: no usable current device");
    return WRLS_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress((void**)&ptr, g_static_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      set_error("wrls_batch_tick_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return WRLS_ERR_CUDA;
    }
    g_static_addr[dev] = ptr;
  }
  *out = g_static_addr[dev];
  return WRLS_OK;
}

template <class SV, int TH, int R, int MODE>
static cudaError_t launch_static_cfg(cudaStream_t cs, void* d_table, int* d_counters) {
  constexpr int sbytes = BlendGeom<TH>::kSmemBytes;
  constexpr int ubytes = update_smem_bytes<SV>();
  constexpr int nt = kTW * TH / R;
  cudaError_t e = cudaFuncSetAttribute(k_batch_blend<SV, TH, R, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, sbytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_batch_update<SV>, cudaFuncAttributeMaxDynamicSharedMemorySize, ubytes);
  if (e != cudaSuccess) return e;
  int ou = 0, ob = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ou, k_batch_update<SV>, kTileThreads, ubytes);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ob, k_batch_blend<SV, TH, R, MODE>, nt, sbytes);
  if (e != cudaSuccess) return e;
  const int sms = sm_count();
  const BatchHeader* hdr = (const BatchHeader*)d_table;
  const FrameWork* fw = (const FrameWork*)((char*)d_table + sizeof(BatchHeader));
  k_batch_update<SV><<<sms * (ou > 0 ? ou : 1), kTileThreads, ubytes, cs>>>(hdr, fw, d_counters);
  k_batch_blend<SV, TH, R, MODE><<<sms * (ob > 0 ? ob : 1), nt, sbytes, cs>>>(hdr, fw, d_counters);
  return cudaGetLastError();
}

template <class SV, int MODE>
static cudaError_t launch_static_mode(int cfg, cudaStream_t cs, void* d_table, int* d_counters) {
  switch (cfg) {
    case 0: return launch_static_cfg<SV, 16, 4, MODE>(cs, d_table, d_counters);
    case 1: return launch_static_cfg<SV, 8, 4, MODE>(cs, d_table, d_counters);
    case 2: return launch_static_cfg<SV, 16, 2, MODE>(cs, d_table, d_counters);
    case 3: return launch_static_cfg<SV, 32, 4, MODE>(cs, d_table, d_counters);
  }
  return cudaErrorInvalidValue;
}

template <class SV>
static cudaError_t launch_static(int mode, int cfg, cudaStream_t cs, void* d_table, int* d_counters) {
  return mode == 0 ? launch_static_mode<SV, 0>(cfg, cs, d_table, d_counters)
                   : launch_static_mode<SV, 1>(cfg, cs, d_table, d_counters);
}

extern "C" wrls_status wrls_batch_tick_static(const wrls_frame_io* frames, int n, void* cuda_stream) {
  if (!frames) { set_error("wrls_batch_tick_static: frames is NULL"); return WRLS_ERR_INVALID_ARG; }
  if (n < 1 || n > kStaticBatchMax) {
    set_error("wrls_batch_tick_static: n = %d frames outside [1, %d] (the static work table holds at most %d)",
              n, kStaticBatchMax, kStaticBatchMax);
    return WRLS_ERR_INVALID_ARG;
  }
  const int prec = frames[0].stream ? frames[0].stream->prm.state_precision : -1;
  const int mode = frames[0].stream ? frames[0].stream->prm.blend_mode : -1;
  for (int i = 0; i < n; ++i) {
    const wrls_frame_io& io = frames[i];
    if (!io.stream || !io.radiance || !io.motion || !io.out) {
      set_error("wrls_batch_tick_static: frame %d has a NULL stream, radiance, motion or out", i);
      return WRLS_ERR_INVALID_ARG;
    }
    if (((uintptr_t)io.radiance | (uintptr_t)io.motion | (uintptr_t)io.out) & 3u) {
      set_error("wrls_batch_tick_static: frame %d buffers must be 4-byte aligned", i);
      return WRLS_ERR_INVALID_ARG;
    }
    if (io.stream->prm.state_precision != prec || io.stream->prm.blend_mode != mode) {
      set_error("wrls_batch_tick_static: all streams of a call must share one state precision and blend mode");
      return WRLS_ERR_INVALID_ARG;
    }
    if (io.stream->ext) {
      set_error("wrls_batch_tick_static: streams on the extended path are not batched");
      return WRLS_ERR_INVALID_ARG;
    }
    for (int k = 0; k < i; ++k)
      if (frames[k].stream == io.stream) {
        set_error("wrls_batch_tick_static: stream of frame %d appears twice", i);
        return WRLS_ERR_INVALID_ARG;
      }
  }
  void* scratch = nullptr;
  wrls_status st = static_scratch_address(&scratch);
  if (st != WRLS_OK) return st;
  int cfg = 0;
  size_t most = 0;
  for (int i = 0; i < n; ++i) {
    const size_t px = (size_t)frames[i].stream->W * frames[i].stream->H;
    if (px > most) { most = px; cfg = blend_sync_config(frames[i].stream->blend_cfg); }
  }
  const int th_b = blend_rows(cfg);
  // The table is built on the stack and passed by value to k_static_fill: the launch copies
  // the parameter, so the stack buffer may go out of scope when the call returns.
  StaticTable host_table;
  memset(&host_table, 0, sizeof(host_table));
  BatchHeader* hdr = (BatchHeader*)host_table.bytes;
  FrameWork* fw = (FrameWork*)(host_table.bytes + sizeof(BatchHeader));
  int tiles_u = 0, tiles_b = 0;
  for (int i = 0; i < n; ++i) {
    wrls_stream* s = frames[i].stream;
    const StateDesc& pv = s->state[s->cur];
    const StateDesc& nx = s->state[next_copy(s)];
    FrameWork& w = fw[i];
    w.maps = pv.maps;
    w.stage_ok = pv.stage_ok ? 1 : 0;
    w.err = s->err;
    w.kp = s->kp;
    w.prev_base = pv.base;
    w.next_base = nx.base;
    w.plane_stride = pv.plane_stride;
    w.rad = frames[i].radiance;
    w.mot = frames[i].motion;
    w.out = frames[i].out;
    w.pitch = pv.pitch;
    w.W = s->W;
    w.H = s->H;
    w.reset = s->need_reset ? 1 : 0;
    w.tiles_x = (s->W + kTW - 1) / kTW;
    w.begin_update = tiles_u;
    w.begin_blend = tiles_b;
    tiles_u += w.tiles_x * ((s->H + kTH - 1) / kTH);
    tiles_b += w.tiles_x * ((s->H + th_b - 1) / th_b);
  }
  hdr->n = n;
  hdr->total_update = tiles_u;
  hdr->total_blend = tiles_b;
  cudaStream_t cs = (cudaStream_t)cuda_stream;
  int* counters = (int*)((unsigned char*)scratch + kStaticCountersOffset);
  const int bytes = (int)(sizeof(BatchHeader) + (size_t)n * sizeof(FrameWork));
  k_static_fill<<<1, 256, 0, cs>>>(host_table, (bytes + 15) / 16 * 16, (unsigned char*)scratch);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    switch (prec) {
      case 0: e = launch_static<StateF32>(mode, cfg, cs, scratch, counters); break;
      case 1: e = launch_static<StateBF16>(mode, cfg, cs, scratch, counters); break;
      default: e = launch_static<StateF16>(mode, cfg, cs, scratch, counters); break;
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("wrls_batch_tick_static: %s", cudaGetErrorString(e));
    return WRLS_ERR_CUDA;
  }
  for (int i = 0; i < n; ++i) {
    wrls_stream* s = frames[i].stream;
    s->cur = next_copy(s);
    s->need_reset = false;
    s->has_frame = true;
    s->frames++;
  }
  return WRLS_OK;
}
