// Shared device/host helpers of the hef library (internal header).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <mutex>
#include <unordered_map>

#include <nvtx3/nvToolsExt.h>

#include "../../include/hef.h"

namespace hef {

// ---------------------------------------------------------------------------
// host-side error reporting (thread-local message, see hef_last_error)

hef_status set_error(hef_status s, const char* fmt, ...);

#define HEF_CHECK_CUDA(call)                                                  \
  do {                                                                        \
    cudaError_t err_ = (call);                                                \
    if (err_ != cudaSuccess)                                                  \
      return ::hef::set_error(HEF_ERR_CUDA, "%s failed: %s (%s:%d)", #call,   \
                              cudaGetErrorString(err_), __FILE__, __LINE__);  \
  } while (0)

#define HEF_CHECK_LAUNCH() HEF_CHECK_CUDA(cudaGetLastError())

// Raise a kernel's dynamic shared-memory limit to `bytes` (once per kernel,
// device and size).
hef_status ensure_smem(const void* func, int bytes);
#define HEF_ENSURE_SMEM(func, bytes)                                              \
  do {                                                                            \
    hef_status s_ = ::hef::ensure_smem(reinterpret_cast<const void*>(func), (int)(bytes)); \
    if (s_ != HEF_OK) return s_;                                                  \
  } while (0)

// Launch accounting and optional CUDA-event timing of selected kernels (see
// hef_launch_count / hef_trace_kernels in hef.h).  Every kernel launch of the
// library goes through HEF_LAUNCH(name, stream, kernel<<<...>>>(...)).
struct LaunchTrace {
  int slot;
  LaunchTrace(const char* name, cudaStream_t st);
  ~LaunchTrace();
  cudaStream_t st;
};

#define HEF_LAUNCH(name, st, ...)                 \
  do {                                            \
    ::hef::LaunchTrace hef_lt_((name), (st));     \
    __VA_ARGS__;                                  \
  } while (0)

// NVTX range around a C-ABI call, named for the step of the method it runs
// (header-only NVTX: a no-op unless a profiler is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define HEF_NVTX(name) ::hef::NvtxRange hef_nvtx_(name)

// Bounds checks of the debugging build (-DHEF_DEBUG=1): dbg_index(i, lim,
// status) returns i when 0 <= i < lim; otherwise it sets HEF_BOUNDS in the
// incidence's status word and returns 0, so the access stays inside its
// array.  In the regular build it returns i unchecked.
#ifndef HEF_DEBUG
#define HEF_DEBUG 0
#endif
__device__ __forceinline__ int dbg_index(int i, int lim, const unsigned int* status) {
#if HEF_DEBUG
  if ((unsigned int)i >= (unsigned int)lim) {
    atomicOr(const_cast<unsigned int*>(status), HEF_BOUNDS);
    return 0;
  }
#else
  (void)lim;
  (void)status;
#endif
  return i;
}

constexpr int kThreads = 256;

// Programmatic dependent launch (sm_90 and later).  A kernel launched by
// launch_dependent() may be scheduled while the previous kernel of its stream
// drains; it calls pdl_wait() before its first access to memory that an
// earlier kernel writes or reads (the wait returns once the previous grid has
// completed and its writes are visible; it is a no-op for a kernel launched
// without the attribute), and pdl_trigger() after that wait, which lets the
// next such kernel be scheduled.  Triggering only after the wait keeps the
// order transitive: when kernel i+1 starts, kernel i-1 has completed.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent_smem(void (*kernel)(KArgs...), unsigned grid, unsigned block,
                                         size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Cooperative launch: the runtime starts the grid only with every CTA
// resident at once (or refuses a grid that can never be), which is what a
// kernel with grid-wide barriers needs when other work shares the GPU.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_cooperative_smem(void (*kernel)(KArgs...), unsigned grid, unsigned block,
                                           size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kernel)(KArgs...), unsigned grid, unsigned block,
                                    cudaStream_t st, Args... args) {
  return launch_dependent_smem(kernel, grid, block, 0, st, args...);
}

inline int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  return sms;
}

// Grid for a grid-stride loop over `work` items: at most `per_sm` CTAs of
// kThreads per SM (a fixed size, so per-CTA partial sums are reproducible).
// CTAs of `kernel` (with `threads` threads and `smem` dynamic shared memory)
// that fit on one SM at once, looked up once per kernel.
template <typename F>
inline int resident_ctas(F* kernel, int threads, size_t smem = 0) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(reinterpret_cast<const void*>(kernel));
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess ||
      n < 1)
    n = 1;
  cache[reinterpret_cast<const void*>(kernel)] = n;
  return n;
}

inline int stride_grid(long long work, int per_sm = 4) {
  long long want = (work + kThreads - 1) / kThreads;
  long long cap = (long long)num_sms() * per_sm;
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

// ---------------------------------------------------------------------------
// workspace carving: a bump allocator over a caller buffer.  With base ==
// nullptr it only measures.

struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
  size_t bytes() const { return (off + 255) & ~size_t(255); }
};

// ---------------------------------------------------------------------------
// device helpers

template <typename T>
__device__ __forceinline__ double to_d(T x) {
  return static_cast<double>(x);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over lanes that share the same (lane mod S); S is a power of two <= 32.
// On return lanes 0..S-1 hold the sums for s = lane.
__device__ __forceinline__ double warp_sum_strided(double v, int S) {
  for (int o = 16; o >= S; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Last-CTA-done: every CTA calls this after writing its partial results
// (by all threads).  Returns true in exactly one CTA, the last to arrive; that
// CTA then sees every other CTA's partials and resets the counter so the
// kernel can be replayed (CUDA graphs).
__device__ __forceinline__ bool last_block_done(unsigned int* counter) {
  __shared__ bool is_last;
  // the CTA barrier orders every thread's writes before thread 0's fence,
  // which publishes them (cumulatively) ahead of its arrival
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    is_last = (prev == gridDim.x * gridDim.y * gridDim.z - 1);
  }
  __syncthreads();
  if (is_last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;
  }
  return is_last;
}

// Deterministic reduction of NQ per-thread quantities into per-CTA partials
// part[blockIdx.x * NQ + q] (warp shuffles, then warps in a fixed order).
template <int NQ>
__device__ __forceinline__ void block_partials(const double (&v)[NQ],
                                               double* part) {
  __shared__ double red[NQ][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double s = warp_sum(v[q]);
    if (lane == 0) red[q][wid] = s;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
    part[(size_t)blockIdx.x * NQ + threadIdx.x] = s;
  }
  __syncthreads();
}

// Two-level deterministic grid reduction.  Each CTA has written its nslot
// partial sums to part[blockIdx.x * nslot + slot] (all threads done); the last
// CTA of each group of kRedGroup consecutive CTAs sums its group in CTA order
// into gpart, and the last group leader sums the groups in order into `out`
// (nslot doubles, shared memory).  Returns true in exactly that final CTA.
// Counters must be zero on entry; they are zero again on exit.
constexpr int kRedGroup = 32;

struct GridRed {
  double* part;        // nblk x nslot
  double* gpart;       // ceil(nblk / kRedGroup) x nslot
  unsigned int* gcnt;  // ceil(nblk / kRedGroup) counters
  unsigned int* tcnt;  // 1 counter
};

// In one CTA of at least kThreads threads (the first kThreads work, all
// take part in the barriers): out[slot] = sum over q < nq of
// src[q * nslot + slot] for every slot < nslot.  P threads share a slot (each
// sums a fixed strided subset of q in order), then a fixed shared-memory tree
// combines them: the result does not depend on scheduling.  Ends synced.
__device__ __forceinline__ void block_sum_columns(const double* __restrict__ src, int nq, int nslot,
                                                  double* out) {
  __shared__ double buf[kThreads];
  const int T = kThreads, t = threadIdx.x;
  const bool act = t < T;
  int P = 1;
  if (nslot > 32) {
    P = 8;
  } else {
    while (P * 2 * nslot <= T) P *= 2;
  }
  const int C = T / P;  // slots per round
  for (int c0 = 0; c0 < nslot; c0 += C) {
    const int slot = c0 + t % C, p = t / C;
    double acc = 0.0;
    if (act && slot < nslot) {
      int q = p;
      for (; q + 3 * P < nq; q += 4 * P) {
        const double v0 = __ldcg(src + (size_t)q * nslot + slot);
        const double v1 = __ldcg(src + (size_t)(q + P) * nslot + slot);
        const double v2 = __ldcg(src + (size_t)(q + 2 * P) * nslot + slot);
        const double v3 = __ldcg(src + (size_t)(q + 3 * P) * nslot + slot);
        acc += v0;
        acc += v1;
        acc += v2;
        acc += v3;
      }
      for (; q < nq; q += P) acc += __ldcg(src + (size_t)q * nslot + slot);
    }
    if (act) buf[t] = acc;
    __syncthreads();
    for (int h = P / 2; h >= 1; h >>= 1) {
      if (act && p < h) buf[t] += buf[t + h * C];
      __syncthreads();
    }
    if (act && p == 0 && slot < nslot) out[slot] = buf[t];
    __syncthreads();
  }
}

__device__ __forceinline__ bool grid_reduce(const GridRed& r, int nslot, double* out) {
  __shared__ int role;
  const int nblk = gridDim.x, b = blockIdx.x;
  const int g = b / kRedGroup, g0 = g * kRedGroup;
  const int gs = min(kRedGroup, nblk - g0);
  const int ngroups = (nblk + kRedGroup - 1) / kRedGroup;
  // arrival: the CTA barrier orders the partial writes of every thread before
  // thread 0's fence, which publishes them ahead of the atomic (only the
  // arriving thread fences: the other threads' unrelated stores need not wait)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    role = (atomicAdd(&r.gcnt[g], 1u) == (unsigned)gs - 1) ? 1 : 0;
    if (role) __threadfence();
  }
  __syncthreads();
  if (!role) return false;
  block_sum_columns(r.part + (size_t)g0 * nslot, gs, nslot, r.gpart + (size_t)g * nslot);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    r.gcnt[g] = 0u;
    role = (atomicAdd(r.tcnt, 1u) == (unsigned)ngroups - 1) ? 2 : 0;
    if (role) __threadfence();
  }
  __syncthreads();
  if (role != 2) return false;
  __threadfence();
  block_sum_columns(r.gpart, ngroups, nslot, out);
  if (threadIdx.x == 0) *r.tcnt = 0u;
  __syncthreads();
  return true;
}

// Double-float addition (Knuth's two-sum of the high parts, the low parts
// added and renormalised): about 44 significant bits from FP32 operations.
struct DFloat {
  float hi, lo;
};
__device__ __forceinline__ DFloat df_add(DFloat a, DFloat b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v)),
                            __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

inline int red_groups(int nblk) { return (nblk + kRedGroup - 1) / kRedGroup; }

// In one CTA: out[slot] = sum over b < nblk of part[b * nslot + slot], for
// every slot < nslot.  One warp per slot, lanes stride over the partials, then
// a fixed shuffle tree: the result does not depend on scheduling.  Ends with
// __syncthreads (out may be shared memory).
__device__ __forceinline__ void reduce_slots(const double* __restrict__ part, int nblk,
                                             int nslot, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  for (int slot = wid; slot < nslot; slot += nw) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int b = lane;
    for (; b + 96 < nblk; b += 128) {
      a0 += __ldcg(part + (size_t)b * nslot + slot);
      a1 += __ldcg(part + (size_t)(b + 32) * nslot + slot);
      a2 += __ldcg(part + (size_t)(b + 64) * nslot + slot);
      a3 += __ldcg(part + (size_t)(b + 96) * nslot + slot);
    }
    for (; b < nblk; b += 32) a0 += __ldcg(part + (size_t)b * nslot + slot);
    double acc = warp_sum((a0 + a1) + (a2 + a3));
    if (lane == 0) out[slot] = acc;
  }
  __syncthreads();
}

}  // namespace hef
