// Shared device/host helpers of the hef library (internal header).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>

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

constexpr int kThreads = 256;

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
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
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
      a0 += part[(size_t)b * nslot + slot];
      a1 += part[(size_t)(b + 32) * nslot + slot];
      a2 += part[(size_t)(b + 64) * nslot + slot];
      a3 += part[(size_t)(b + 96) * nslot + slot];
    }
    for (; b < nblk; b += 32) a0 += part[(size_t)b * nslot + slot];
    double acc = warp_sum((a0 + a1) + (a2 + a3));
    if (lane == 0) out[slot] = acc;
  }
  __syncthreads();
}

}  // namespace hef
