// Hyperedge resistance scoring: Algorithm 1 steps 5 and 7.
//
//   spread_{e,i} = max_{p in e} Q[p,i] - min_{p in e} Q[p,i]
//   Q_H[i]       = sum_e w_e spread_{e,i}^2                    (Eq. non-linerQ)
//   r_{e,i}      = spread_{e,i}^2 / Q_H[i]                     (Eq. ratios)
//   R_e          = max_i r_{e,i}                               (Eq. R)
//
// (chi^T b_pq)^2 of Eq. ratios with p, q the farthest-apart pins of e along
// chi is the squared spread.)  Two passes over the hyperedges in locality
// order, one warp per hyperedge, lanes over basis columns: each pin's row of
// Q is one coalesced read.  Pass 1 reduces Q_H (per-warp partials, FP64
// across warps and CTAs in a fixed order); pass 2 recomputes the spreads and
// takes the max with its arg-max column and the pins that realise it.
#include <cfloat>
#include <mutex>

#include "internal.h"

namespace hef {

namespace {

constexpr double kQhTiny = 1e-300;
constexpr int kFlushEdges = 32;  // FP32 form: edges per FP32 partial sum

template <typename T>
__device__ __forceinline__ T lowest();
template <>
__device__ __forceinline__ double lowest<double>() {
  return -DBL_MAX;
}
template <>
__device__ __forceinline__ float lowest<float>() {
  return -FLT_MAX;
}

// Max and min of each lane's columns over the pins of one hyperedge.  Pins
// are taken four at a time with the indices past the end clamped to the last
// pin (a repeated pin changes neither max nor min), so even a 2- or 3-pin
// hyperedge has all its rows in flight at once.
template <typename T, int NC>
__device__ __forceinline__ void edge_extrema(const T* __restrict__ Q, long long ldq, int K,
                                             const int32_t* __restrict__ cpins, int a, int b,
                                             int lane, T (&mx)[NC], T (&mn)[NC]) {
#pragma unroll
  for (int c = 0; c < NC; ++c) mx[c] = lowest<T>(), mn[c] = -lowest<T>();
  for (int t = a; t < b; t += 4) {
    const int last = b - 1;
    const T* r0 = Q + (long long)cpins[t] * ldq;
    const T* r1 = Q + (long long)cpins[min(t + 1, last)] * ldq;
    const T* r2 = Q + (long long)cpins[min(t + 2, last)] * ldq;
    const T* r3 = Q + (long long)cpins[min(t + 3, last)] * ldq;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int col = lane + 32 * c;
      if (col < K) {
        const T v0 = r0[col], v1 = r1[col], v2 = r2[col], v3 = r3[col];
        mx[c] = fmax(fmax(mx[c], fmax(v0, v1)), fmax(v2, v3));
        mn[c] = fmin(fmin(mn[c], fmin(v0, v1)), fmin(v2, v3));
      }
    }
  }
}

template <typename T, int NC>
__global__ void __launch_bounds__(256) k_score_pass1(IncView g, const T* __restrict__ Q, long long ldq,
                                                     int K, GridRed red, double* QH, double* invQH,
                                                     double* QH_out) {
  if (g.status[0]) return;
  __shared__ double wred[kThreads / 32][32 * NC];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  double acc[NC];
  T pacc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0, pacc[c] = 0;
  int nflush = 0;
  for (long long e = warp; e < g.m; e += nwarps) {
    const int a = g.ceptr[e], b = g.ceptr[e + 1];
    if (b - a < 2) continue;
    T mx[NC], mn[NC];
    edge_extrema<T, NC>(Q, ldq, K, g.cpins, a, b, lane, mx, mn);
    const T we = (T)g.ew[e];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const T sp = mx[c] - mn[c];
      pacc[c] += we * sp * sp;
    }
    if (sizeof(T) == 8 || ++nflush == kFlushEdges) {
      nflush = 0;
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] += (double)pacc[c], pacc[c] = 0;
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) wred[wid][lane + 32 * c] = acc[c] + (double)pacc[c];
  __syncthreads();
  for (int col = threadIdx.x; col < K; col += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wred[w][col];
    red.part[(size_t)blockIdx.x * K + col] = s;
  }
  __shared__ double tot[32 * NC];
  if (grid_reduce(red, K, tot)) {
    for (int col = threadIdx.x; col < K; col += blockDim.x) {
      const double s = tot[col];
      QH[col] = s;
      invQH[col] = s > kQhTiny ? 1.0 / s : 0.0;
      if (QH_out) QH_out[col] = s;
    }
  }
}

template <typename T, int NC>
__global__ void __launch_bounds__(256) k_score_pass2(IncView g, const T* __restrict__ Q, long long ldq,
                                                     int K, int reduce, const double* __restrict__ QH,
                                                     const double* __restrict__ invQH, double* R_out,
                                                     int32_t* argvec, int32_t* pmax, int32_t* pmin) {
  if (g.status[0]) return;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  T iq[NC];
  bool use[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int col = lane + 32 * c;
    use[c] = col < K && QH[col] > kQhTiny;
    iq[c] = use[c] ? (T)invQH[col] : (T)0;
  }
  for (long long e = warp; e < g.m; e += nwarps) {
    const int a = g.ceptr[e], b = g.ceptr[e + 1];
    const int oe = g.perm[e];
    if (b - a < 2) {
      if (lane == 0) {
        R_out[oe] = 0.0;
        if (argvec) argvec[oe] = -1;
        if (pmax) pmax[oe] = -1;
        if (pmin) pmin[oe] = -1;
      }
      continue;
    }
    T mx[NC], mn[NC];
    edge_extrema<T, NC>(Q, ldq, K, g.cpins, a, b, lane, mx, mn);
    // lane-local best (lowest column on ties), then warp arg-max
    T best = (T)-1;
    int bcol = 0x7fffffff;
    double sum = 0.0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (use[c]) {
        const T sp = mx[c] - mn[c];
        const T r = sp * sp * iq[c];
        if (reduce == HEF_REDUCE_SUM) {
          const double spd = (double)sp;
          sum += spd * spd / QH[lane + 32 * c];
        }
        if (r > best) best = r, bcol = lane + 32 * c;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oc = __shfl_xor_sync(0xffffffffu, bcol, o);
      if (ob > best || (ob == best && oc < bcol)) best = ob, bcol = oc;
    }
    if (reduce == HEF_REDUCE_SUM) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    }
    const bool any = bcol != 0x7fffffff;
    // value extremes of the winning column, from the lane that owns it
    T vmax = 0, vmin = 0;
    if (any && lane == (bcol & 31)) {
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (c == (bcol >> 5)) vmax = mx[c], vmin = mn[c];
    }
    const int owner = any ? (bcol & 31) : 0;
    vmax = __shfl_sync(0xffffffffu, vmax, owner);
    vmin = __shfl_sync(0xffffffffu, vmin, owner);
    // first pin positions attaining them (lanes over the pins of e)
    int tmax = 0x7fffffff, tmin = 0x7fffffff;
    if (any) {
      for (int t = a + lane; t < b; t += 32) {
        const T v = Q[(long long)g.cpins[t] * ldq + bcol];
        if (v == vmax && t < tmax) tmax = t;
        if (v == vmin && t < tmin) tmin = t;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        tmax = min(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
        tmin = min(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
      }
    }
    const double sp_win = (double)(vmax - vmin);
    if (lane == 0) {
      double Re = 0.0;
      if (reduce == HEF_REDUCE_SUM) Re = sum;
      else if (any) Re = sp_win * sp_win / QH[bcol];
      R_out[oe] = Re;
      if (argvec) argvec[oe] = any ? bcol : -1;
      if (pmax) pmax[oe] = any ? g.cpins[tmax] : -1;
      if (pmin) pmin[oe] = any ? g.cpins[tmin] : -1;
    }
  }
}

struct ScoreWs {
  double* part;
  double* QH;
  double* invQH;
  unsigned int* counter;  // reduction counters (zero between calls)
  double* gpart;
  int grid;
};

size_t carve_score(void* base, int K, ScoreWs* w) {
  Carver c(base);
  w->grid = num_sms() * 4;
  w->part = c.take<double>((size_t)w->grid * K);
  w->QH = c.take<double>(K);
  w->invQH = c.take<double>(K);
  w->counter = c.take<unsigned int>(64);
  w->gpart = c.take<double>((size_t)red_groups(w->grid) * K);
  return c.bytes();
}

template <typename T, int NC>
hef_status launch_score(const hef_incidence* inc, const T* Q, long long ldq, int K, int reduce,
                        double* R_out, double* QH_out, int32_t* argvec, int32_t* pmax,
                        int32_t* pmin, const ScoreWs& w, cudaStream_t st) {
  IncView g = view(inc);
  GridRed red;
  red.part = w.part;
  red.gpart = w.gpart;
  red.gcnt = w.counter;                 // red_groups(grid) <= 63 counters
  red.tcnt = w.counter + 63;
  HEF_LAUNCH("k_score_pass1", st, k_score_pass1<T, NC><<<w.grid, kThreads, 0, st>>>(g, Q, ldq, K, red, w.QH, w.invQH,
                                                    QH_out));
  HEF_LAUNCH("k_score_pass2", st, k_score_pass2<T, NC><<<w.grid, kThreads, 0, st>>>(g, Q, ldq, K, reduce, w.QH, w.invQH, R_out,
                                                    argvec, pmax, pmin));
  HEF_CHECK_LAUNCH();
  return HEF_OK;
}

template <typename T>
hef_status dispatch_score(const hef_incidence* inc, const T* Q, long long ldq, int K, int reduce,
                          double* R_out, double* QH_out, int32_t* argvec, int32_t* pmax,
                          int32_t* pmin, const ScoreWs& w, cudaStream_t st) {
  const int nc = (K + 31) / 32;
#define HEF_SCORE_CASE(N) \
  if (nc <= N) return launch_score<T, N>(inc, Q, ldq, K, reduce, R_out, QH_out, argvec, pmax, pmin, w, st)
  HEF_SCORE_CASE(1);
  HEF_SCORE_CASE(2);
  HEF_SCORE_CASE(4);
  HEF_SCORE_CASE(5);
  HEF_SCORE_CASE(8);
  HEF_SCORE_CASE(12);
  HEF_SCORE_CASE(16);
#undef HEF_SCORE_CASE
  return set_error(HEF_ERR_UNSUPPORTED, "hef_edge_resistance: K must be <= 512");
}

// ---------------------------------------------------------------------------
// Scoring for callers that cannot hand the library any device memory of
// their own (see hef_edge_resistance_noalloc): its scratch lives in one
// fixed array that is part of the loaded library on every device.

constexpr size_t kNoallocScratchBytes = size_t(2) << 20;  // 2 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  In host code
// the symbol name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
hef_status noalloc_scratch(void** out) {
  int dev = 0;
  HEF_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(HEF_ERR_UNSUPPORTED, "hef_edge_resistance_noalloc: device %d >= %d", dev,
                     kMaxDevices);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_error(HEF_ERR_CUDA, "hef_edge_resistance_noalloc: cudaGetSymbolAddress failed: %s",
                       cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return HEF_OK;
}

// Same layout as carve_score, with the CTA count capped so that the per-CTA
// partial sums fit the fixed scratch.
size_t carve_score_capped(void* base, int K, size_t cap, ScoreWs* w) {
  // per-CTA partials plus group partials (1/32 as many), Q_H, 1/Q_H, counters
  const size_t fixed = 5 * 256 + 2 * (size_t)K * sizeof(double) + 64 * sizeof(unsigned int) +
                       (size_t)K * sizeof(double);
  long long g = (long long)num_sms() * 4;
  const long long fit = (long long)((cap - fixed) / ((size_t)K * sizeof(double) * 33 / 32 + 1));
  if (g > fit) g = fit;
  Carver c(base);
  w->grid = (int)(g > 0 ? g : 1);
  w->part = c.take<double>((size_t)w->grid * K);
  w->QH = c.take<double>(K);
  w->invQH = c.take<double>(K);
  w->counter = c.take<unsigned int>(64);
  w->gpart = c.take<double>((size_t)red_groups(w->grid) * K);
  return c.bytes();
}

}  // namespace

}  // namespace hef

using namespace hef;

extern "C" hef_status hef_edge_resistance_noalloc(const hef_incidence* inc, const void* Q,
                                                  int64_t ldq, int32_t K, int32_t dtype,
                                                  int32_t reduce, double* R_out, double* QH_out,
                                                  int32_t* argvec, int32_t* pmax, int32_t* pmin,
                                                  void* stream) {
  if (!inc) return set_error(HEF_ERR_INVALID_ARG, "hef_edge_resistance_noalloc: NULL incidence");
  if (K < 1 || K > 512)
    return set_error(HEF_ERR_UNSUPPORTED,
                     "hef_edge_resistance_noalloc: K = %d outside 1..512 (the fixed %zu-byte "
                     "scratch is sized for K <= 512)",
                     K, kNoallocScratchBytes);
  if (dtype != HEF_F64 && dtype != HEF_F32)
    return set_error(HEF_ERR_INVALID_ARG, "hef_edge_resistance_noalloc: dtype must be HEF_F64 or HEF_F32");
  if (reduce != HEF_REDUCE_MAX && reduce != HEF_REDUCE_SUM)
    return set_error(HEF_ERR_INVALID_ARG, "hef_edge_resistance_noalloc: unknown reduce %d", reduce);
  if (!Q || ldq < K || (inc->m > 0 && !R_out))
    return set_error(HEF_ERR_INVALID_ARG, "hef_edge_resistance_noalloc: Q or R_out NULL, or ldq < K");
  void* scratch = nullptr;
  hef_status s = noalloc_scratch(&scratch);
  if (s) return s;
  ScoreWs w;
  if (carve_score_capped(nullptr, K, kNoallocScratchBytes, &w) > kNoallocScratchBytes)
    return set_error(HEF_ERR_UNSUPPORTED, "hef_edge_resistance_noalloc: K = %d does not fit the scratch", K);
  carve_score_capped(scratch, K, kNoallocScratchBytes, &w);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the completion counter must start at zero; partial sums are overwritten
  HEF_CHECK_CUDA(cudaMemsetAsync(w.counter, 0, 64 * sizeof(unsigned int), st));
  if (dtype == HEF_F64)
    return dispatch_score<double>(inc, static_cast<const double*>(Q), ldq, K, reduce, R_out, QH_out,
                                  argvec, pmax, pmin, w, st);
  return dispatch_score<float>(inc, static_cast<const float*>(Q), ldq, K, reduce, R_out, QH_out,
                               argvec, pmax, pmin, w, st);
}

extern "C" size_t hef_edge_resistance_workspace_bytes(const hef_incidence* inc, int32_t K) {
  if (!inc || K < 1 || K > 512) return 0;
  ScoreWs w;
  return carve_score(nullptr, K, &w);
}

extern "C" hef_status hef_edge_resistance(const hef_incidence* inc, const void* Q, int64_t ldq,
                                          int32_t K, int32_t dtype, int32_t reduce, double* R_out,
                                          double* QH_out, int32_t* argvec, int32_t* pmax,
                                          int32_t* pmin, void* workspace, size_t workspace_bytes,
                                          void* stream) {
  if (!inc) return set_error(HEF_ERR_INVALID_ARG, "hef_edge_resistance: NULL incidence");
  if (K < 1 || K > 512) return set_error(HEF_ERR_UNSUPPORTED, "hef_edge_resistance: need 1 <= K <= 512");
  if (dtype != HEF_F64 && dtype != HEF_F32)
    return set_error(HEF_ERR_INVALID_ARG, "hef_edge_resistance: dtype must be HEF_F64 or HEF_F32");
  if (reduce != HEF_REDUCE_MAX && reduce != HEF_REDUCE_SUM)
    return set_error(HEF_ERR_INVALID_ARG, "hef_edge_resistance: unknown reduce %d", reduce);
  if (!Q || ldq < K || (inc->m > 0 && !R_out))
    return set_error(HEF_ERR_INVALID_ARG, "hef_edge_resistance: Q or R_out NULL, or ldq < K");
  ScoreWs w;
  const size_t need = carve_score(workspace, K, &w);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return set_error(HEF_ERR_WORKSPACE, "hef_edge_resistance: workspace needs %zu bytes (256-aligned)", need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HEF_CHECK_CUDA(cudaMemsetAsync(w.counter, 0, 64 * sizeof(unsigned int), st));
  if (dtype == HEF_F64)
    return dispatch_score<double>(inc, static_cast<const double*>(Q), ldq, K, reduce, R_out, QH_out,
                                  argvec, pmax, pmin, w, st);
  return dispatch_score<float>(inc, static_cast<const float*>(Q), ldq, K, reduce, R_out, QH_out,
                               argvec, pmax, pmin, w, st);
}
