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
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cfloat>
#include <climits>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "internal.h"
#include "umma.cuh"

namespace hef {

namespace {

constexpr double kQhTiny = 1e-300;
constexpr int kGroup1 = 8;      // hyperedges per warp task in pass 1
constexpr int kMaxStages = 8;    // stages of the staged pass 1
constexpr size_t kStageSmem = 220 * 1024;  // shared memory per CTA for its stages and the rest
constexpr size_t kMaxSmemOptin = 227 * 1024;  // per-CTA limit of the sm_100 family
constexpr int kPinStage = 96;   // pins of a pass-1 task staged in shared memory
constexpr int kWorkSlot = 60;    // counters [60], [61]: work distribution of the passes

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

// An element of Q in the working type T (a BF16 basis widens exactly).
template <typename T, typename QT>
__device__ __forceinline__ T qw(QT x) {
  if constexpr (std::is_same<QT, __nv_bfloat16>::value) return (T)__bfloat162float(x);
  else return (T)x;
}

// Next group of 32 hyperedges for the calling warp (dynamic distribution:
// one atomic per group on a counter that starts each call at zero).
__device__ __forceinline__ long long next_group(unsigned int* work) {
  unsigned int grp = 0;
  if ((threadIdx.x & 31) == 0) grp = atomicAdd(work, 1u);
  return (long long)__shfl_sync(0xffffffffu, grp, 0);
}

// Extrema of two hyperedges at once (pins [a0, b0) and [a1, b1), warp-uniform):
// four clamped pin rows of each are in flight together.
template <typename T, int NC, typename PinAt, typename QT>
__device__ __forceinline__ void two_edge_extrema(const QT* __restrict__ Q, long long ldq, int K,
                                                 PinAt cpins, int a0, int b0,
                                                 int a1, int b1, int lane, T (&mx0)[NC],
                                                 T (&mn0)[NC], T (&mx1)[NC], T (&mn1)[NC]) {
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    mx0[c] = lowest<T>(), mn0[c] = -lowest<T>();
    mx1[c] = lowest<T>(), mn1[c] = -lowest<T>();
  }
  int t0 = a0, t1 = a1;
  while (t0 < b0 || t1 < b1) {
    const bool u0 = t0 < b0, u1 = t1 < b1;
    const int l0 = b0 - 1, l1 = b1 - 1;
    const QT* r[8];
    r[0] = Q + (long long)(u0 ? cpins(t0) : 0) * ldq;
    r[1] = Q + (long long)(u0 ? cpins(min(t0 + 1, l0)) : 0) * ldq;
    r[2] = Q + (long long)(u0 ? cpins(min(t0 + 2, l0)) : 0) * ldq;
    r[3] = Q + (long long)(u0 ? cpins(min(t0 + 3, l0)) : 0) * ldq;
    r[4] = Q + (long long)(u1 ? cpins(t1) : 0) * ldq;
    r[5] = Q + (long long)(u1 ? cpins(min(t1 + 1, l1)) : 0) * ldq;
    r[6] = Q + (long long)(u1 ? cpins(min(t1 + 2, l1)) : 0) * ldq;
    r[7] = Q + (long long)(u1 ? cpins(min(t1 + 3, l1)) : 0) * ldq;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int col = lane + 32 * c;
      if (col < K) {
        T v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = qw<T>(r[q][col]);
        if (u0) {
          mx0[c] = fmax(fmax(mx0[c], fmax(v[0], v[1])), fmax(v[2], v[3]));
          mn0[c] = fmin(fmin(mn0[c], fmin(v[0], v[1])), fmin(v[2], v[3]));
        }
        if (u1) {
          mx1[c] = fmax(fmax(mx1[c], fmax(v[4], v[5])), fmax(v[6], v[7]));
          mn1[c] = fmin(fmin(mn1[c], fmin(v[4], v[5])), fmin(v[6], v[7]));
        }
      }
    }
    t0 += 4;
    t1 += 4;
  }
}

// Column extrema of one large hyperedge by a whole CTA: warp w takes pin
// batches w, w + 8, ...; partial extrema meet in shared memory (smx/smn,
// [warp][32 NC]).  On return every thread's columns (lane + 32 c) hold the
// hyperedge's extrema in mx/mn.
template <typename T, int NC, typename QT>
__device__ __forceinline__ void cta_edge_extrema(const QT* __restrict__ Q, long long ldq, int K,
                                                 const int32_t* __restrict__ cpins, int nv,
                                                 const unsigned int* status, int a, int b,
                                                 T* smx, T* smn, T (&mx)[NC], T (&mn)[NC]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int c = 0; c < NC; ++c) mx[c] = lowest<T>(), mn[c] = -lowest<T>();
  for (int t = a + 4 * wid; t < b; t += 4 * nw) {
    const int last = b - 1;
    const QT* r0 = Q + (long long)dbg_index(cpins[t], nv, status) * ldq;
    const QT* r1 = Q + (long long)dbg_index(cpins[min(t + 1, last)], nv, status) * ldq;
    const QT* r2 = Q + (long long)dbg_index(cpins[min(t + 2, last)], nv, status) * ldq;
    const QT* r3 = Q + (long long)dbg_index(cpins[min(t + 3, last)], nv, status) * ldq;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int col = lane + 32 * c;
      if (col < K) {
        const T v0 = qw<T>(r0[col]), v1 = qw<T>(r1[col]), v2 = qw<T>(r2[col]), v3 = qw<T>(r3[col]);
        mx[c] = fmax(fmax(mx[c], fmax(v0, v1)), fmax(v2, v3));
        mn[c] = fmin(fmin(mn[c], fmin(v0, v1)), fmin(v2, v3));
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    smx[wid * 32 * NC + lane + 32 * c] = mx[c];
    smn[wid * 32 * NC + lane + 32 * c] = mn[c];
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    T a_ = lowest<T>(), b_ = -lowest<T>();
    for (int w = 0; w < nw; ++w) {
      a_ = fmax(a_, smx[w * 32 * NC + lane + 32 * c]);
      b_ = fmin(b_, smn[w * 32 * NC + lane + 32 * c]);
    }
    mx[c] = a_, mn[c] = b_;
  }
  __syncthreads();
}

// Pass 1, large hyperedges: CTA b handles list entries b, b + grid, ...; its
// sum of w_e spread^2 per column goes to bpart[b][col] (FP64).
template <typename T, int NC, typename QT = T>
__global__ void __launch_bounds__(256) k_score_big1(IncView g, const QT* __restrict__ Q, long long ldq,
                                                    int K, double* bpart, T* spread, int ldsp) {
  // the staged pass 1 may start beside this one: it reads bpart only after
  // its dependency wait
  pdl_trigger();
  if (g.status[0]) return;
  __shared__ T smx[8 * 32 * NC], smn[8 * 32 * NC];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nbig = g.big_pos[g.m];
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0;
  for (int bi = blockIdx.x; bi < nbig; bi += gridDim.x) {
    const int e = g.big_idx[bi];
    T mx[NC], mn[NC];
    cta_edge_extrema<T, NC, QT>(Q, ldq, K, g.cpins, g.n, g.status, g.ceptr[e], g.ceptr[e + 1], smx,
                                smn, mx, mn);
    const double we = g.ew[e];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double sp = (double)(mx[c] - mn[c]);
      acc[c] += we * sp * sp;
      if (spread && wid == 0 && lane + 32 * c < K)
        spread[(long long)e * ldsp + lane + 32 * c] = mx[c] - mn[c];
    }
  }
  if (wid == 0) {
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (lane + 32 * c < K) bpart[(size_t)blockIdx.x * K + lane + 32 * c] = acc[c];
  }
}

// Q_H from the per-CTA partials (K per CTA, already in red.part) and the large
// hyperedges' partials, in a fixed order; run by the CTA that completes the
// grid reduction.
template <int NC>
__device__ __forceinline__ void finish_qh(const GridRed& red, int K, const double* __restrict__ bpart,
                                          int nbpart, double* QH, double* invQH, double* QH_out) {
  // k_score_big1 (bpart) complete: a no-op unless this pass was launched as
  // its programmatic dependent
  pdl_wait();
  __shared__ double tot[32 * NC];
  if (grid_reduce(red, K, tot)) {
    for (int col = threadIdx.x; col < K; col += blockDim.x) {
      double s = tot[col];
      for (int q = 0; q < nbpart; ++q) s += bpart[(size_t)q * K + col];
      QH[col] = s;
      invQH[col] = s > kQhTiny ? 1.0 / s : 0.0;
      if (QH_out) QH_out[col] = s;
    }
  }
}

// Pass 1, hyperedges with 2..kBigEdge pins, rows of Q gathered by the warps:
// warp per group of kGroup1 consecutive hyperedges (two at a time), their
// spreads stored row-major (spread[e K + i]) when `spread` is given; Q_H[i] =
// sum of per-CTA partials, then the large hyperedges' partials bpart, in a
// fixed order.
template <typename T, int NC, typename QT = T>
__global__ void __launch_bounds__(256) k_score_pass1(IncView g, const QT* __restrict__ Q, long long ldq,
                                                     int K, GridRed red, const double* __restrict__ bpart,
                                                     int nbpart, double* QH, double* invQH,
                                                     double* QH_out, unsigned int* work,
                                                     T* spread, int ldsp) {
  if (g.status[0]) return;
  __shared__ double wred[kThreads / 32][32 * NC];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double acc[NC];
  T pacc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0, pacc[c] = 0;
  // static assignment (the FP64 partials must not depend on scheduling):
  // warp w takes groups of kGroup1 hyperedges w, w + nwarps, ...
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long ngroups = ((long long)g.m + kGroup1 - 1) / kGroup1;
  (void)work;
  __shared__ int spins[kThreads / 32][kPinStage];  // the group's first pins
  for (long long grp = warp; grp < ngroups; grp += nwarps) {
    const long long e = grp * kGroup1 + lane;
    int a = 0, b = 0;
    if (lane < kGroup1 && e < g.m) a = g.ceptr[e], b = g.ceptr[e + 1];
    // the group's pin ids in one coalesced read (the extrema then wait on one
    // round trip, Q, instead of two)
    const int gp0 = __shfl_sync(0xffffffffu, a, 0);
    const int gp1 = __shfl_sync(0xffffffffu, b, min(kGroup1, (int)(g.m - grp * kGroup1)) - 1);
    const int npin = min(gp1 - gp0, kPinStage);
    __syncwarp();  // the previous group's reads of spins are done
    for (int q = lane; q < npin; q += 32) spins[wid][q] = g.cpins[gp0 + q];
    __syncwarp();
    auto pin_at = [&](int t) {
      return dbg_index(t - gp0 < npin ? spins[wid][t - gp0] : g.cpins[t], g.n, g.status);
    };
    if (b - a < 2 || b - a > kBigEdge) b = a;  // not scored here
    const T wl = (lane < kGroup1 && e < g.m) ? (T)g.ew[e] : (T)0;
    T* sprow = spread ? spread + grp * kGroup1 * ldsp : nullptr;  // row-major spreads of the group
    for (int i = 0; i < kGroup1; i += 2) {
      const int a0 = __shfl_sync(0xffffffffu, a, i), b0 = __shfl_sync(0xffffffffu, b, i);
      const int a1 = __shfl_sync(0xffffffffu, a, i + 1), b1 = __shfl_sync(0xffffffffu, b, i + 1);
      const T w0 = __shfl_sync(0xffffffffu, wl, i), w1 = __shfl_sync(0xffffffffu, wl, i + 1);
      if (a0 == b0 && a1 == b1) continue;
      T mx0[NC], mn0[NC], mx1[NC], mn1[NC];
      two_edge_extrema<T, NC>(Q, ldq, K, pin_at, a0, b0, a1, b1, lane, mx0, mn0, mx1, mn1);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int col = lane + 32 * c;
        if (b0 > a0) {
          const T sp = mx0[c] - mn0[c];
          pacc[c] += w0 * sp * sp;
          if (sprow && col < K) sprow[(long long)i * ldsp + col] = sp;
        }
        if (b1 > a1) {
          const T sp = mx1[c] - mn1[c];
          pacc[c] += w1 * sp * sp;
          if (sprow && col < K) sprow[(long long)(i + 1) * ldsp + col] = sp;
        }
      }
    }
    // FP32 partial sums span one group (kGroup1 hyperedges); FP64 beyond
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] += (double)pacc[c], pacc[c] = 0;
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) wred[wid][lane + 32 * c] = acc[c];
  __syncthreads();
  for (int col = threadIdx.x; col < K; col += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wred[w][col];
    red.part[(size_t)blockIdx.x * K + col] = s;
  }
  finish_qh<NC>(red, K, bpart, nbpart, QH, invQH, QH_out);
}


// Pass 1 with the pin rows staged in shared memory by bulk asynchronous
// copies (the same sums as k_score_pass1).  CTA b takes a contiguous range of
// windows of CSC slots (see kWinSlots) and streams the Q rows of their slots,
// in slot order, through a ring of `nst` stages of kWinSlots rows (row pitch
// `pitch` elements, `row_bytes` a multiple of 16): slot t sits in ring row
// (t - first slot of the range) mod (nst kWinSlots).  Warp 0 produces: it
// copies window j's rows (G4: four-row tensor-map gathers, tile::gather4 with
// a box one row high; else one bulk copy per row) once the consumers have
// released window j - nst
// (plus the window after the range, whose rows the range's last hyperedges
// may reach), with the offsets and weights of the hyperedges the window owns
// (aligned supersets of ceptr[ef..el] and ew[ef..el), when at most
// kMetaEdges - 8 of them); the pin ids and the window table are loaded a
// group of kGroupWin windows ahead.  Warps 1..15 consume: for window w, once
// windows w and w + 1 have landed, each scores the window's hyperedges (first
// slot in w; at most kBigEdge pins, so they end within w + 1) w, w + 15, ...
// from shared memory, lanes over columns.  Waits are bounded: on expiry the
// kernel sets HEF_WAIT_TIMEOUT in `status`, stops, waits (bounded) for the
// copies it issued and still takes part in the reduction.
static_assert(kBigEdge <= kWinSlots, "a scored hyperedge must end within the next window");
constexpr int kPinRegs = (kWinSlots + 31) / 32;
constexpr int kBulkThreads = 512;  // warp 0 produces, warps 1..15 consume
constexpr int kConsumers = kBulkThreads / 32 - 1;
constexpr int kGroupWin = 8;    // windows per prefetch group of the producer
constexpr int kMetaEdges = 128;  // hyperedge offsets / weights staged per window
constexpr int kFlushWin = 8;     // windows per working-type partial sum of a consumer warp
constexpr uint32_t kCopyWaitIters = 1u << 20;

template <typename T, int NC, bool G4>
__global__ void __launch_bounds__(kBulkThreads, 1)
    k_score_pass1_bulk(IncView g, const T* __restrict__ Q, long long ldq, int K, int pitch,
                       uint32_t row_bytes, int nst, GridRed red, const double* __restrict__ bpart,
                       int nbpart, double* QH, double* invQH, double* QH_out, T* spread,
                       int ldsp, const T* __restrict__ ewT, unsigned int* status,
                       const __grid_constant__ CUtensorMap tmap) {
  using namespace umma;
  if (g.status[0]) return;
  extern __shared__ __align__(128) unsigned char stage_raw[];
  // the ring from the first 128-byte boundary (the launch adds 128 bytes)
  unsigned char* ring_raw = stage_raw + ((128u - (umma::smem_u32(stage_raw) & 127u)) & 127u);
  T* ring = reinterpret_cast<T*>(ring_raw);
  __shared__ uint64_t full[kMaxStages], empty[kMaxStages];
  __shared__ __align__(16) int m_ceptr[kMaxStages][kMetaEdges];
  __shared__ __align__(16) T m_ew[kMaxStages][kMetaEdges];
  __shared__ int meta[kMaxStages][3];  // ef, el, offsets staged
  __shared__ int abort_flag;
  __shared__ long long issued;
  volatile int* abort_v = &abort_flag;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long nwin = num_windows(g.P);
  // this CTA's windows [wb, we) and the windows it copies [wb, wc): one
  // more when it has any, whose first slots its last hyperedges may reach
  const long long wb = nwin * blockIdx.x / gridDim.x, we = nwin * (blockIdx.x + 1) / gridDim.x;
  const long long wc = (we > wb && we < nwin) ? we + 1 : we;
  const int ring_rows = nst * kWinSlots;
  if (threadIdx.x == 0) {
    for (int q = 0; q < nst; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kConsumers);
    }
    abort_flag = 0;
    issued = wb;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0;
  auto fail = [&]() {
    if (lane == 0) {
      *abort_v = 1;
      atomicOr(&status[0], HEF_WAIT_TIMEOUT);
    }
  };
  if (wid == 0) {
    // ---- producer
    // group buffers of kGroupWin windows from g0: the pin ids (per-row copies:
    // lane l holds slots l and l + 32 of window g0 + d in pc[d]; gather4: lane
    // l holds slots 4 (l mod 16) .. + 3 of window g0 + 2 h + l / 16 in pc4[h])
    // and win_edge[g0 + l] for l <= kGroupWin
    constexpr int kRegs = G4 ? 1 : kPinRegs;
    constexpr int kBufs = G4 ? kGroupWin / 2 : kGroupWin;
    int pc[kBufs][kRegs], pn[kBufs][kRegs];
    int4 pc4[kBufs], pn4[kBufs];
    int wc_e = 0, wn_e = 0;
    auto load_group = [&](long long g0, int (&pp)[kBufs][kRegs], int4 (&pp4)[kBufs], int& wl) {
      if constexpr (G4) {
#pragma unroll
        for (int h = 0; h < kBufs; ++h) {
          const long long jw = g0 + 2 * h + (lane >> 4);
          const long long t = jw * kWinSlots + 4 * (lane & 15);
          pp4[h] = (jw < wc && t < g.P) ? *reinterpret_cast<const int4*>(g.cpins + t)
                                        : make_int4(0, 0, 0, 0);
          if (HEF_DEBUG) {
            // slots past P read as pin 0 of the padded array: only real slots are checked
            pp4[h].x = t < g.P ? dbg_index(pp4[h].x, g.n, g.status) : pp4[h].x;
            pp4[h].y = t + 1 < g.P ? dbg_index(pp4[h].y, g.n, g.status) : pp4[h].y;
            pp4[h].z = t + 2 < g.P ? dbg_index(pp4[h].z, g.n, g.status) : pp4[h].z;
            pp4[h].w = t + 3 < g.P ? dbg_index(pp4[h].w, g.n, g.status) : pp4[h].w;
          }
        }
      } else {
#pragma unroll
        for (int d = 0; d < kBufs; ++d)
#pragma unroll
          for (int u = 0; u < kRegs; ++u) {
            const long long t = (g0 + d) * kWinSlots + lane + 32 * u;
            pp[d][u] = (g0 + d < wc && lane + 32 * u < kWinSlots && t < g.P)
                           ? dbg_index(g.cpins[t], g.n, g.status)
                           : 0;
          }
      }
      wl = (lane <= kGroupWin && g0 + lane <= nwin) ? g.win_edge[g0 + lane] : 0;
    };
    load_group(wb, pc, pc4, wc_e);
    long long j = wb;
    bool stop = false;
    for (long long g0 = wb; g0 < wc && !stop; g0 += kGroupWin) {
      load_group(g0 + kGroupWin, pn, pn4, wn_e);
#pragma unroll
      for (int d = 0; d < kGroupWin; ++d) {
        j = g0 + d;
        if (j >= wc) break;
        if (*abort_v) {
          stop = true;
          break;
        }
        const int q = (int)((j - wb) % nst);
        const long long use = (j - wb) / nst;
        if (use > 0) {
          const bool ok = __all_sync(0xffffffffu, mbar_wait(&empty[q], (uint32_t)((use - 1) & 1),
                                                            kCopyWaitIters));
          if (!ok) {
            fail();
            stop = true;
            break;
          }
        }
        const int ef = __shfl_sync(0xffffffffu, wc_e, d), el = __shfl_sync(0xffffffffu, wc_e, d + 1);
        const int rows = (int)min((long long)kWinSlots, (long long)g.P - j * kWinSlots);
        // offsets ceptr[c0, c0 + cn) and weights ewT[w0, w0 + wn): 16-byte aligned
        // supersets (within the arrays' 256-byte padded allocations)
        constexpr int kWv = 16 / sizeof(T);
        const int c0 = ef & ~3, cn = ((el + 4) & ~3) - c0;
        const int w0 = ef & ~(kWv - 1), wn = ((el + kWv - 1) & ~(kWv - 1)) - w0;
        const bool mok = el >= ef && el - ef + 8 <= kMetaEdges;
        const int copied = G4 ? (rows + 3) / 4 * 4 : rows;  // gather4 moves whole groups of four
        const uint32_t bytes =
            (uint32_t)copied * row_bytes + (mok ? (uint32_t)(cn * 4 + wn * (int)sizeof(T)) : 0u);
        if (lane == 0) {
          meta[q][0] = ef;
          meta[q][1] = el;
          meta[q][2] = mok;
          mbar_arrive_expect_tx(&full[q], bytes);
        }
        __syncwarp();
        T* dst = ring + (size_t)q * kWinSlots * pitch;
        if constexpr (G4) {
          const int r4 = 4 * (lane & 15);
          if ((lane >> 4) == (d & 1) && r4 < rows) {
            const int4 pv = pc4[d >> 1];
            // rows past the window's end repeat its row r4
            gather4_g2s(dst + (size_t)r4 * pitch, &tmap, pv.x, r4 + 1 < rows ? pv.y : pv.x,
                        r4 + 2 < rows ? pv.z : pv.x, r4 + 3 < rows ? pv.w : pv.x, &full[q]);
          }
        } else {
#pragma unroll
          for (int u = 0; u < kRegs; ++u) {
            const int r = lane + 32 * u;
            if (r < rows)
              bulk_g2s(dst + (size_t)r * pitch, Q + (long long)pc[d][u] * ldq, row_bytes, &full[q]);
          }
        }
        if (mok && lane == 0) {
          bulk_g2s(&m_ceptr[q][0], g.ceptr + c0, (uint32_t)cn * 4u, &full[q]);
          if (wn > 0) bulk_g2s(&m_ew[q][0], ewT + w0, (uint32_t)(wn * sizeof(T)), &full[q]);
        }
        j = j + 1;
      }
#pragma unroll
      for (int d = 0; d < kBufs; ++d) {
        pc4[d] = pn4[d];
#pragma unroll
        for (int u = 0; u < kRegs; ++u) pc[d][u] = pn[d][u];
      }
      wc_e = wn_e;
    }
    if (lane == 0) issued = j;
  } else {
    // ---- consumers
    const int cw = wid - 1;
    T pacc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) pacc[c] = 0;
    for (long long w = wb; w < we; ++w) {
      const int q = (int)((w - wb) % nst);
      bool got = mbar_wait(&full[q], (uint32_t)(((w - wb) / nst) & 1), kCopyWaitIters);
      if (w + 1 < wc)
        got = got && mbar_wait(&full[(w + 1 - wb) % nst], (uint32_t)(((w + 1 - wb) / nst) & 1),
                               kCopyWaitIters);
      got = __all_sync(0xffffffffu, got);
      if (!got || *abort_v) {
        if (!got) fail();
        break;
      }
      const int ef = meta[q][0], el = meta[q][1];
      const bool mok = meta[q][2] != 0;
      const int c0 = ef & ~3, w0 = ef & ~(16 / (int)sizeof(T) - 1);
      const int row_w = q * kWinSlots;  // ring row of the window's first slot
      const long long slot_w = w * kWinSlots;
      const long long slot_end = min(wc * kWinSlots, (long long)g.P);
      for (int e = ef + cw; e < el; e += kConsumers) {
        int a, b;
        T we_;
        if (mok) a = m_ceptr[q][e - c0], b = m_ceptr[q][e + 1 - c0], we_ = m_ew[q][e - w0];
        else a = g.ceptr[e], b = g.ceptr[e + 1], we_ = ewT[e];
        const int k = b - a;
        // staged: slots [w kWinSlots, min(wc kWinSlots, P)); a >= w kWinSlots
        if (k < 2 || k > kBigEdge || (long long)b > slot_end) continue;
        const int r0 = row_w + (int)(a - slot_w);  // ring row of the first pin
        T mx[NC], mn[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) mx[c] = lowest<T>(), mn[c] = -lowest<T>();
        for (int t = 0; t < k; t += 4) {
          const T* rp[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            int x = r0 + min(t + u, k - 1);
            x = x >= ring_rows ? x - ring_rows : x;
            rp[u] = ring + x * pitch + lane;
          }
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            if (lane + 32 * c < K) {
              const T v0 = rp[0][32 * c], v1 = rp[1][32 * c];
              const T v2 = rp[2][32 * c], v3 = rp[3][32 * c];
              mx[c] = fmax(fmax(mx[c], fmax(v0, v1)), fmax(v2, v3));
              mn[c] = fmin(fmin(mn[c], fmin(v0, v1)), fmin(v2, v3));
            }
          }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int col = lane + 32 * c;
          const T sp = mx[c] - mn[c];
          if (col < K) {
            pacc[c] += we_ * sp * sp;
            if (spread) spread[(long long)e * ldsp + col] = sp;
          }
        }
      }
      // partial sums in the working type over kFlushWin windows; FP64 beyond
      if ((w - wb) % kFlushWin == kFlushWin - 1) {
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] += (double)pacc[c], pacc[c] = 0;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[q]);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] += (double)pacc[c];
  }
  __syncthreads();
  // every copy has landed before the ring is reused or the CTA exits: the
  // last use of each stage (a no-op unless a wait expired)
  if (threadIdx.x == 0)
    for (long long j = issued - nst > wb ? issued - nst : wb; j < issued; ++j)
      mbar_wait(&full[(j - wb) % nst], (uint32_t)(((j - wb) / nst) & 1), kCopyWaitIters);
  __syncthreads();
  // per-warp sums in the (now idle) ring: [warp][32 NC]
  double* wred = reinterpret_cast<double*>(ring_raw);
#pragma unroll
  for (int c = 0; c < NC; ++c) wred[wid * 32 * NC + lane + 32 * c] = acc[c];
  __syncthreads();
  for (int col = threadIdx.x; col < K; col += blockDim.x) {
    double sum = 0.0;
    for (int w = 0; w < kBulkThreads / 32; ++w) sum += wred[w * 32 * NC + col];
    red.part[(size_t)blockIdx.x * K + col] = sum;
  }
  finish_qh<NC>(red, K, bpart, nbpart, QH, invQH, QH_out);
}

// Pass 2 for one hyperedge whose extrema a warp holds (lanes over columns):
// arg-max column (lowest on ties), its pins (lowest position on ties), R_e.
template <typename T, int NC, typename QT>
__device__ __forceinline__ void score_edge_out(IncView g, const QT* __restrict__ Q, long long ldq,
                                               int K, int reduce, const double* __restrict__ invQH,
                                               const T (&iq)[NC], const bool (&use)[NC], int e,
                                               int a, int b, const T (&mx)[NC], const T (&mn)[NC],
                                               double* R_out, int32_t* argvec, int32_t* pmax,
                                               int32_t* pmin) {
  const int lane = threadIdx.x & 31;
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
        sum += spd * spd * invQH[lane + 32 * c];
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
  T vmax = 0, vmin = 0;
  if (any && lane == (bcol & 31)) {
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (c == (bcol >> 5)) vmax = mx[c], vmin = mn[c];
  }
  const int owner = any ? (bcol & 31) : 0;
  vmax = __shfl_sync(0xffffffffu, vmax, owner);
  vmin = __shfl_sync(0xffffffffu, vmin, owner);
  int tmax = 0x7fffffff, tmin = 0x7fffffff;
  if (any) {
    for (int t = a + lane; t < b; t += 32) {
      const T v = qw<T>(Q[(long long)dbg_index(g.cpins[t], g.n, g.status) * ldq + bcol]);
      if (v == vmax && t < tmax) tmax = t;
      if (v == vmin && t < tmin) tmin = t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      tmax = min(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
      tmin = min(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
    }
  }
  if (lane == 0) {
    const int oe = g.perm[e];
    double Re = 0.0;
    if (reduce == HEF_REDUCE_SUM) Re = sum;
    else if (any) {
      const double spw = (double)(vmax - vmin);
      Re = spw * spw * invQH[bcol];  // as in k_score_ratio
    }
    R_out[oe] = Re;
    if (argvec) argvec[oe] = any ? bcol : -1;
    if (pmax) pmax[oe] = any ? g.cpins[tmax] : -1;
    if (pmin) pmin[oe] = any ? g.cpins[tmin] : -1;
  }
}

template <typename T, int NC>
__device__ __forceinline__ void load_use(const double* __restrict__ QH, const double* __restrict__ invQH,
                                         int K, T (&iq)[NC], bool (&use)[NC]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int col = lane + 32 * c;
    use[c] = col < K && QH[col] > kQhTiny;
    iq[c] = use[c] ? (T)invQH[col] : (T)0;
  }
}

// Pass 2, large hyperedges (one CTA each; warp 0 writes the outputs).
template <typename T, int NC, typename QT = T>
__global__ void __launch_bounds__(256) k_score_big2(IncView g, const QT* __restrict__ Q, long long ldq,
                                                    int K, int reduce, const double* __restrict__ QH,
                                                    const double* __restrict__ invQH, double* R_out,
                                                    int32_t* argvec, int32_t* pmax, int32_t* pmin) {
  if (g.status[0]) return;
  __shared__ T smx[8 * 32 * NC], smn[8 * 32 * NC];
  T iq[NC];
  bool use[NC];
  load_use<T, NC>(QH, invQH, K, iq, use);
  const int nbig = g.big_pos[g.m];
  for (int bi = blockIdx.x; bi < nbig; bi += gridDim.x) {
    const int e = g.big_idx[bi];
    const int a = g.ceptr[e], b = g.ceptr[e + 1];
    T mx[NC], mn[NC];
    cta_edge_extrema<T, NC, QT>(Q, ldq, K, g.cpins, g.n, g.status, a, b, smx, smn, mx, mn);
    if ((threadIdx.x >> 5) == 0)
      score_edge_out<T, NC, QT>(g, Q, ldq, K, reduce, invQH, iq, use, e, a, b, mx, mn, R_out, argvec,
                                pmax, pmin);
  }
}

// Pass 2, the other hyperedges: warp per group of 32, two at a time; those
// with < 2 pins get 0 / -1.
template <typename T, int NC, typename QT = T>
__global__ void __launch_bounds__(256) k_score_pass2(IncView g, const QT* __restrict__ Q, long long ldq,
                                                     int K, int reduce, const double* __restrict__ QH,
                                                     const double* __restrict__ invQH, double* R_out,
                                                     int32_t* argvec, int32_t* pmax, int32_t* pmin,
                                                     unsigned int* work) {
  if (g.status[0]) return;
  const int lane = threadIdx.x & 31;
  T iq[NC];
  bool use[NC];
  load_use<T, NC>(QH, invQH, K, iq, use);
  const long long ngroups = ((long long)g.m + 31) / 32;
  for (;;) {
    const long long grp = next_group(work);
    if (grp >= ngroups) break;
    const long long e = grp * 32 + lane;
    int a = 0, b = 0;
    if (e < g.m) a = g.ceptr[e], b = g.ceptr[e + 1];
    if (e < g.m && b - a < 2) {  // degenerate: no score, no routing
      const int oe = g.perm[e];
      R_out[oe] = 0.0;
      if (argvec) argvec[oe] = -1;
      if (pmax) pmax[oe] = -1;
      if (pmin) pmin[oe] = -1;
    }
    if (b - a < 2 || b - a > kBigEdge) b = a;
    for (int i = 0; i < 32; i += 2) {
      const int a0 = __shfl_sync(0xffffffffu, a, i), b0 = __shfl_sync(0xffffffffu, b, i);
      const int a1 = __shfl_sync(0xffffffffu, a, i + 1), b1 = __shfl_sync(0xffffffffu, b, i + 1);
      if (a0 == b0 && a1 == b1) continue;
      T mx0[NC], mn0[NC], mx1[NC], mn1[NC];
      two_edge_extrema<T, NC>(Q, ldq, K, [&](int t) { return dbg_index(g.cpins[t], g.n, g.status); },
                              a0, b0, a1, b1, lane,
                              mx0, mn0, mx1, mn1);
      if (b0 > a0)
        score_edge_out<T, NC, QT>(g, Q, ldq, K, reduce, invQH, iq, use, (int)(grp * 32 + i), a0, b0,
                                  mx0, mn0, R_out, argvec, pmax, pmin);
      if (b1 > a1)
        score_edge_out<T, NC, QT>(g, Q, ldq, K, reduce, invQH, iq, use, (int)(grp * 32 + i + 1), a1,
                                  b1, mx1, mn1, R_out, argvec, pmax, pmin);
    }
  }
}

// Pass 2 from the spreads that pass 1 stored (row-major, spread[e ldsp + i],
// rows 16-byte aligned; every hyperedge with >= 2 pins has them): thread per
// hyperedge, its row read with 16-byte loads, kRatioVecs of them in flight.
// Ratios and the arg-max column in the working type as in Eq. ratios (lowest
// column on ties); R_e from the spread in FP64 (times 1/Q_H); the routing pins from one
// gather of the arg-max column over the hyperedge's pins (lowest position on
// ties).  Gives exactly what k_score_pass2 / k_score_big2 give without
// gathering every column of Q again.
constexpr int kRatioVecs = 4;

template <typename T>
__global__ void __launch_bounds__(256) k_score_ratio(IncView g, const T* __restrict__ Q, long long ldq,
                                                     int K, int reduce, const double* __restrict__ QH,
                                                     const double* __restrict__ invQH,
                                                     const T* __restrict__ spread, int ldsp,
                                                     double* R_out, int32_t* argvec, int32_t* pmax,
                                                     int32_t* pmin) {
  if (g.status[0]) return;
  constexpr int V = 16 / sizeof(T);  // elements per 16-byte load
  constexpr int B = V * kRatioVecs;  // columns per batch
  extern __shared__ unsigned char iq_raw[];
  T* iq = reinterpret_cast<T*>(iq_raw);  // K: 1 / Q_H in the working type, 0 when unused
  for (int i = threadIdx.x; i < K; i += blockDim.x) iq[i] = QH[i] > kQhTiny ? (T)invQH[i] : (T)0;
  __syncthreads();
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < g.m;
       e += (long long)gridDim.x * blockDim.x) {
    const int a = g.ceptr[e], b = g.ceptr[e + 1];
    const int oe = g.perm[e];
    if (b - a < 2) {  // degenerate: no score, no routing
      R_out[oe] = 0.0;
      if (argvec) argvec[oe] = -1;
      if (pmax) pmax[oe] = -1;
      if (pmin) pmin[oe] = -1;
      continue;
    }
    const uint4* row = reinterpret_cast<const uint4*>(spread + e * ldsp);
    T best = (T)-1, spb = 0;
    int bcol = -1;
    double sum = 0.0;
    for (int i0 = 0; i0 < K; i0 += B) {
      T sp[B];
#pragma unroll
      for (int u = 0; u < kRatioVecs; ++u) {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (i0 + u * V < K) v = __ldg(row + i0 / V + u);
        memcpy(&sp[u * V], &v, 16);
      }
#pragma unroll
      for (int q = 0; q < B; ++q) {
        const int i = i0 + q;
        if (i >= K || iq[i] == (T)0) continue;
        const T r = sp[q] * sp[q] * iq[i];
        if (reduce == HEF_REDUCE_SUM) {
          const double spd = (double)sp[q];
          sum += spd * spd * invQH[i];
        }
        if (r > best) best = r, bcol = i, spb = sp[q];
      }
    }
    const bool any = bcol >= 0;
    int tmax = a, tmin = a;
    if (any && (pmax || pmin)) {
      // extrema of column bcol over the pins, lowest position on ties
      T vmax = Q[(long long)dbg_index(g.cpins[a], g.n, g.status) * ldq + bcol], vmin = vmax;
      for (int t = a + 1; t < b; ++t) {
        const T v = qw<T>(Q[(long long)dbg_index(g.cpins[t], g.n, g.status) * ldq + bcol]);
        if (v > vmax) vmax = v, tmax = t;
        if (v < vmin) vmin = v, tmin = t;
      }
    }
    double Re = 0.0;
    if (reduce == HEF_REDUCE_SUM) Re = sum;
    else if (any) {  // times the FP64 1/Q_H (an FP64 division costs about ten FP64 operations)
      const double spw = (double)spb;
      Re = spw * spw * invQH[bcol];
    }
    R_out[oe] = Re;
    if (argvec) argvec[oe] = any ? bcol : -1;
    if (pmax) pmax[oe] = any ? g.cpins[tmax] : -1;
    if (pmin) pmin[oe] = any ? g.cpins[tmin] : -1;
  }
}

// Pass 2 from the stored spreads for the max reduction (Eq. R), eight lanes
// per hyperedge: lane l of a group reads 16-byte chunks l, l + 8, ... of the
// row, so each load instruction of a warp covers four rows in full 128-byte
// lines instead of 32 rows in 16-byte pieces.  Each lane keeps the largest
// ratio of its columns (lowest column on ties, scanning upwards) and the
// group combines by value, then column, which selects the same column as a
// scan of the whole row.  The routing pins: the lanes split the hyperedge's
// pins the same way and combine the extrema of the arg-max column by value,
// then position.  R_e, the arg-max column and the routing pins are therefore
// bit-identical to k_score_ratio's.
constexpr int kRatioLanes = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_score_ratio8(IncView g, const T* __restrict__ Q, long long ldq,
                                                      int K, const double* __restrict__ QH,
                                                      const double* __restrict__ invQH,
                                                      const T* __restrict__ spread, int ldsp,
                                                      double* R_out, int32_t* argvec, int32_t* pmax,
                                                      int32_t* pmin) {
  if (g.status[0]) return;
  constexpr int V = 16 / sizeof(T);  // elements per 16-byte chunk
  constexpr int U = 4;               // chunks of a lane in flight
  extern __shared__ unsigned char iq_raw[];
  T* iq = reinterpret_cast<T*>(iq_raw);  // K: 1 / Q_H in the working type, 0 when unused
  for (int i = threadIdx.x; i < K; i += blockDim.x) iq[i] = QH[i] > kQhTiny ? (T)invQH[i] : (T)0;
  __syncthreads();
  const int lane = threadIdx.x & 31, sub = lane & (kRatioLanes - 1);
  const int nchunk = (K + V - 1) / V;
  const long long groups_per_warp = 32 / kRatioLanes;
  const long long wglob = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long wstride = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long eb = wglob * groups_per_warp; eb < g.m; eb += wstride * groups_per_warp) {
    const long long e = eb + (lane >> 3);
    const bool valid = e < g.m;
    int a = 0, b = 0;
    if (valid) a = g.ceptr[e], b = g.ceptr[e + 1];
    const bool scored = valid && b - a >= 2;
    T best = (T)-1, spb = 0;
    int bcol = -1;
    if (scored) {
      const uint4* row = reinterpret_cast<const uint4*>(spread + e * ldsp);
      for (int c0 = sub; c0 < nchunk; c0 += U * kRatioLanes) {
        T sp[U][V];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          uint4 v = make_uint4(0u, 0u, 0u, 0u);
          if (c0 + u * kRatioLanes < nchunk) v = __ldg(row + c0 + u * kRatioLanes);
          memcpy(&sp[u][0], &v, 16);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int q = 0; q < V; ++q) {
            const int i = (c0 + u * kRatioLanes) * V + q;
            if (i >= K || iq[i] == (T)0) continue;
            const T r = sp[u][q] * sp[u][q] * iq[i];
            if (r > best) best = r, bcol = i, spb = sp[u][q];
          }
      }
    }
    // combine the group's candidates: larger ratio, then lower column
#pragma unroll
    for (int o = kRatioLanes / 2; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const T os = __shfl_xor_sync(0xffffffffu, spb, o);
      const int oc = __shfl_xor_sync(0xffffffffu, bcol, o);
      if (oc >= 0 && (bcol < 0 || ob > best || (ob == best && oc < bcol))) best = ob, bcol = oc, spb = os;
    }
    const bool any = scored && bcol >= 0;
    T vmax = lowest<T>(), vmin = -lowest<T>();
    int tmax = INT_MAX, tmin = INT_MAX;
    if (any && (pmax || pmin)) {
      for (int t = a + sub; t < b; t += kRatioLanes) {
        const T v = qw<T>(Q[(long long)dbg_index(g.cpins[t], g.n, g.status) * ldq + bcol]);
        if (tmax == INT_MAX || v > vmax) vmax = v, tmax = t;
        if (tmin == INT_MAX || v < vmin) vmin = v, tmin = t;
      }
    }
#pragma unroll
    for (int o = kRatioLanes / 2; o > 0; o >>= 1) {
      const T ovx = __shfl_xor_sync(0xffffffffu, vmax, o), ovn = __shfl_xor_sync(0xffffffffu, vmin, o);
      const int otx = __shfl_xor_sync(0xffffffffu, tmax, o), otn = __shfl_xor_sync(0xffffffffu, tmin, o);
      if (otx != INT_MAX && (tmax == INT_MAX || ovx > vmax || (ovx == vmax && otx < tmax))) vmax = ovx, tmax = otx;
      if (otn != INT_MAX && (tmin == INT_MAX || ovn < vmin || (ovn == vmin && otn < tmin))) vmin = ovn, tmin = otn;
    }
    if (valid && sub == 0) {
      const int oe = g.perm[e];
      double Re = 0.0;
      if (any) {  // times the FP64 1/Q_H, as k_score_ratio
        const double spw = (double)spb;
        Re = spw * spw * invQH[bcol];
      }
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
  double* bpart;          // large hyperedges: per-CTA partial Q_H sums
  void* spread;           // m x K spreads of pass 1 (NULL: pass 2 gathers Q again)
  int grid;
  int bgrid;
};

// Row pitch (elements) of the stored spreads: K rounded up to 16 bytes.
inline int spread_ld(int K, size_t esz) {
  const int v = (int)(16 / esz);
  return (K + v - 1) / v * v;
}

// Workspace of hef_edge_resistance; the spread rows take the FP32 pitch in
// 8-byte slots, enough for either dtype (the size query does not know it).
size_t carve_score(void* base, int K, long long m, ScoreWs* w) {
  Carver c(base);
  w->grid = num_sms() * 4;
  w->part = c.take<double>((size_t)w->grid * K);
  w->QH = c.take<double>(K);
  w->invQH = c.take<double>(K);
  w->counter = c.take<unsigned int>(64);
  w->gpart = c.take<double>((size_t)red_groups(w->grid) * K);
  w->bgrid = num_sms();
  w->bpart = c.take<double>((size_t)w->bgrid * K);
  w->spread = c.take<double>((size_t)(m > 0 ? m : 1) * spread_ld(K, sizeof(float)));
  return c.bytes();
}

// Scores with the embedding-farthest pair (HEF_REDUCE_EMBED; reading A7's
// alternative for "p and q are the most distant nodes in the embedding
// space", Eq. ratios).  One warp per hyperedge: lanes take the pin pairs
// (a < b, positions in the hyperedge) in row-major order, strided by 32;
// each squared distance is summed over the columns in ascending order with
// round-to-nearest FP64 operations; the largest wins, ties to the first
// pair.  Then lanes take the columns: r_i = (Q[p,i] - Q[q,i])^2 / Q_H[i] over
// the usable columns, the largest wins, ties to the lowest i.
template <typename T, typename QT = T>
__global__ void __launch_bounds__(256) k_score_embed(IncView g, const QT* __restrict__ Q,
                                                     long long ldq, int K,
                                                     const double* __restrict__ QH,
                                                     double* __restrict__ R_out,
                                                     int32_t* __restrict__ argvec,
                                                     int32_t* __restrict__ pmax,
                                                     int32_t* __restrict__ pmin) {
  const int lane = threadIdx.x & 31;
  const long long wg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (wg >= g.m) return;
  const int i = (int)wg;
  if (g.status[0]) return;
  const int e = g.perm[i];
  const int a0 = g.ceptr[i], k = g.ceptr[i + 1] - a0;
  double R = 0.0;
  int av = -1, px = -1, pn = -1;
  if (k >= 2) {
    // pairs (a, b), a < b, in row-major order; this lane starts at pair `lane`
    int a = 0, b = 1 + lane;
    while (a < k - 1 && b >= k) {
      const int over = b - k;
      ++a;
      b = a + 1 + over;
    }
    double bd = -1.0;
    long long bt = -1;
    int ba = 0, bb = 1;
    while (a < k - 1) {
      const long long ra = (long long)dbg_index(g.cpins[a0 + a], g.n, g.status) * ldq;
      const long long rb = (long long)dbg_index(g.cpins[a0 + b], g.n, g.status) * ldq;
      double d = 0.0;
      for (int c = 0; c < K; ++c) {
        const double diff = __dsub_rn(qw<double>(Q[ra + c]), qw<double>(Q[rb + c]));
        d = __dadd_rn(d, __dmul_rn(diff, diff));
      }
      const long long t = (long long)a * k + b;  // increases with the pair order
      if (d > bd) bd = d, bt = t, ba = a, bb = b;
      b += 32;
      while (a < k - 1 && b >= k) {
        const int over = b - k;
        ++a;
        b = a + 1 + over;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double od = __shfl_xor_sync(0xffffffffu, bd, o);
      const long long ot = __shfl_xor_sync(0xffffffffu, bt, o);
      const int oa = __shfl_xor_sync(0xffffffffu, ba, o), ob = __shfl_xor_sync(0xffffffffu, bb, o);
      if (od > bd || (od == bd && ot >= 0 && (bt < 0 || ot < bt))) bd = od, bt = ot, ba = oa, bb = ob;
    }
    const int p = dbg_index(g.cpins[a0 + ba], g.n, g.status);
    const int q = dbg_index(g.cpins[a0 + bb], g.n, g.status);
    double br = -1.0;
    int bi = -1;
    for (int c = lane; c < K; c += 32) {
      const double qh = QH[c];
      if (!(qh > 1e-300)) continue;
      const double diff =
          __dsub_rn(qw<double>(Q[(long long)p * ldq + c]), qw<double>(Q[(long long)q * ldq + c]));
      const double r = __ddiv_rn(__dmul_rn(diff, diff), qh);
      if (r > br) br = r, bi = c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double orr = __shfl_xor_sync(0xffffffffu, br, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (oi >= 0 && (bi < 0 || orr > br || (orr == br && oi < bi))) br = orr, bi = oi;
    }
    if (bi >= 0) {
      R = br, av = bi;
      const bool hi = qw<double>(Q[(long long)p * ldq + bi]) >= qw<double>(Q[(long long)q * ldq + bi]);
      px = hi ? p : q;
      pn = hi ? q : p;
    }
  }
  if (lane == 0) {
    R_out[e] = R;
    if (argvec) argvec[e] = av;
    if (pmax) pmax[e] = px;
    if (pmin) pmin[e] = pn;
  }
}

// Tensor map of the row-major n x ldq matrix Q with a box of one row of bw
// elements (for tile::gather4); false when it cannot be encoded.
template <typename T>
bool encode_rows_map(CUtensorMap* tm, const T* Q, long long ldq, long long n, int bw) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
  if (!fn || n < 1 || n > 0x7fffffffll) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)ldq, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)ldq * sizeof(T)};
  const cuuint32_t box[2] = {(cuuint32_t)bw, 1u};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = fn(tm, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                        2, const_cast<T*>(Q), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
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
  // grids of co-resident CTAs only
  const int g2 = std::min(w.grid, num_sms() * resident_ctas(k_score_pass2<T, NC>, kThreads));
  T* spread = static_cast<T*>(w.spread);
  const int ldsp = spread_ld(K, sizeof(T));
  HEF_LAUNCH("k_score_big1", st, k_score_big1<T, NC><<<w.bgrid, kThreads, 0, st>>>(g, Q, ldq, K, w.bpart,
                                                                                   spread, ldsp));
  // pass 1 staged through shared memory when the rows can be bulk-copied
  // (16-byte aligned rows; a row pitch of 16-byte multiples) and at least two
  // stages fit; by four-row tensor-map gathers when a box row (K rounded up
  // to 32 bytes, at most 256 elements) fits in the pitch; otherwise the warps
  // gather the rows
  const bool aligned = (reinterpret_cast<uintptr_t>(Q) % 16 == 0) && ((size_t)ldq * sizeof(T)) % 16 == 0;
  const int bw = (int)(((size_t)K * sizeof(T) + 31) / 32 * 32 / sizeof(T));
  CUtensorMap tmap;
  memset(&tmap, 0, sizeof(tmap));
  bool g4 = aligned && bw <= 256 && bw <= ldq && encode_rows_map(&tmap, Q, ldq, inc->n, bw);
  const uint32_t row_bytes = g4 ? (uint32_t)(bw * sizeof(T)) : (uint32_t)(((size_t)K * sizeof(T) + 15) / 16 * 16);
  const size_t stage_bytes = (size_t)kWinSlots * row_bytes;
  // stages: as many as fit next to the kernel's static shared memory (and
  // 128 bytes to align the ring)
  static thread_local int stat = -1;  // static bytes of this instantiation
  if (stat < 0) {
    cudaFuncAttributes fa;
    HEF_CHECK_CUDA(cudaFuncGetAttributes(&fa, k_score_pass1_bulk<T, NC, true>));
    stat = (int)fa.sharedSizeBytes;
  }
  const size_t avail = kStageSmem > (size_t)stat + 128 ? kStageSmem - stat - 128 : 0;
  const int nst = (int)std::min<size_t>(kMaxStages, avail / stage_bytes);
  // the ring also holds the per-warp sums at the end
  const size_t smem =
      std::max(nst * stage_bytes, (size_t)(kBulkThreads / 32) * 32 * NC * sizeof(double)) + 128;
  const bool bulk = aligned && nst >= 2 && smem + stat <= kMaxSmemOptin && num_sms() <= w.grid;
  if (bulk) {
    const int pitch = (int)(row_bytes / sizeof(T));
    if (g4) {
      HEF_ENSURE_SMEM((k_score_pass1_bulk<T, NC, true>), (int)smem);
      // a programmatic dependent of k_score_big1: it runs beside it and waits
      // for it only before the reduction that reads bpart
      HEF_LAUNCH("k_score_pass1", st,
                 HEF_CHECK_CUDA(launch_dependent_smem(
                     k_score_pass1_bulk<T, NC, true>, num_sms(), kBulkThreads, smem, st, g, Q, ldq, K,
                     pitch, row_bytes, nst, red, w.bpart, w.bgrid, w.QH, w.invQH, QH_out, spread, ldsp,
                     scal_view<T>(inc).ew, inc->status, tmap)));
    } else {
      HEF_ENSURE_SMEM((k_score_pass1_bulk<T, NC, false>), (int)smem);
      HEF_LAUNCH("k_score_pass1", st,
                 HEF_CHECK_CUDA(launch_dependent_smem(
                     k_score_pass1_bulk<T, NC, false>, num_sms(), kBulkThreads, smem, st, g, Q, ldq,
                     K, pitch, row_bytes, nst, red, w.bpart, w.bgrid, w.QH, w.invQH, QH_out, spread,
                     ldsp, scal_view<T>(inc).ew, inc->status, tmap)));
    }
  } else {
    const int g1 = std::min(w.grid, num_sms() * resident_ctas(k_score_pass1<T, NC>, kThreads));
    HEF_LAUNCH("k_score_pass1", st, k_score_pass1<T, NC><<<g1, kThreads, 0, st>>>(
                                        g, Q, ldq, K, red, w.bpart, w.bgrid, w.QH, w.invQH, QH_out,
                                        w.counter + kWorkSlot, spread, ldsp));
  }
  if (reduce == HEF_REDUCE_EMBED) {
    const int ge = (int)(((long long)(inc->m > 0 ? inc->m : 1) * 32 + kThreads - 1) / kThreads);
    HEF_LAUNCH("k_score_embed", st, k_score_embed<T><<<ge, kThreads, 0, st>>>(
                                        g, Q, ldq, K, w.QH, R_out, argvec, pmax, pmin));
    HEF_CHECK_LAUNCH();
    return HEF_OK;
  }
  if (spread && reduce == HEF_REDUCE_MAX) {
    const int g3 = stride_grid((long long)(inc->m > 0 ? inc->m : 1) * kRatioLanes, 8);
    HEF_LAUNCH("k_score_ratio", st, k_score_ratio8<T><<<g3, kThreads, K * sizeof(T), st>>>(
                                        g, Q, ldq, K, w.QH, w.invQH, spread, ldsp, R_out, argvec,
                                        pmax, pmin));
    HEF_CHECK_LAUNCH();
    return HEF_OK;
  }
  if (spread) {  // the sum reduction adds a row's terms in column order
    const int g3 = stride_grid(inc->m > 0 ? inc->m : 1, 8);
    HEF_LAUNCH("k_score_ratio", st, k_score_ratio<T><<<g3, kThreads, K * sizeof(T), st>>>(
                                        g, Q, ldq, K, reduce, w.QH, w.invQH, spread, ldsp, R_out,
                                        argvec, pmax, pmin));
    HEF_CHECK_LAUNCH();
    return HEF_OK;
  }
  HEF_LAUNCH("k_score_big2", st, k_score_big2<T, NC><<<w.bgrid, kThreads, 0, st>>>(
                                     g, Q, ldq, K, reduce, w.QH, w.invQH, R_out, argvec, pmax, pmin));
  HEF_LAUNCH("k_score_pass2", st, k_score_pass2<T, NC><<<g2, kThreads, 0, st>>>(
                                      g, Q, ldq, K, reduce, w.QH, w.invQH, R_out, argvec, pmax, pmin,
                                      w.counter + kWorkSlot + 1));
  HEF_CHECK_LAUNCH();
  return HEF_OK;
}

// BF16 basis: spreads, Q_H partials and ratios in FP32 from BF16 loads;
// pass 1 gathers the rows (the staged form copies FP32 / FP64 rows) and pass
// 2 gathers them again (no stored spreads).
template <int NC>
hef_status launch_score_bf16(const hef_incidence* inc, const __nv_bfloat16* Q, long long ldq, int K,
                             int reduce, double* R_out, double* QH_out, int32_t* argvec,
                             int32_t* pmax, int32_t* pmin, const ScoreWs& w, cudaStream_t st) {
  using QT = __nv_bfloat16;
  IncView g = view(inc);
  GridRed red;
  red.part = w.part;
  red.gpart = w.gpart;
  red.gcnt = w.counter;
  red.tcnt = w.counter + 63;
  HEF_LAUNCH("k_score_big1", st, (k_score_big1<float, NC, QT><<<w.bgrid, kThreads, 0, st>>>(
                                     g, Q, ldq, K, w.bpart, nullptr, 0)));
  const int g1 = std::min(w.grid, num_sms() * resident_ctas(k_score_pass1<float, NC, QT>, kThreads));
  HEF_LAUNCH("k_score_pass1", st, (k_score_pass1<float, NC, QT><<<g1, kThreads, 0, st>>>(
                                      g, Q, ldq, K, red, w.bpart, w.bgrid, w.QH, w.invQH, QH_out,
                                      w.counter + kWorkSlot, nullptr, 0)));
  if (reduce == HEF_REDUCE_EMBED) {
    const int ge = (int)(((long long)(inc->m > 0 ? inc->m : 1) * 32 + kThreads - 1) / kThreads);
    HEF_LAUNCH("k_score_embed", st, (k_score_embed<float, QT><<<ge, kThreads, 0, st>>>(
                                        g, Q, ldq, K, w.QH, R_out, argvec, pmax, pmin)));
    HEF_CHECK_LAUNCH();
    return HEF_OK;
  }
  const int g2 = std::min(w.grid, num_sms() * resident_ctas(k_score_pass2<float, NC, QT>, kThreads));
  HEF_LAUNCH("k_score_big2", st, (k_score_big2<float, NC, QT><<<w.bgrid, kThreads, 0, st>>>(
                                     g, Q, ldq, K, reduce, w.QH, w.invQH, R_out, argvec, pmax, pmin)));
  HEF_LAUNCH("k_score_pass2", st, (k_score_pass2<float, NC, QT><<<g2, kThreads, 0, st>>>(
                                      g, Q, ldq, K, reduce, w.QH, w.invQH, R_out, argvec, pmax, pmin,
                                      w.counter + kWorkSlot + 1)));
  HEF_CHECK_LAUNCH();
  return HEF_OK;
}

hef_status dispatch_score_bf16(const hef_incidence* inc, const __nv_bfloat16* Q, long long ldq,
                               int K, int reduce, double* R_out, double* QH_out, int32_t* argvec,
                               int32_t* pmax, int32_t* pmin, const ScoreWs& w, cudaStream_t st) {
  const int nc = (K + 31) / 32;
#define HEF_SCORE_CASE(N) \
  if (nc <= N) return launch_score_bf16<N>(inc, Q, ldq, K, reduce, R_out, QH_out, argvec, pmax, pmin, w, st)
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
  // Q_H, 1/Q_H, counters, one partial row per SM for the large-hyperedge pass
  // (bgrid = num_sms() rows, as taken below), a spare group-partial row and
  // the alignment of the six takes; what is left holds the per-CTA partials
  // and their group partials (1/32 as many)
  const size_t fixed = 6 * 256 + 2 * (size_t)K * sizeof(double) + 64 * sizeof(unsigned int) +
                       (size_t)K * sizeof(double) + (size_t)num_sms() * K * sizeof(double);
  if (fixed >= cap) return cap + 1;
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
  w->bgrid = num_sms();
  w->bpart = c.take<double>((size_t)w->bgrid * K);
  w->spread = nullptr;  // no room: pass 2 gathers Q again
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
  if (dtype != HEF_F64 && dtype != HEF_F32 && dtype != HEF_BF16)
    return set_error(HEF_ERR_INVALID_ARG,
                     "hef_edge_resistance_noalloc: dtype must be HEF_F64, HEF_F32 or HEF_BF16");
  if (reduce != HEF_REDUCE_MAX && reduce != HEF_REDUCE_SUM && reduce != HEF_REDUCE_EMBED)
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
  if (dtype == HEF_BF16)
    return dispatch_score_bf16(inc, static_cast<const __nv_bfloat16*>(Q), ldq, K, reduce, R_out,
                               QH_out, argvec, pmax, pmin, w, st);
  return dispatch_score<float>(inc, static_cast<const float*>(Q), ldq, K, reduce, R_out, QH_out,
                               argvec, pmax, pmin, w, st);
}

extern "C" size_t hef_edge_resistance_workspace_bytes(const hef_incidence* inc, int32_t K) {
  if (!inc || K < 1 || K > 512) return 0;
  ScoreWs w;
  return carve_score(nullptr, K, inc->m, &w);
}

extern "C" hef_status hef_edge_resistance(const hef_incidence* inc, const void* Q, int64_t ldq,
                                          int32_t K, int32_t dtype, int32_t reduce, double* R_out,
                                          double* QH_out, int32_t* argvec, int32_t* pmax,
                                          int32_t* pmin, void* workspace, size_t workspace_bytes,
                                          void* stream) {
  HEF_NVTX("hef_edge_resistance (Algorithm 1 steps 5, 7)");
  if (!inc) return set_error(HEF_ERR_INVALID_ARG, "hef_edge_resistance: NULL incidence");
  if (K < 1 || K > 512) return set_error(HEF_ERR_UNSUPPORTED, "hef_edge_resistance: need 1 <= K <= 512");
  if (dtype != HEF_F64 && dtype != HEF_F32 && dtype != HEF_BF16)
    return set_error(HEF_ERR_INVALID_ARG,
                     "hef_edge_resistance: dtype must be HEF_F64, HEF_F32 or HEF_BF16");
  if (reduce != HEF_REDUCE_MAX && reduce != HEF_REDUCE_SUM && reduce != HEF_REDUCE_EMBED)
    return set_error(HEF_ERR_INVALID_ARG, "hef_edge_resistance: unknown reduce %d", reduce);
  if (!Q || ldq < K || (inc->m > 0 && !R_out))
    return set_error(HEF_ERR_INVALID_ARG, "hef_edge_resistance: Q or R_out NULL, or ldq < K");
  ScoreWs w;
  const size_t need = carve_score(workspace, K, inc->m, &w);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return set_error(HEF_ERR_WORKSPACE, "hef_edge_resistance: workspace needs %zu bytes (256-aligned)", need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HEF_CHECK_CUDA(cudaMemsetAsync(w.counter, 0, 64 * sizeof(unsigned int), st));
  if (dtype == HEF_F64)
    return dispatch_score<double>(inc, static_cast<const double*>(Q), ldq, K, reduce, R_out, QH_out,
                                  argvec, pmax, pmin, w, st);
  if (dtype == HEF_BF16)
    return dispatch_score_bf16(inc, static_cast<const __nv_bfloat16*>(Q), ldq, K, reduce, R_out,
                               QH_out, argvec, pmax, pmin, w, st);
  return dispatch_score<float>(inc, static_cast<const float*>(Q), ldq, K, reduce, R_out, QH_out,
                               argvec, pmax, pmin, w, st);
}
