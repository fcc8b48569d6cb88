// Orthonormalisation: Algorithm 1 step 4 ("Gram-Schmidt"), done as CholQR2
// on the mean-free basis.  Pass 1: G = V^T V - c c^T / n (c = V^T 1),
// G = R1^T R1, Q1 = (V - 1 mu^T) R1^-1.  Pass 2: the same on Q1, whose Gram
// matrix is I + E with E at rounding level, so R2 = I + X with X the
// first-order Cholesky correction of E (FP64), Q = Q1 R2^-1, R = R2 R1.  R1
// and R2 are upper triangular with positive diagonals, so Q spans the same
// nested column spaces as V: it is the Gram-Schmidt Q up to rounding.
//
// Kernels
//  k_gram         partial Gram of a row chunk: thread = 8x8 block of the
//                 upper triangle, FP32 (or FP64) accumulation per chunk, FP64
//                 partials; k_gram_reduce sums chunks in a fixed order.
//  k_chol_aug     one CTA: Gauss elimination of [G | I] -> [R | R^-T] (the
//                 inverse comes out of the same K pivot steps).  FP32 in
//                 shared memory for the FP32 form's first pass; FP64 (global
//                 scratch) as the exact path: the FP64 form's first pass, and
//                 the fallback when a fast pass reports near rank deficiency.
//  k_chol_series  second pass: R2 = I + X1, R2^-1 = I - X1 (X1 = upper part of
//                 E with halved diagonal); exact to O(|E|^2); falls back to the
//                 exact path when |E| is not small.
//  k_apply        in place Q = (V - 1 mu^T) Rinv: row blocks in shared memory,
//                 column blocks last to first (a column is overwritten only
//                 after every later column has used it), 4 x 8 outputs per
//                 thread.
#include "internal.h"

namespace hef {

namespace {

constexpr int kGB = 8;       // Gram: rows/cols of the block a thread owns
constexpr int kPR = 32;      // Gram: rows per shared-memory panel
constexpr int kPairs = 256;  // Gram: block pairs (threads) per CTA
constexpr int kACB = 64;     // apply: output columns per block
constexpr int kPB = 16;      // elimination: pivots per panel

inline int round8(int K) { return (K + 7) & ~7; }

template <typename T>
struct Acc;
template <>
struct Acc<double> {
  using type = double;
};
template <>
struct Acc<float> {
  using type = float;
};

// Block pair index -> (bi, bj), bi <= bj, row-major over the upper triangle.
__device__ __forceinline__ void pair_of(int p, int nb, int& bi, int& bj) {
  int i = 0;
  while (p >= nb - i) {
    p -= nb - i;
    ++i;
  }
  bi = i;
  bj = i + p;
}

template <typename T>
__global__ void __launch_bounds__(kPairs) k_gram(const T* __restrict__ V, long long ldv, int n,
                                                 int K, int Kp, int rows_per_chunk, double* part,
                                                 double* colpart) {
  using A = typename Acc<T>::type;
  extern __shared__ unsigned char sm_raw[];
  T* Ps = reinterpret_cast<T*>(sm_raw);  // kPR x Kp
  const int nb = Kp / kGB;
  const int npairs = nb * (nb + 1) / 2;
  const int pair = blockIdx.y * kPairs + threadIdx.x;
  const bool active = pair < npairs;
  int bi = 0, bj = 0;
  if (active) pair_of(pair, nb, bi, bj);
  const int chunk = blockIdx.x;
  const long long r0 = (long long)chunk * rows_per_chunk;
  const long long r1 = min((long long)n, r0 + rows_per_chunk);
  A acc[kGB][kGB];
  A cs[kGB];
#pragma unroll
  for (int a = 0; a < kGB; ++a) {
    cs[a] = 0;
#pragma unroll
    for (int b = 0; b < kGB; ++b) acc[a][b] = 0;
  }
  for (long long r = r0; r < r1; r += kPR) {
    __syncthreads();
    for (int e = threadIdx.x; e < kPR * Kp; e += blockDim.x) {
      const int rr = e / Kp, cc = e % Kp;
      const long long row = r + rr;
      Ps[e] = (row < r1 && cc < K) ? V[row * ldv + cc] : (T)0;
    }
    __syncthreads();
    if (active) {
      const int nr = (int)min((long long)kPR, r1 - r);
      for (int rr = 0; rr < nr; ++rr) {
        const T* prow = Ps + rr * Kp;
        A a[kGB], b[kGB];
#pragma unroll
        for (int q = 0; q < kGB; ++q) {
          a[q] = prow[bi * kGB + q];
          b[q] = prow[bj * kGB + q];
        }
#pragma unroll
        for (int x = 0; x < kGB; ++x)
#pragma unroll
          for (int y = 0; y < kGB; ++y) acc[x][y] += a[x] * b[y];
        if (bi == bj) {
#pragma unroll
          for (int q = 0; q < kGB; ++q) cs[q] += a[q];
        }
      }
    }
  }
  if (active) {
    double* P = part + ((size_t)chunk * npairs + pair) * (kGB * kGB);
#pragma unroll
    for (int x = 0; x < kGB; ++x)
#pragma unroll
      for (int y = 0; y < kGB; ++y) P[x * kGB + y] = (double)acc[x][y];
    if (bi == bj) {
#pragma unroll
      for (int q = 0; q < kGB; ++q) colpart[(size_t)chunk * Kp + bi * kGB + q] = (double)cs[q];
    }
  }
}

// G (K x K, symmetric, FP64) and c (K): fixed-order sums over chunks.
__global__ void k_gram_reduce(const double* __restrict__ part, const double* __restrict__ colpart,
                              int K, int Kp, int nchunk, double* G, double* c) {
  const int nb = Kp / kGB;
  const int npairs = nb * (nb + 1) / 2;
  const long long nel = (long long)npairs * kGB * kGB;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nel + Kp;
       idx += (long long)gridDim.x * blockDim.x) {
    if (idx < nel) {
      const int pair = (int)(idx / (kGB * kGB)), xy = (int)(idx % (kGB * kGB));
      int bi, bj;
      pair_of(pair, nb, bi, bj);
      const int i = bi * kGB + xy / kGB, j = bj * kGB + xy % kGB;
      if (i >= K || j >= K || (bi == bj && i > j)) continue;
      double s = 0.0;
      for (int q = 0; q < nchunk; ++q) s += part[(size_t)q * nel + idx];
      G[(size_t)i * K + j] = s;
      G[(size_t)j * K + i] = s;
    } else {
      const int i = (int)(idx - nel);
      if (i >= K) continue;
      double s = 0.0;
      for (int q = 0; q < nchunk; ++q) s += colpart[(size_t)q * Kp + i];
      c[i] = s;
    }
  }
}

// A = G - c c^T / n (FP64, and an FP32 copy for the fast factorisation),
// over the whole grid so the one-CTA factorisation does no FP64 set-up work.
__global__ void k_gram_project(const double* __restrict__ G, const double* __restrict__ c, int K,
                               double n, double* A64, float* A32) {
  const long long KK = (long long)K * K;
  const double inv_n = 1.0 / n;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < KK;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / K), j = (int)(idx % K);
    const double v = G[idx] - c[i] * (c[j] * inv_n);
    A64[idx] = v;
    A32[idx] = (float)v;
  }
}

struct CholOut {
  void* Rinv;      // Kp x Kp, element type T, upper triangular, zero padded
  void* mu;        // Kp, element type T
  double* R;       // K x K upper (FP64), for R_out
  int* kept;       // K
  int* rank;       // 1
  int* flag;       // [0] exact pass needed
};

// Barrier among the first `count` threads of the CTA (named barrier `id`).
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// 1 / sqrt(pivot) in the elimination's arithmetic type.
template <typename C>
__device__ __forceinline__ C pivot_rsqrt(C d);
template <>
__device__ __forceinline__ float pivot_rsqrt<float>(float d) {
  return rsqrtf(d);  // the fast path's R is refined by the second CholQR pass
}
template <>
__device__ __forceinline__ double pivot_rsqrt<double>(double d) {
  return 1.0 / sqrt(d);
}

// Gauss elimination of [A | I] with A = G - c c^T / n: after pivot j, row j
// holds R[j][j..K) on the left and (R^-T)[j][0..j] on the right.  Columns
// whose pivot is <= tol * G_jj are dropped (their rows stay zero).
// C: arithmetic type; W: the K x 2K work matrix (shared or global memory).
// fast = 1: report (flag) any kept pivot <= 1e-4 G_jj instead of trusting
// it.  fast = 0: exact path; runs only when `flag` is set unless `always`.
template <typename C, typename T, int THREADS = 1024>
__global__ void __launch_bounds__(THREADS) k_chol_aug(const double* __restrict__ G,
                                                   const double* __restrict__ c,
                                                   const C* __restrict__ Aproj, int K, int Kp,
                                                   double n, double tol, C* Wg, int use_smem,
                                                   int fast, int always, CholOut o) {
  extern __shared__ unsigned char sm_raw[];
  __shared__ C ref[512], thr_keep[512], thr_near[512];
  __shared__ int pk[kPB];  // kept flags of the current panel
  __shared__ int near_def;
  if (!fast && !always && o.flag[0] == 0) return;
  C* W = use_smem ? reinterpret_cast<C*>(sm_raw) : Wg;
  const int W2 = 2 * K;
  for (int i = (int)(threadIdx.x >> 5); i < K; i += (int)(blockDim.x >> 5)) {
    C* row = W + (size_t)i * W2;
    for (int j = (int)(threadIdx.x & 31); j < W2; j += 32)
      row[j] = j < K ? Aproj[(size_t)i * K + j] : (j - K == i ? (C)1 : (C)0);
  }
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    // pivot thresholds in the elimination's own type (no FP64 on the pivot path)
    const double gi = G[(size_t)i * K + i];
    ref[i] = (C)gi;
    thr_keep[i] = (C)(tol * gi);
    thr_near[i] = (C)(1e-4 * gi);
  }
  if (threadIdx.x == 0) near_def = 0;
  __syncthreads();
  // Blocked: a panel of kPB pivots is eliminated among its own rows by kPB
  // warps (warp w owns panel row j0 + w; two named-barrier steps per pivot:
  // the owner of row j scales it, then the later panel rows eliminate column
  // j), then every later row takes the panel's rank-kPB update in one sweep.
  // Row j's live columns after its pivot: left j..K-1, right 0..j (K + 1
  // values).
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j0 = 0; j0 < K; j0 += kPB) {
    const int jend = min(K, j0 + kPB);
    if (wid < kPB) {
      const int i = j0 + wid;
      C* rowi = W + (size_t)i * W2;
      for (int j = j0; j < jend; ++j) {
        C* rowj = W + (size_t)j * W2;
        if (i == j) {  // owner: pivot, kept flag, scale the live columns
          int kj = 0;
          C pinv = 0;
          if (lane == 0) {
            const C d = rowj[j];
            kj = (ref[j] > (C)0 && d > thr_keep[j]) ? 1 : 0;
            if (fast && kj && d <= thr_near[j]) near_def = 1;
            if (kj) pinv = pivot_rsqrt<C>(d);
            o.kept[j] = kj;
            pk[j - j0] = kj;
          }
          kj = __shfl_sync(0xffffffffu, kj, 0);
          pinv = __shfl_sync(0xffffffffu, pinv, 0);
          for (int q0 = lane; q0 <= K; q0 += 32) {
            const int q = q0 < K - j ? j + q0 : K + (q0 - (K - j));
            rowj[q] = kj ? rowj[q] * pinv : (C)0;
          }
        }
        named_sync(1, kPB * 32);
        if (i > j && i < jend && pk[j - j0]) {  // eliminate column j from row i
          const C r = rowj[i];
          const int nleft = K - j - 1;
          for (int q0 = lane; q0 < K; q0 += 32) {
            const int q = q0 < nleft ? j + 1 + q0 : K + (q0 - nleft);
            rowi[q] -= r * rowj[q];
          }
        }
        named_sync(1, kPB * 32);
      }
    }
    __syncthreads();
    // rank-kPB update of rows i >= jend.  Their live columns (left jend..K-1,
    // right 0..jend-1) are the contiguous range [jend, K + jend) of the row.
    int npb = 0;
#pragma unroll
    for (int p = 0; p < kPB; ++p) npb += (j0 + p < jend) ? 1 : 0;
    if (sizeof(C) == 4 && (K & 3) == 0 && (jend & 3) == 0) {
      // FP32: four columns per lane (16-byte shared-memory accesses), kUR rows
      // per warp at a time, so that a lane has 4 kUR independent FMA chains
      // (one row with 1024 threads, whose 64 registers hold no more)
      constexpr int kUR = THREADS >= 1024 ? 1 : 4;
      for (int i0 = jend + wid * kUR; i0 < K; i0 += nw * kUR) {
        float rj[kUR][kPB];
#pragma unroll
        for (int r = 0; r < kUR; ++r)
#pragma unroll
          for (int p = 0; p < kPB; ++p)
            rj[r][p] = (i0 + r < K && p < npb && pk[p]) ? (float)W[(size_t)(j0 + p) * W2 + i0 + r] : 0.0f;
        for (int v = lane; v < K / 4; v += 32) {
          float4 acc[kUR];
#pragma unroll
          for (int r = 0; r < kUR; ++r)
            acc[r] = i0 + r < K ? reinterpret_cast<const float4*>(
                                      reinterpret_cast<const float*>(W + (size_t)(i0 + r) * W2) + jend)[v]
                                : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int p = 0; p < kPB; ++p) {
            const float4 b =
                reinterpret_cast<const float4*>(reinterpret_cast<float*>(W + (size_t)(j0 + p) * W2) + jend)[v];
#pragma unroll
            for (int r = 0; r < kUR; ++r) {
              acc[r].x -= rj[r][p] * b.x, acc[r].y -= rj[r][p] * b.y;
              acc[r].z -= rj[r][p] * b.z, acc[r].w -= rj[r][p] * b.w;
            }
          }
#pragma unroll
          for (int r = 0; r < kUR; ++r)
            if (i0 + r < K)
              reinterpret_cast<float4*>(reinterpret_cast<float*>(W + (size_t)(i0 + r) * W2) + jend)[v] = acc[r];
        }
      }
    } else {
      for (int i = jend + wid; i < K; i += nw) {
        C* rowi = W + (size_t)i * W2 + jend;
        C rj[kPB];
#pragma unroll
        for (int p = 0; p < kPB; ++p)
          rj[p] = (p < npb && pk[p]) ? W[(size_t)(j0 + p) * W2 + i] : (C)0;
        for (int q0 = lane; q0 < K; q0 += 32) {
          C acc = rowi[q0];
#pragma unroll
          for (int p = 0; p < kPB; ++p) acc -= rj[p] * W[(size_t)(j0 + p) * W2 + jend + q0];
          rowi[q0] = acc;
        }
      }
    }
    __syncthreads();
  }
  // outputs: R (FP64), Rinv = (R^-T)^T (type T), mu, rank, flag
  T* Rinv = static_cast<T*>(o.Rinv);
  T* mu = static_cast<T*>(o.mu);
  // lanes run along W's rows (conflict-free shared-memory reads)
  for (int j = (int)(threadIdx.x >> 5); j < Kp; j += (int)(blockDim.x >> 5)) {
    for (int i = (int)(threadIdx.x & 31); i < Kp; i += 32) {
      C v = 0;
      if (i < K && j < K && i <= j) v = W[(size_t)j * W2 + K + i];
      Rinv[(size_t)i * Kp + j] = (T)v;
      if (o.R && i < K && j < K) o.R[(size_t)j * K + i] = (j <= i) ? (double)W[(size_t)j * W2 + i] : 0.0;
    }
  }
  for (int i = threadIdx.x; i < Kp; i += blockDim.x) mu[i] = i < K ? (T)(c[i] / n) : (T)0;
  __syncthreads();
  if (threadIdx.x == 0) {
    int r = 0;
    for (int j = 0; j < K; ++j) r += o.kept[j];
    *o.rank = r;
    if (fast) o.flag[0] = near_def;
  }
}

// The FP32 form's first-pass factorisation when [A | I] fits in shared memory
// (Kq = K rounded up to 4, Kq <= kPanelMaxK; the padded pivots are dropped):
// the same elimination, outputs and pivot rules as k_chol_aug with fast = 1,
// organised so that one CTA keeps all its warps busy.  Per panel of kCP
// pivots:
//  (a) warp 0 eliminates [D | I] in registers, D the panel's diagonal block
//      (lane c < 16 holds column c of D, lane 16 + c column c of I): R11 and
//      the lower triangular T with T D = R11, i.e. the panel's row operations;
//  (b) all threads apply T to the panel rows' other live columns
//      [jend, Kq + j0) (the right half's block at Kq + j0 becomes T itself);
//  (c) rows i >= jend take the rank-kCP update on their live columns
//      [jend, Kq + jend) in 4 x 4 tiles (multipliers R[p][i] read as float4).
// R^-1 leaves transposed through the left half of W (skewed 32 x 32 blocks,
// no bank conflicts on either side) so that its global stores coalesce.
constexpr int kCP = 16;
constexpr int kPanelThreads = 512;
constexpr int kPanelMaxK = 160;

inline size_t panel_smem(int K) {
  const size_t Kq = (size_t)((K + 3) & ~3);
  return Kq * 2 * Kq * sizeof(float);
}
inline bool panel_supported(int K) { return ((K + 3) & ~3) <= kPanelMaxK; }

template <typename T>  // float: R^-1 and mu of the FP32 and BF16 forms
__global__ void __launch_bounds__(kPanelThreads, 1) k_chol_panels(const double* __restrict__ G,
                                                              const double* __restrict__ c,
                                                              const float* __restrict__ Aproj, int K,
                                                              int Kp, double n, double tol, CholOut o) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ float ref[kPanelMaxK], thr_keep[kPanelMaxK], thr_near[kPanelMaxK];
  __shared__ float Ts[kCP][kCP];
  __shared__ int keptS[kPanelMaxK];
  __shared__ int near_def;
  float* W = reinterpret_cast<float*>(sm_raw);
  const int Kq = (K + 3) & ~3, W2 = 2 * Kq;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // [A | I]: every load of A issued before the first store (A is L2-resident)
  {
    constexpr int kIt = (kPanelMaxK * kPanelMaxK / 4 + kPanelThreads - 1) / kPanelThreads;
    const int nq = Kq / 4;
    if ((K & 3) == 0) {  // rows of A are whole float4s
      float4 buf[kIt];
#pragma unroll
      for (int t = 0; t < kIt; ++t) {
        const int idx = tid + t * kPanelThreads;
        buf[t] = idx < K * nq ? reinterpret_cast<const float4*>(Aproj)[idx] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int t = 0; t < kIt; ++t) {
        const int idx = tid + t * kPanelThreads;
        if (idx < K * nq) reinterpret_cast<float4*>(W + (size_t)(idx / nq) * W2)[idx % nq] = buf[t];
      }
    } else {
      for (int idx = tid; idx < Kq * Kq; idx += kPanelThreads) {
        const int i = idx / Kq, j = idx % Kq;
        W[(size_t)i * W2 + j] = (i < K && j < K) ? Aproj[(size_t)i * K + j] : 0.0f;
      }
    }
    // right half: the identity on rows < K
    for (int idx = tid; idx < Kq * nq; idx += kPanelThreads) {
      const int i = idx / nq, q = idx % nq, d = i - 4 * q;
      const float one = i < K ? 1.0f : 0.0f;
      reinterpret_cast<float4*>(W + (size_t)i * W2 + Kq)[q] =
          make_float4(d == 0 ? one : 0.f, d == 1 ? one : 0.f, d == 2 ? one : 0.f, d == 3 ? one : 0.f);
    }
    for (int i = tid; i < Kq; i += kPanelThreads) {
      const double gi = i < K ? G[(size_t)i * K + i] : 0.0;
      ref[i] = (float)gi;
      thr_keep[i] = (float)(tol * gi);
      thr_near[i] = (float)(1e-4 * gi);
    }
    if (tid == 0) near_def = 0;
  }
  __syncthreads();
  for (int j0 = 0; j0 < Kq; j0 += kCP) {
    const int np = min(kCP, Kq - j0), jend = j0 + np;  // np is a multiple of 4
    // (a)
    if (wid == 0) {
      const int col = lane & 15;
      const bool left = lane < 16;
      float v[kCP];
#pragma unroll
      for (int r = 0; r < kCP; ++r)
        v[r] = left ? ((r < np && col < np) ? W[(size_t)(j0 + r) * W2 + j0 + col] : 0.0f)
                    : (r == col ? 1.0f : 0.0f);
      const int jl = j0 + col;
      const float my_ref = jl < Kq ? ref[jl] : 0.0f;
      const float my_keep = jl < Kq ? thr_keep[jl] : 0.0f;
      const float my_near = jl < Kq ? thr_near[jl] : 0.0f;
      unsigned kept_mask = 0;
      int near = 0;
#pragma unroll
      for (int p = 0; p < kCP; ++p) {
        if (p < np) {  // warp-uniform
          const float d = __shfl_sync(0xffffffffu, v[p], p);
          const float rf = __shfl_sync(0xffffffffu, my_ref, p);
          const float tk = __shfl_sync(0xffffffffu, my_keep, p);
          const float tn = __shfl_sync(0xffffffffu, my_near, p);
          const int kj = (j0 + p < K && rf > 0.0f && d > tk) ? 1 : 0;
          near |= (kj && d <= tn) ? 1 : 0;
          kept_mask |= (unsigned)kj << p;
          v[p] *= kj ? rsqrtf(d) : 0.0f;  // R refined by the second CholQR pass
          if (kj) {
#pragma unroll
            for (int i = p + 1; i < kCP; ++i) {
              const float r = __shfl_sync(0xffffffffu, v[p], i);  // scaled (j0 + p, j0 + i)
              v[i] -= r * v[p];
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < kCP; ++r) {
        if (left) {
          if (r < np && col < np) W[(size_t)(j0 + r) * W2 + j0 + col] = r <= col ? v[r] : 0.0f;
        } else {
          Ts[r][col] = v[r];
          if (r < np && col < np) W[(size_t)(j0 + r) * W2 + Kq + j0 + col] = v[r];
        }
      }
      if (lane < np && j0 + lane < K) {
        const int kj = (int)((kept_mask >> lane) & 1u);
        keptS[j0 + lane] = kj;
        o.kept[j0 + lane] = kj;
      }
      if (lane == 0 && near) near_def = 1;
    }
    __syncthreads();
    // (b) two items (row r, 4 columns) per thread at most: np (Kq - np) / 4 <= 2 x 512
    {
      const int ncg = (Kq - np) / 4;
      const int nit = np * ncg;
      float4 res[2];
#pragma unroll
      for (int sl = 0; sl < 2; ++sl) {
        const int it = tid + sl * kPanelThreads;
        res[sl] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (it < nit) {
          const int r = it / ncg, cg = it % ncg;
          const float* base = W + (size_t)j0 * W2 + jend + 4 * cg;
          for (int p = 0; p <= r; ++p) {
            const float t = Ts[r][p];
            const float4 x = *reinterpret_cast<const float4*>(base + (size_t)p * W2);
            res[sl].x += t * x.x, res[sl].y += t * x.y, res[sl].z += t * x.z, res[sl].w += t * x.w;
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int sl = 0; sl < 2; ++sl) {
        const int it = tid + sl * kPanelThreads;
        if (it < nit) {
          const int r = it / ncg, cg = it % ncg;
          *reinterpret_cast<float4*>(W + (size_t)(j0 + r) * W2 + jend + 4 * cg) = res[sl];
        }
      }
    }
    __syncthreads();
    // (c)
    {
      const int ncg = Kq / 4;
      const int nit = (Kq - jend) / 4 * ncg;
      for (int it = tid; it < nit; it += kPanelThreads) {
        const int i0 = jend + 4 * (it / ncg), c0 = jend + 4 * (it % ncg);
        float4 acc[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r] = *reinterpret_cast<const float4*>(W + (size_t)(i0 + r) * W2 + c0);
#pragma unroll
        for (int p = 0; p < kCP; ++p) {
          if (p < np) {
            const float* rowp = W + (size_t)(j0 + p) * W2;
            const float4 a = *reinterpret_cast<const float4*>(rowp + i0);
            const float4 b = *reinterpret_cast<const float4*>(rowp + c0);
            const float am[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              acc[r].x -= am[r] * b.x, acc[r].y -= am[r] * b.y;
              acc[r].z -= am[r] * b.z, acc[r].w -= am[r] * b.w;
            }
          }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) *reinterpret_cast<float4*>(W + (size_t)(i0 + r) * W2 + c0) = acc[r];
      }
    }
    __syncthreads();
  }
  // outputs: R (FP64, row j: columns i >= j), then R^-1 = (R^-T)^T by way of
  // the left half, mu, rank, flag
  if (o.R)
    for (int idx = tid; idx < K * K; idx += kPanelThreads) {
      const int j = idx / K, i = idx % K;
      o.R[idx] = j <= i ? (double)W[(size_t)j * W2 + i] : 0.0;
    }
  __syncthreads();
  {
    // block (bi, bj), bi <= bj; lane l moves (i, j) = (32 bi + (l + t) % 32,
    // 32 bj + l): bank (W2 + 1) l + const on the read, W2 ((l + t) % 32) + l
    // on the write, distinct over the warp (W2 even)
    const int nb = (Kq + 31) / 32;
    const int npair = nb * (nb + 1) / 2;
    for (int pr = wid; pr < npair; pr += kPanelThreads / 32) {
      int bi = 0, rem = pr;
      while (rem >= nb - bi) rem -= nb - bi, ++bi;
      const int bj = bi + rem;
      const int j = 32 * bj + lane;
      for (int t = 0; t < 32; ++t) {
        const int i = 32 * bi + ((lane + t) & 31);
        if (i < Kq && j < Kq && i <= j) W[(size_t)i * W2 + j] = W[(size_t)j * W2 + Kq + i];
      }
    }
  }
  __syncthreads();
  T* Rinv = static_cast<T*>(o.Rinv);
  T* mu = static_cast<T*>(o.mu);
  // Kp is a multiple of 8: four columns of R^-1 per store
  const int kp4 = Kp / 4;
  for (int idx = tid; idx < Kp * kp4; idx += kPanelThreads) {
    const int i = idx / kp4, j0 = 4 * (idx % kp4);
    float x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = j0 + u;
      x[u] = (i < K && j < K && i <= j) ? W[(size_t)i * W2 + j] : 0.0f;
    }
    reinterpret_cast<float4*>(Rinv)[idx] = make_float4(x[0], x[1], x[2], x[3]);
  }
  for (int i = tid; i < Kp; i += kPanelThreads) mu[i] = i < K ? (T)(c[i] / n) : (T)0;
  if (wid == 0) {
    int r = 0;
    for (int j = lane; j < K; j += 32) r += keptS[j];
    r = __reduce_add_sync(0xffffffffu, r);
    if (lane == 0) {
      *o.rank = r;
      o.flag[0] = near_def;
    }
  }
}

// Second pass from the Gram of Q1 (= I + E up to rounding): R2 = I + X1 and
// R2^-1 = I - X1, X1 = strict upper part of E plus half its diagonal.  Sets
// flag[0] when max|E| > gtol (the exact path then recomputes; flag must be
// zero on entry).  Columns with G_jj == 0 (dropped in pass 1) stay dropped.
template <typename T>
__global__ void k_chol_series(const double* __restrict__ G, const double* __restrict__ c, int K,
                              int Kp, double n, double gtol, CholOut o) {
  T* Rinv = static_cast<T*>(o.Rinv);
  T* mu = static_cast<T*>(o.mu);
  bool bad = false;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)Kp * Kp;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / Kp), j = (int)(idx % Kp);
    double rv = 0.0, riv = 0.0;
    if (i < K && j < K && i <= j) {
      const bool ki = G[(size_t)i * K + i] > 0.0, kj = G[(size_t)j * K + j] > 0.0;
      if (ki && kj) {
        const double e = G[(size_t)i * K + j] - c[i] * c[j] / n - (i == j ? 1.0 : 0.0);
        if (!(fabs(e) <= gtol)) bad = true;
        const double x = (i == j) ? 0.5 * e : e;
        rv = (i == j ? 1.0 : 0.0) + x;
        riv = (i == j ? 1.0 : 0.0) - x;
      }
    }
    Rinv[idx] = (T)riv;
    if (i < K && j < K) o.R[(size_t)i * K + j] = rv;
  }
  if (bad) atomicOr(o.flag, 1);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Kp;
       i += (long long)gridDim.x * blockDim.x) {
    mu[i] = i < K ? (T)(c[i] / n) : (T)0;
    if (i < K) o.kept[i] = G[(size_t)i * K + i] > 0.0 ? 1 : 0;
  }
}

// rank = number of kept columns, or -1 when a tensor-core wait timed out
// (flag[1]).
__global__ void k_rank(const int* kept, int K, const int* flag, int* rank) {
  if (threadIdx.x == 0) {
    int r = 0;
    for (int j = 0; j < K; ++j) r += kept[j];
    *rank = flag[1] ? -1 : r;
  }
}

// Q = (V - 1 mu^T) Rinv in place.  CTA: RB rows x all Kp columns in shared
// memory (row stride Kp + 1), output blocks of kACB columns from the last;
// thread: 4 rows x 8 columns.
// stage_r = 0 (large K in FP64): Rinv is read from global memory (L1/L2)
// instead of being staged per column block.
template <typename T>
__global__ void __launch_bounds__(256) k_apply(T* V, long long ldv, int n, int K, int Kp,
                                               const T* __restrict__ Rinv,
                                               const T* __restrict__ mu, int RB, int stage_r) {
  extern __shared__ unsigned char sm_raw[];
  const int ldv_s = Kp + 1;
  T* Vs = reinterpret_cast<T*>(sm_raw);     // RB x (Kp + 1)
  T* Rs = Vs + (size_t)RB * ldv_s;          // Kp x kACB
  Rs = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(Rs) + 15) & ~uintptr_t(15));
  const long long r0 = (long long)blockIdx.x * RB;
  const int nrow = (int)min((long long)RB, (long long)n - r0);
  for (int e = threadIdx.x; e < RB * Kp; e += blockDim.x) {
    const int rr = e / Kp, cc = e % Kp;
    Vs[rr * ldv_s + cc] = (rr < nrow && cc < K) ? V[(r0 + rr) * ldv + cc] - mu[cc] : (T)0;
  }
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;  // 8 column groups x RB/4 row groups
  const int nblk = (Kp + kACB - 1) / kACB;
  for (int J = nblk - 1; J >= 0; --J) {
    const int c0 = J * kACB;
    const int cw = min(kACB, Kp - c0);
    const int iend = c0 + cw;  // Rinv upper triangular: rows < iend
    __syncthreads();
    if (stage_r) {
      for (int e = threadIdx.x; e < iend * kACB; e += blockDim.x) {
        const int i = e / kACB, jj = e % kACB;
        Rs[e] = (jj < cw) ? Rinv[(size_t)i * Kp + c0 + jj] : (T)0;
      }
    }
    __syncthreads();
    T acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0;
    const T* vrow = Vs + (ty * 4) * ldv_s;
#pragma unroll 4
    for (int i = 0; i < iend; ++i) {
      T a[4], b[8];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = vrow[r * ldv_s + i];
      if (stage_r) {
        const T* rrow = Rs + i * kACB + tx * 8;
#pragma unroll
        for (int q = 0; q < 8; ++q) b[q] = rrow[q];
      } else {
        const T* rrow = Rinv + (size_t)i * Kp + c0 + tx * 8;
#pragma unroll
        for (int q = 0; q < 8; ++q) b[q] = (tx * 8 + q < cw) ? __ldg(rrow + q) : (T)0;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[r][q] += a[r] * b[q];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int col = c0 + tx * 8 + q;
        if (tx * 8 + q < cw) Vs[(ty * 4 + r) * ldv_s + col] = acc[r][q];
      }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nrow * K; e += blockDim.x) {
    const int rr = e / K, cc = e % K;
    V[(r0 + rr) * ldv + cc] = Vs[rr * ldv_s + cc];
  }
}

// R_out = R2 * R1 (both upper triangular, FP64).
__global__ void k_trmm_upper(const double* R2, const double* R1, int K, double* Rout) {
  const long long KK = (long long)K * K;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < KK;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / K), j = (int)(idx % K);
    double s = 0.0;
    for (int l = i; l <= j; ++l) s += R2[(size_t)i * K + l] * R1[(size_t)l * K + j];
    Rout[idx] = (i <= j) ? s : 0.0;
  }
}

struct OrthoWs {
  double* part;
  double* colpart;
  double* G;
  double* c;
  double* Wg;  // K x 2K FP64 scratch of the exact path
  double* A64; // projected Gram (FP64)
  float* A32;  // projected Gram (FP32 copy)
  double* R1;
  double* R2;
  void* Rinv;
  void* mu;
  int* kept;
  int* rank;
  int* flag;
  float* tcs;  // tensor-core apply scratch (FP32 form)
  int nchunk;
  int rows_per_chunk;
  int ngroups;
};

size_t carve_ortho(void* base, long long n, int K, int dtype, OrthoWs* w) {
  Carver cv(base);
  const int Kp = round8(K);
  const int nb = Kp / kGB;
  const int npairs = nb * (nb + 1) / 2;
  w->ngroups = (npairs + kPairs - 1) / kPairs;
  int nchunk = (num_sms() * 2 + w->ngroups - 1) / w->ngroups;
  const long long max_chunks = (n + kPR - 1) / kPR;
  if (nchunk > max_chunks) nchunk = (int)(max_chunks > 0 ? max_chunks : 1);
  w->nchunk = nchunk;
  w->rows_per_chunk = (int)(((n + nchunk - 1) / nchunk + kPR - 1) / kPR * kPR);
  const size_t KK = (size_t)K * K;
  const size_t esz = dtype == HEF_F64 ? 8 : 4;  // of R^-1 and mu (FP32 for the BF16 basis)
  size_t npart = (size_t)nchunk * npairs * kGB * kGB;
  if (dtype != HEF_F64 && gram_tc_supported(K)) {
    const size_t tc = gram_tc_part_doubles(n, K);
    if (tc > npart) npart = tc;
  }
  w->part = cv.take<double>(npart);
  w->colpart = cv.take<double>((size_t)nchunk * Kp);
  w->G = cv.take<double>(KK);
  w->c = cv.take<double>(K);
  w->Wg = cv.take<double>(2 * KK);
  w->A64 = cv.take<double>(KK);
  w->A32 = cv.take<float>(KK);
  w->R1 = cv.take<double>(KK);
  w->R2 = cv.take<double>(KK);
  w->Rinv = cv.take<char>((size_t)Kp * Kp * esz);
  w->mu = cv.take<char>((size_t)Kp * esz);
  w->kept = cv.take<int>(K);
  w->rank = cv.take<int>(4);
  w->flag = cv.take<int>(4);
  w->tcs = cv.take<float>(dtype != HEF_F64 && apply_tc_supported(K) ? apply_tc_scratch_floats(K) : 1);
  return cv.bytes();
}

// bf16: V holds the basis as BF16 (T = float is then the type of R^-1 and
// the elimination; the Gram and the apply run on the tensor cores).
template <typename T>
hef_status run_ortho(long long n, int K, T* V, long long ldv, double* R_out, int* rank_out,
                     const OrthoWs& w, cudaStream_t st, bool bf16 = false) {
  const int Kp = round8(K);
  const size_t gram_smem = (size_t)kPR * Kp * sizeof(T);
  HEF_ENSURE_SMEM(k_gram<T>, (int)gram_smem);
  const dim3 ggrid(w.nchunk, w.ngroups);
  const int nb = Kp / kGB;
  const long long nel = (long long)nb * (nb + 1) / 2 * kGB * kGB;
  const int rgrid = stride_grid(nel + Kp, 4);
  int stage_r = 1;
  auto apply_smem = [&](int rb) {
    return ((size_t)rb * (Kp + 1) + (stage_r ? (size_t)Kp * kACB : 0)) * sizeof(T) + 16;
  };
  int RB = 128;
  while (RB > 32 && apply_smem(RB) > 200 * 1024) RB /= 2;
  if (apply_smem(RB) > 200 * 1024) {
    stage_r = 0;
    RB = 128;
    while (RB > 32 && apply_smem(RB) > 200 * 1024) RB /= 2;
  }
  if (apply_smem(RB) > 200 * 1024)
    return set_error(HEF_ERR_UNSUPPORTED, "hef_orthonormalize: K = %d too large", K);
  HEF_ENSURE_SMEM(k_apply<T>, (int)apply_smem(RB));
  const int agrid = (int)((n + RB - 1) / RB);
  const int athreads = RB * 2;  // (RB / 4) row groups x 8 column groups
  // FP32 form: the FP32 elimination works in shared memory when [A | I]
  // fits (K <= 160), else in the (L2-resident) FP64 scratch reused as FP32
  const size_t fast_smem = (size_t)K * 2 * K * sizeof(float);
  const bool fast_ok = sizeof(T) == 4;
  const bool fast_in_smem = fast_ok && fast_smem <= 200 * 1024;
  const bool panels = fast_ok && panel_supported(K);
  if (fast_in_smem) HEF_ENSURE_SMEM((k_chol_aug<float, T>), fast_smem);
  if (panels) HEF_ENSURE_SMEM(k_chol_panels<T>, panel_smem(K));
  const double tol = sizeof(T) == 8 ? 1e-12 : 1e-5;
  // second pass: the first-order factor of the near-identity Gram is exact to
  // O(|E|^2); a BF16 basis leaves |E| near its rounding (~4e-3), where the
  // O(|E|^2) term is far below that precision
  const double gtol = sizeof(T) == 8 ? 1e-8 : (bf16 ? 1e-2 : 1e-4);
  double* Rs[2] = {w.R1, w.R2};

  const bool use_tc = sizeof(T) == 4 && gram_tc_supported(K);
  const bool want_R = R_out != nullptr;
  HEF_CHECK_CUDA(cudaMemsetAsync(w.flag, 0, 4 * sizeof(int), st));
  for (int pass = 0; pass < 2; ++pass) {
    CholOut o{w.Rinv, w.mu, Rs[pass], w.kept, w.rank, w.flag};
    if (use_tc) {
      hef_status s = gram_tc(V, bf16, ldv, n, K, w.part, w.G, w.c, w.flag + 1, st);
      if (s) return s;
    } else {
      HEF_LAUNCH("k_gram", st, k_gram<T><<<ggrid, kPairs, gram_smem, st>>>(
                                   V, ldv, (int)n, K, Kp, w.rows_per_chunk, w.part, w.colpart));
      HEF_LAUNCH("k_gram_reduce", st, k_gram_reduce<<<rgrid, kThreads, 0, st>>>(
                                          w.part, w.colpart, K, Kp, w.nchunk, w.G, w.c));
      HEF_CHECK_LAUNCH();
    }
    if (pass == 0) {
      if (!want_R) o.R = nullptr;
      HEF_LAUNCH("k_gram_project", st, k_gram_project<<<stride_grid((long long)K * K, 2), kThreads, 0,
                                                         st>>>(w.G, w.c, K, (double)n, w.A64, w.A32));
      if (fast_ok) {
        if (panels) {
          HEF_LAUNCH("k_chol_panels", st, k_chol_panels<T><<<1, kPanelThreads, panel_smem(K), st>>>(
                                              w.G, w.c, w.A32, K, Kp, (double)n, tol, o));
        } else {
          HEF_LAUNCH("k_chol_aug", st, k_chol_aug<float, T><<<1, 1024, fast_in_smem ? fast_smem : 0, st>>>(
                                           w.G, w.c, w.A32, K, Kp, (double)n, tol,
                                           fast_in_smem ? nullptr : reinterpret_cast<float*>(w.Wg),
                                           fast_in_smem ? 1 : 0, 1, 0, o));
        }
      }
      // exact FP64 path: always for the FP64 form, on demand for the FP32 form
      HEF_LAUNCH("k_chol_aug", st, k_chol_aug<double, T><<<1, 1024, 0, st>>>(
                                       w.G, w.c, w.A64, K, Kp, (double)n, tol, w.Wg, 0, 0,
                                       fast_ok ? 0 : 1, o));
    } else {
      HEF_CHECK_CUDA(cudaMemsetAsync(w.flag, 0, sizeof(int), st));  // flag[0] only
      HEF_LAUNCH("k_chol_series", st, k_chol_series<T><<<stride_grid((long long)Kp * Kp, 2),
                                                        kThreads, 0, st>>>(
                                          w.G, w.c, K, Kp, (double)n, gtol, o));
      HEF_LAUNCH("k_gram_project_exact", st,
                 k_gram_project<<<stride_grid((long long)K * K, 2), kThreads, 0, st>>>(
                     w.G, w.c, K, (double)n, w.A64, w.A32));
      HEF_LAUNCH("k_chol_aug", st, k_chol_aug<double, T><<<1, 1024, 0, st>>>(
                                       w.G, w.c, w.A64, K, Kp, (double)n, tol, w.Wg, 0, 0, 0, o));
      HEF_LAUNCH("k_rank", st, k_rank<<<1, 32, 0, st>>>(w.kept, K, w.flag, w.rank));
    }
    HEF_CHECK_LAUNCH();
    if (sizeof(T) == 4 && apply_tc_supported(K)) {
      hef_status s = apply_tc(V, bf16, ldv, n, K, static_cast<const float*>(w.Rinv), Kp,
                              static_cast<const float*>(w.mu), w.tcs, w.flag + 1, st);
      if (s) return s;
    } else {
      HEF_LAUNCH("k_apply", st, k_apply<T><<<agrid, athreads, apply_smem(RB), st>>>(
                                    V, ldv, (int)n, K, Kp, static_cast<const T*>(w.Rinv),
                                    static_cast<const T*>(w.mu), RB, stage_r));
      HEF_CHECK_LAUNCH();
    }
  }
  if (R_out) {
    HEF_LAUNCH("k_trmm_upper", st, k_trmm_upper<<<stride_grid((long long)K * K, 4), kThreads, 0,
                                                  st>>>(w.R2, w.R1, K, R_out));
    HEF_CHECK_LAUNCH();
  }
  if (rank_out)
    HEF_CHECK_CUDA(cudaMemcpyAsync(rank_out, w.rank, sizeof(int), cudaMemcpyDeviceToDevice, st));
  return HEF_OK;
}

}  // namespace

}  // namespace hef

using namespace hef;

extern "C" size_t hef_orthonormalize_workspace_bytes(int64_t n, int32_t K, int32_t dtype) {
  if (n < 1 || K < 1 || K > 512 || (dtype != HEF_F64 && dtype != HEF_F32 && dtype != HEF_BF16))
    return 0;
  if (dtype == HEF_BF16 && !(gram_tc_supported(K) && apply_tc_supported(K))) return 0;
  OrthoWs w;
  return carve_ortho(nullptr, n, K, dtype, &w);
}

extern "C" hef_status hef_orthonormalize(int64_t n, int32_t K, int32_t dtype, void* V, int64_t ldv,
                                         double* R_out, int32_t* rank_out, void* workspace,
                                         size_t workspace_bytes, void* stream) {
  HEF_NVTX("hef_orthonormalize (Algorithm 1 step 4)");
  if (n < 1 || K < 1) return set_error(HEF_ERR_INVALID_ARG, "hef_orthonormalize: need n, K >= 1");
  if (K > 512) return set_error(HEF_ERR_UNSUPPORTED, "hef_orthonormalize: K must be <= 512");
  if (n >= (1ll << 31) - 1)
    return set_error(HEF_ERR_UNSUPPORTED, "hef_orthonormalize: n must be < 2^31 - 1");
  if (dtype != HEF_F64 && dtype != HEF_F32 && dtype != HEF_BF16)
    return set_error(HEF_ERR_INVALID_ARG,
                     "hef_orthonormalize: dtype must be HEF_F64, HEF_F32 or HEF_BF16");
  if (dtype == HEF_BF16 && !(gram_tc_supported(K) && apply_tc_supported(K)))
    return set_error(HEF_ERR_UNSUPPORTED, "hef_orthonormalize: the BF16 basis needs K <= 511");
  const size_t esz = dtype == HEF_F64 ? 8 : (dtype == HEF_BF16 ? 2 : 4);
  if (!V || ldv < K || (ldv * esz) % 16 || (reinterpret_cast<uintptr_t>(V) & 15))
    return set_error(HEF_ERR_INVALID_ARG,
                     "hef_orthonormalize: V NULL, ldv < K or rows not 16-byte aligned");
  OrthoWs w;
  const size_t need = carve_ortho(workspace, n, K, dtype, &w);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return set_error(HEF_ERR_WORKSPACE,
                     "hef_orthonormalize: workspace needs %zu bytes (256-aligned)", need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == HEF_F64)
    return run_ortho<double>(n, K, static_cast<double*>(V), ldv, R_out, rank_out, w, st);
  return run_ortho<float>(n, K, static_cast<float*>(V), ldv, R_out, rank_out, w, st,
                          dtype == HEF_BF16);
}
