// Orthonormalisation: Algorithm 1 step 4 ("Gram-Schmidt"), done as CholQR2
// on the mean-free basis: G = V^T V - c c^T / n (c = V^T 1), R1 = chol(G)
// in FP64, Q1 = (V - 1 mu^T) R1^-1; the same again on Q1 (which removes the
// rounding left by the first pass); Q = Q1 R2^-1, R = R2 R1.  Q spans the
// same nested column spaces as Gram-Schmidt in column order would, with a
// positive diagonal, so it equals the Gram-Schmidt Q up to rounding.
//
// Kernels: k_gram (tiled, split over rows, per-chunk partials), k_gram_reduce
// (fixed-order sum), k_chol (one CTA, FP64: pivoted-out rank-deficient
// columns, triangular inverse), k_apply (in place, row blocks in shared
// memory, column blocks last to first so each column is overwritten only
// after every later column has used it).
#include "internal.h"

namespace hef {

namespace {

constexpr int kTileG = 32;  // Gram output tile
constexpr int kPanel = 32;  // rows per Gram panel

template <typename T>
struct Acc;  // per-panel accumulator type of the Gram kernel
template <>
struct Acc<double> {
  using type = double;
  static constexpr int flush = 1;  // panels between flushes to the FP64 sum
};
template <>
struct Acc<float> {
  using type = float;
  static constexpr int flush = 8;
};

// Partial Gram tile (bi, bj) over one chunk of rows, plus column sums when
// bi == bj.  Thread (ty, tx) of a 16 x 16 layout owns a 2 x 2 output block.
template <typename T>
__global__ void __launch_bounds__(256) k_gram(const T* __restrict__ V, long long ldv, int n, int K,
                                              int nb, int rows_per_chunk, double* part,
                                              double* colpart) {
  using A = typename Acc<T>::type;
  __shared__ T As[kPanel][kTileG + 1];
  __shared__ T Bs[kPanel][kTileG + 1];
  // tile pair index -> (bi, bj), bi <= bj
  int t = blockIdx.x, bi = 0;
  while (t >= nb - bi) {
    t -= nb - bi;
    ++bi;
  }
  const int bj = bi + t;
  const int chunk = blockIdx.y;
  const long long r0 = (long long)chunk * rows_per_chunk;
  const long long r1 = min((long long)n, r0 + rows_per_chunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int ci = bi * kTileG, cj = bj * kTileG;
  double acc[2][2] = {{0, 0}, {0, 0}};
  double csum = 0.0;
  A pacc[2][2] = {{0, 0}, {0, 0}};
  A pcs = 0;
  int npanel = 0;
  for (long long r = r0; r < r1; r += kPanel) {
    for (int e = threadIdx.x; e < kPanel * kTileG; e += blockDim.x) {
      const int rr = e / kTileG, cc = e % kTileG;
      const long long row = r + rr;
      const bool ok = row < r1;
      As[rr][cc] = (ok && ci + cc < K) ? V[row * ldv + ci + cc] : (T)0;
      Bs[rr][cc] = (ok && cj + cc < K) ? V[row * ldv + cj + cc] : (T)0;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < kPanel; ++rr) {
      const A a0 = As[rr][ty * 2], a1 = As[rr][ty * 2 + 1];
      const A b0 = Bs[rr][tx * 2], b1 = Bs[rr][tx * 2 + 1];
      pacc[0][0] += a0 * b0;
      pacc[0][1] += a0 * b1;
      pacc[1][0] += a1 * b0;
      pacc[1][1] += a1 * b1;
    }
    if (bi == bj && threadIdx.x < kTileG) {
      for (int rr = 0; rr < kPanel; ++rr) pcs += As[rr][threadIdx.x];
    }
    __syncthreads();
    if (++npanel == Acc<T>::flush) {
      npanel = 0;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          acc[a][b] += (double)pacc[a][b];
          pacc[a][b] = 0;
        }
      csum += (double)pcs;
      pcs = 0;
    }
  }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) acc[a][b] += (double)pacc[a][b];
  csum += (double)pcs;
  double* P = part + (size_t)chunk * K * K;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const int i = ci + ty * 2 + a, j = cj + tx * 2 + b;
      if (i < K && j < K) P[(size_t)i * K + j] = acc[a][b];
    }
  if (bi == bj && threadIdx.x < kTileG && ci + threadIdx.x < K)
    colpart[(size_t)chunk * K + ci + threadIdx.x] = csum;
}

// G[i][j] (i <= j, mirrored) and c[i]: fixed-order sums over chunks.
__global__ void k_gram_reduce(const double* part, const double* colpart, int K, int nchunk,
                              double* G, double* c) {
  const long long KK = (long long)K * K;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < KK + K;
       idx += (long long)gridDim.x * blockDim.x) {
    if (idx < KK) {
      const int i = (int)(idx / K), j = (int)(idx % K);
      if (i > j) continue;
      double s = 0.0;
      for (int q = 0; q < nchunk; ++q) s += part[(size_t)q * KK + idx];
      G[(size_t)i * K + j] = s;
      G[(size_t)j * K + i] = s;
    } else {
      const int i = (int)(idx - KK);
      double s = 0.0;
      for (int q = 0; q < nchunk; ++q) s += colpart[(size_t)q * K + i];
      c[i] = s;
    }
  }
}

// One CTA: A = G - c c^T / n (upper triangle), right-looking Cholesky with
// rank-deficient columns dropped (pivot <= tol * G_ii, the column's squared
// norm before projection; tol 1e-12 in FP64, 1e-5 in FP32: a Cholesky pivot
// only resolves relative residuals above about sqrt(eps)), then
// R^-1 by back substitution (one warp per column).  A lives in shared memory
// when it fits, else in the global scratch `Ag`.
template <typename T>
__global__ void __launch_bounds__(1024) k_chol(const double* __restrict__ G,
                                               const double* __restrict__ c, int K, double n,
                                               double tol, double* Ag, double* R, double* Rinv,
                                               T* RinvT, T* muT, int* kept, int* rank,
                                               int use_smem) {
  extern __shared__ double dsm[];
  __shared__ double rrow[512];
  __shared__ double diag0[512];
  __shared__ double piv;
  __shared__ int keep_j;
  double* A = use_smem ? dsm : Ag;
  const long long KK = (long long)K * K;
  for (long long idx = threadIdx.x; idx < KK; idx += blockDim.x) {
    const int i = (int)(idx / K), j = (int)(idx % K);
    A[idx] = G[idx] - c[i] * c[j] / n;
    R[idx] = 0.0;
    Rinv[idx] = 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    // reference for rank detection: the squared norm before any projection
    // (the projected pivot carries rounding of order eps * this)
    diag0[i] = G[(size_t)i * K + i];
    muT[i] = (T)(c[i] / n);
  }
  __syncthreads();
  for (int j = 0; j < K; ++j) {
    if (threadIdx.x == 0) {
      const double d = A[(size_t)j * K + j];
      keep_j = (diag0[j] > 0.0 && d > tol * diag0[j]) ? 1 : 0;
      piv = keep_j ? sqrt(d) : 0.0;
      kept[j] = keep_j;
    }
    __syncthreads();
    const int kj = keep_j;
    const double pv = piv;
    __syncthreads();  // all have read before thread 0 writes the next pivot
    if (!kj) continue;  // uniform across the CTA
    for (int i = j + threadIdx.x; i < K; i += blockDim.x) {
      const double r = (i == j) ? pv : A[(size_t)j * K + i] / pv;
      rrow[i] = r;
      R[(size_t)j * K + i] = r;
    }
    __syncthreads();
    const int w = K - j - 1;
    for (long long idx = threadIdx.x; idx < (long long)w * w; idx += blockDim.x) {
      const int i = j + 1 + (int)(idx / w), l = j + 1 + (int)(idx % w);
      if (l >= i) A[(size_t)i * K + l] -= rrow[i] * rrow[l];
    }
    __syncthreads();
  }
  // R^-1: column j solves R x = e_j over the kept indices (back substitution).
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wid; j < K; j += nw) {
    if (!kept[j]) continue;
    const double xj = 1.0 / R[(size_t)j * K + j];
    if (lane == 0) Rinv[(size_t)j * K + j] = xj;
    __syncwarp();
    for (int i = j - 1; i >= 0; --i) {
      if (!kept[i]) continue;
      double s = 0.0;
      for (int l = i + 1 + lane; l <= j; l += 32) s += R[(size_t)i * K + l] * Rinv[(size_t)l * K + j];
      s = warp_sum(s);
      if (lane == 0) Rinv[(size_t)i * K + j] = -s / R[(size_t)i * K + i];
      __syncwarp();
    }
  }
  __syncthreads();
  for (long long idx = threadIdx.x; idx < KK; idx += blockDim.x) RinvT[idx] = (T)Rinv[idx];
  if (threadIdx.x == 0) {
    int r = 0;
    for (int j = 0; j < K; ++j) r += kept[j];
    *rank = r;
  }
}

// Q = (V - 1 mu^T) Rinv in place.  One CTA per RB-row block.
template <typename T>
__global__ void __launch_bounds__(256) k_apply(T* V, long long ldv, int n, int K,
                                               const T* __restrict__ Rinv, const T* __restrict__ mu,
                                               int RB, int CB) {
  extern __shared__ unsigned char sm_raw[];
  T* Vs = reinterpret_cast<T*>(sm_raw);        // RB x K
  T* Rs = Vs + (size_t)RB * K;                  // K x CB
  const long long r0 = (long long)blockIdx.x * RB;
  const int nrow = (int)min((long long)RB, (long long)n - r0);
  for (int e = threadIdx.x; e < RB * K; e += blockDim.x) {
    const int rr = e / K, cc = e % K;
    Vs[e] = rr < nrow ? V[(r0 + rr) * ldv + cc] - mu[cc] : (T)0;
  }
  const int tx = threadIdx.x % CB, ty = threadIdx.x / CB, nty = blockDim.x / CB;
  const int nblk = (K + CB - 1) / CB;
  for (int J = nblk - 1; J >= 0; --J) {
    const int c0 = J * CB;
    const int iend = min(K, c0 + CB);  // Rinv upper triangular: rows < iend
    __syncthreads();
    for (int e = threadIdx.x; e < iend * CB; e += blockDim.x) {
      const int i = e / CB, jj = e % CB;
      Rs[e] = (c0 + jj < K) ? Rinv[(size_t)i * K + c0 + jj] : (T)0;
    }
    __syncthreads();
    T acc[16];
    const int nr = (RB + nty - 1) / nty;
    for (int q = 0; q < nr; ++q) acc[q] = 0;
    for (int i = 0; i < iend; ++i) {
      const T rv = Rs[i * CB + tx];
      for (int q = 0; q < nr; ++q) {
        const int rr = ty + q * nty;
        if (rr < RB) acc[q] += Vs[rr * K + i] * rv;
      }
    }
    __syncthreads();
    if (c0 + tx < K)
      for (int q = 0; q < nr; ++q) {
        const int rr = ty + q * nty;
        if (rr < RB) Vs[rr * K + c0 + tx] = acc[q];
      }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nrow * K; e += blockDim.x) {
    const int rr = e / K, cc = e % K;
    V[(r0 + rr) * ldv + cc] = Vs[e];
  }
}

// R_out = R2 * R1 (both upper triangular).
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
  double* Ag;
  double* R1;
  double* R2;
  double* Rinv;
  void* RinvT;
  void* muT;
  int* kept;
  int* rank;
  int nchunk;
  int rows_per_chunk;
};

inline int ntiles_of(int K) {
  const int nb = (K + kTileG - 1) / kTileG;
  return nb * (nb + 1) / 2;
}

size_t carve_ortho(void* base, long long n, int K, int dtype, OrthoWs* w) {
  Carver c(base);
  const int tiles = ntiles_of(K);
  int nchunk = (num_sms() * 4 + tiles - 1) / tiles;
  const long long max_chunks = (n + 63) / 64;
  if (nchunk > max_chunks) nchunk = (int)(max_chunks > 0 ? max_chunks : 1);
  w->nchunk = nchunk;
  w->rows_per_chunk = (int)(((n + nchunk - 1) / nchunk + kPanel - 1) / kPanel * kPanel);
  const size_t KK = (size_t)K * K;
  const size_t esz = dtype == HEF_F64 ? 8 : 4;
  w->part = c.take<double>(KK * nchunk);
  w->colpart = c.take<double>((size_t)K * nchunk);
  w->G = c.take<double>(KK);
  w->c = c.take<double>(K);
  w->Ag = c.take<double>(KK);
  w->R1 = c.take<double>(KK);
  w->R2 = c.take<double>(KK);
  w->Rinv = c.take<double>(KK);
  w->RinvT = c.take<char>(KK * esz);
  w->muT = c.take<char>(K * esz);
  w->kept = c.take<int>(K);
  w->rank = c.take<int>(4);
  return c.bytes();
}

template <typename T>
hef_status run_ortho(long long n, int K, T* V, long long ldv, double* R_out, int* rank_out,
                     const OrthoWs& w, cudaStream_t st) {
  const int nb = (K + kTileG - 1) / kTileG;
  const int tiles = ntiles_of(K);
  const size_t chol_smem = (size_t)K * K * sizeof(double);
  const int use_smem = chol_smem <= 200 * 1024 ? 1 : 0;
  if (use_smem) {
    HEF_CHECK_CUDA(cudaFuncSetAttribute(k_chol<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)chol_smem));
  }
  // apply tiling: largest (RB, CB) whose shared memory fits in 200 KB
  int RB = 64, CB = 32;
  auto smem_of = [&](int rb, int cb) { return ((size_t)rb * K + (size_t)K * cb) * sizeof(T); };
  while (smem_of(RB, CB) > 200 * 1024 && RB > 16) RB /= 2;
  while (smem_of(RB, CB) > 200 * 1024 && CB > 8) CB /= 2;
  if (smem_of(RB, CB) > 200 * 1024 || (RB + (256 / CB) - 1) / (256 / CB) > 16)
    return set_error(HEF_ERR_UNSUPPORTED, "hef_orthonormalize: K = %d too large", K);
  const size_t apply_smem = smem_of(RB, CB);
  HEF_CHECK_CUDA(cudaFuncSetAttribute(k_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)apply_smem));
  const double tol = sizeof(T) == 8 ? 1e-12 : 1e-5;
  const dim3 ggrid(tiles, w.nchunk);
  const int rgrid = stride_grid((long long)K * K + K, 4);
  const int agrid = (int)((n + RB - 1) / RB);
  double* Rs[2] = {w.R1, w.R2};
  for (int pass = 0; pass < 2; ++pass) {
    HEF_LAUNCH("k_gram", st, k_gram<T><<<ggrid, 256, 0, st>>>(V, ldv, (int)n, K, nb, w.rows_per_chunk, w.part, w.colpart));
    HEF_LAUNCH("k_gram_reduce", st, k_gram_reduce<<<rgrid, kThreads, 0, st>>>(w.part, w.colpart, K, w.nchunk, w.G, w.c));
    HEF_LAUNCH("k_chol", st, k_chol<T><<<1, 1024, use_smem ? chol_smem : 0, st>>>(
        w.G, w.c, K, (double)n, tol, w.Ag, Rs[pass], w.Rinv, static_cast<T*>(w.RinvT),
        static_cast<T*>(w.muT), w.kept, w.rank, use_smem));
    HEF_LAUNCH("k_apply", st, k_apply<T><<<agrid, 256, apply_smem, st>>>(V, ldv, (int)n, K, static_cast<const T*>(w.RinvT),
                                               static_cast<const T*>(w.muT), RB, CB));
    HEF_CHECK_LAUNCH();
  }
  if (R_out) {
    HEF_LAUNCH("k_trmm_upper", st, k_trmm_upper<<<rgrid, kThreads, 0, st>>>(w.R2, w.R1, K, R_out));
    HEF_CHECK_LAUNCH();
  }
  if (rank_out) HEF_CHECK_CUDA(cudaMemcpyAsync(rank_out, w.rank, sizeof(int), cudaMemcpyDeviceToDevice, st));
  return HEF_OK;
}

}  // namespace

}  // namespace hef

using namespace hef;

extern "C" size_t hef_orthonormalize_workspace_bytes(int64_t n, int32_t K, int32_t dtype) {
  if (n < 1 || K < 1 || K > 512 || (dtype != HEF_F64 && dtype != HEF_F32)) return 0;
  OrthoWs w;
  return carve_ortho(nullptr, n, K, dtype, &w);
}

extern "C" hef_status hef_orthonormalize(int64_t n, int32_t K, int32_t dtype, void* V, int64_t ldv,
                                         double* R_out, int32_t* rank_out, void* workspace,
                                         size_t workspace_bytes, void* stream) {
  if (n < 1 || K < 1) return set_error(HEF_ERR_INVALID_ARG, "hef_orthonormalize: need n, K >= 1");
  if (K > 512) return set_error(HEF_ERR_UNSUPPORTED, "hef_orthonormalize: K must be <= 512");
  if (n >= (1ll << 31) - 1)
    return set_error(HEF_ERR_UNSUPPORTED, "hef_orthonormalize: n must be < 2^31 - 1");
  if (dtype != HEF_F64 && dtype != HEF_F32)
    return set_error(HEF_ERR_INVALID_ARG, "hef_orthonormalize: dtype must be HEF_F64 or HEF_F32");
  const size_t esz = dtype == HEF_F64 ? 8 : 4;
  if (!V || ldv < K || (ldv * esz) % 16 || (reinterpret_cast<uintptr_t>(V) & 15))
    return set_error(HEF_ERR_INVALID_ARG, "hef_orthonormalize: V NULL, ldv < K or rows not 16-byte aligned");
  OrthoWs w;
  const size_t need = carve_ortho(workspace, n, K, dtype, &w);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return set_error(HEF_ERR_WORKSPACE, "hef_orthonormalize: workspace needs %zu bytes (256-aligned)", need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == HEF_F64)
    return run_ortho<double>(n, K, static_cast<double*>(V), ldv, R_out, rank_out, w, st);
  return run_ortho<float>(n, K, static_cast<float*>(V), ldv, R_out, rank_out, w, st);
}
