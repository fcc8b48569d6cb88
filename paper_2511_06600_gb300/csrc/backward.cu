// Adjoint of the hyperedge effective-resistance path (Algorithm 1 steps 3-7):
// from dL/dR, the gradients dL/dw (hyperedge weights) and dL/dx0 (random
// starts).  The paper defines only the forward; this is its exact derivative
// with the forward's routing (argmax column i*, arg-max/arg-min pins) held.
//
// Scoring (Eqs. non-linerQ, ratios, R): R_e = sp_{e,i*}^2 / Q_H[i*] and
// Q_H[i] = sum_e w_e sp_{e,i}^2, sp the spread between the pins attaining the
// max and the min of column i on e (lowest position on ties, as the forward).
//   Qbar_H[i]   = -sum_{e: i*_e = i} g_e R_e / Q_H[i]
//   spbar_{e,i} = [i = i*_e] 2 g_e sp / Q_H[i] + 2 Qbar_H[i] w_e sp
//   Qbar[p, i] += spbar, Qbar[q, i] -= spbar,  wbar_e += sum_i Qbar_H[i] sp^2
// (the spread adjoints are stored per hyperedge and column with the positions
// of p and q in e, and each vertex then sums its own entries)
// Orthonormalisation (Algorithm 1 step 4): Q R = P V with P = I - 11^T/n and
// R not used downstream, so Abar = (Qbar + Q C) R^-T with
// C = copyltu(-Qbar^T Q) (the lower triangle mirrored), and Vbar = P Abar.
// Dropped columns (R_jj = 0) take no part: R^-1 is the inverse of the kept
// block.
// Krylov chains (Algorithm 1 step 3, Eq. krylov): the forward recurrence is
// x_j = nu_j (M x_{j-1} - alpha_j x_{j-1} - beta_j x_{j-2}), x_0 = nu_0 Pi x0.
// For any values of alpha, beta and nu (> 0) the chain spans the same nested
// Krylov spaces, so V changes only by an upper-triangular factor with a
// positive diagonal, which Q does not see: those coefficients are held fixed.
// The per-step deflation of the trivial eigenvectors is identically zero as a
// function of (w, x0) (Pi commutes with M), so it has no adjoint.  What
// remains is the transposed recurrence with M^T = W D^-1, the derivative of
// M with respect to w (through wh_e, z_e and the degrees), and at j = 0 the
// derivative of the degree-weighted deflation Pi of the start.
//
// Q_H's adjoint is summed with FP64 atomics (gradients agree across runs to
// rounding, not bit for bit); Qbar is gathered per vertex in a fixed order.
// The scoring adjoint is FP64; the QR and Krylov-chain adjoints run in the
// storage type of the form (FP32 for the FP32 form: FP64 runs at 1/64 of the
// rate on this GPU), with Gram-type and weight-gradient sums in FP64.

#include <algorithm>

#include "internal.h"

namespace hef {

namespace {

constexpr double kTiny = 1e-300;

template <typename T>
__device__ __forceinline__ T lowest_v();
template <>
__device__ __forceinline__ double lowest_v<double>() {
  return -1.7976931348623157e308;
}
template <>
__device__ __forceinline__ float lowest_v<float>() {
  return -3.402823466e38f;
}

// ---------------------------------------------------------------- scoring adjoint

// Qbar_H[i] = -sum over edges routed to column i of g_e R_e / Q_H[i].
__global__ void k_bwd_qhbar(IncView g, const double* __restrict__ dR, const double* __restrict__ R,
                            const int32_t* __restrict__ argvec, const double* __restrict__ QH,
                            double* QHbar) {
  if (g.status[0]) return;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < g.m;
       e += (long long)gridDim.x * blockDim.x) {
    const int oe = g.perm[e];
    const int i = argvec[oe];
    if (i >= 0 && QH[i] > kTiny && dR[oe] != 0.0) atomicAdd(&QHbar[i], -dR[oe] * R[oe] / QH[i]);
  }
}

// Warp per hyperedge, lane l owns columns l, l + 32, ... (NC per lane): the
// extrema of every column, then the spread adjoints scattered into Qbar and
// the direct weight term.
template <typename T, int NC>
__global__ void __launch_bounds__(256) k_bwd_scores(IncView g, const T* __restrict__ Q, long long ldq,
                                                    int K, const double* __restrict__ dR,
                                                    const int32_t* __restrict__ argvec,
                                                    const double* __restrict__ QH,
                                                    const double* __restrict__ QHbar, double* spbar,
                                                    int32_t* omax, int32_t* omin, double* wbar) {
  if (g.status[0]) return;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  double iq[NC], qhb[NC];  // 1 / Q_H (0 for skipped columns) and Qbar_H of the lane's columns
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int col = lane + 32 * c;
    iq[c] = (col < K && QH[col] > kTiny) ? 1.0 / QH[col] : 0.0;
    qhb[c] = col < K ? QHbar[col] : 0.0;
  }
  for (long long e = warp; e < g.m; e += nwarps) {
    const int a = g.ceptr[e], b = g.ceptr[e + 1];
    if (b - a < 2) continue;
    T mx[NC], mn[NC];
    int imx[NC], imn[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) mx[c] = lowest_v<T>(), mn[c] = -lowest_v<T>(), imx[c] = a, imn[c] = a;
    for (int t = a; t < b; ++t) {
      const T* row = Q + (long long)dbg_index(g.cpins[t], g.n, g.status) * ldq;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int col = lane + 32 * c;
        if (col < K) {
          const T v = row[col];
          if (v > mx[c]) mx[c] = v, imx[c] = t;
          if (v < mn[c]) mn[c] = v, imn[c] = t;
        }
      }
    }
    const int oe = g.perm[e];
    const double ge = dR[oe];
    const int istar = argvec[oe];
    const double we = g.ew[e];
    double wsum = 0.0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int col = lane + 32 * c;
      if (iq[c] != 0.0) {
        const double sp = (double)mx[c] - (double)mn[c];
        double sb = 2.0 * qhb[c] * we * sp;
        if (col == istar) sb += 2.0 * ge * sp * iq[c];
        wsum += qhb[c] * sp * sp;
        // the spread adjoint and where in e its two pins sit; the vertex
        // pass k_bwd_qbar adds them up per vertex (no atomics, fixed order)
        spbar[e * K + col] = sb;
        omax[e * K + col] = imx[c] - a;
        omin[e * K + col] = imn[c] - a;
      } else if (col < K) {
        spbar[e * K + col] = 0.0;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    if (lane == 0) wbar[e] += wsum;
  }
}

// Qbar[v][i] = sum over the hyperedges e of v of +spbar[e][i] where v is the
// pin attaining the max of column i on e, -spbar[e][i] where it attains the
// min (warp per vertex, lanes over columns; the vertex-major incidence gives
// v's position in each hyperedge).
template <typename T>
__global__ void __launch_bounds__(256) k_bwd_qbar(IncView g, int K, const double* __restrict__ spbar,
                                                  const int32_t* __restrict__ omax,
                                                  const int32_t* __restrict__ omin, T* Qbar) {
  if (g.status[0]) return;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long v = warp; v < g.n; v += nwarps) {
    const int t0 = g.vptr[v], t1 = g.vptr[v + 1];
    for (int c0 = 0; c0 < K; c0 += 32) {
      const int col = c0 + lane;
      double acc = 0.0;
      for (int t = t0; t < t1; ++t) {
        const int e = dbg_index(g.vedge[t], g.m, g.status);
        const int a = g.ceptr[e];
        if (g.ceptr[e + 1] - a < 2 || col >= K) continue;
        const int pos = g.vslot[t] - a;
        const long long q = (long long)e * K + col;
        const double sb = spbar[q];
        if (omax[q] == pos) acc += sb;
        if (omin[q] == pos) acc -= sb;
      }
      if (col < K) Qbar[v * K + col] = (T)acc;
    }
  }
}

// ---------------------------------------------------------------- QR adjoint

// part[chunk][i][j] = sum over the chunk's rows r of Qbar[r][i] * Q[r][j],
// in the storage type within a chunk (FP32 products and sums for the FP32
// form: FP64 runs at 1/64 of the rate) and FP64 across chunks.
template <typename T>
__global__ void k_bwd_xgram(const T* __restrict__ Qbar, const T* __restrict__ Q, long long ldq,
                            long long n, int K, long long rows_per_chunk, double* part) {
  const int chunk = blockIdx.y;
  const long long r0 = (long long)chunk * rows_per_chunk;
  const long long r1 = min(n, r0 + rows_per_chunk);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < K * K; idx += gridDim.x * blockDim.x) {
    const int i = idx / K, j = idx % K;
    T s = 0;
    for (long long r = r0; r < r1; ++r) s += Qbar[r * K + i] * Q[r * ldq + j];
    part[(size_t)chunk * K * K + idx] = (double)s;
  }
}

// C = copyltu(-Qbar^T Q): C[i][j] = -(Qbar^T Q)[max(i,j)][min(i,j)] (summed
// in FP64, stored in the storage type).
template <typename T>
__global__ void k_bwd_copyltu(const double* __restrict__ part, int K, int nchunk, T* C) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < K * K; idx += gridDim.x * blockDim.x) {
    const int i = idx / K, j = idx % K;
    const int hi = i > j ? i : j, lo = i > j ? j : i;
    double s = 0.0;
    for (int q = 0; q < nchunk; ++q) s += part[(size_t)q * K * K + hi * K + lo];
    C[idx] = (T)-s;
  }
}

// Rinv = inverse of the kept block of the upper-triangular R (row-major
// K x K); rows and columns of dropped columns (R_jj = 0) stay zero.  One
// warp per column, back substitution.
template <typename T>
__global__ void k_bwd_rinv(const double* __restrict__ R, int K, double* Rinv, T* RinvT) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) Rinv[idx] = 0.0;
  __syncthreads();
  for (int j = wid; j < K; j += nw) {
    if (R[(size_t)j * K + j] == 0.0) continue;
    if (lane == 0) Rinv[(size_t)j * K + j] = 1.0 / R[(size_t)j * K + j];
    __syncwarp();
    for (int i = j - 1; i >= 0; --i) {
      if (R[(size_t)i * K + i] == 0.0) continue;
      double s = 0.0;
      for (int l = i + 1 + lane; l <= j; l += 32) s += R[(size_t)i * K + l] * Rinv[(size_t)l * K + j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) Rinv[(size_t)i * K + j] = -s / R[(size_t)i * K + i];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) RinvT[idx] = (T)Rinv[idx];
}

// Z = Qbar + Q C (thread per element, storage type).
template <typename T>
__global__ void k_bwd_qr_z(const T* __restrict__ Q, long long ldq, const T* __restrict__ Qbar,
                           const T* __restrict__ C, long long n, int K, T* Z) {
  const long long total = n * K;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long r = idx / K;
    const int j = (int)(idx % K);
    const T* q = Q + r * ldq;
    T s = Qbar[idx];
    for (int i = 0; i < K; ++i) s += q[i] * C[(size_t)i * K + j];
    Z[idx] = s;
  }
}

// Abar = Z R^-T, i.e. Abar[r][j] = sum_{i >= j} Z[r][i] Rinv[j][i] (Rinv is
// upper triangular); storage type.
template <typename T>
__global__ void k_bwd_qr_abar(const T* __restrict__ Z, const T* __restrict__ Rinv, long long n,
                              int K, T* Abar) {
  const long long total = n * K;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long r = idx / K;
    const int j = (int)(idx % K);
    const T* z = Z + r * K;
    const T* ri = Rinv + (size_t)j * K;
    T s = 0;
    for (int i = j; i < K; ++i) s += z[i] * ri[i];
    Abar[idx] = s;
  }
}

// colsum[j] = sum_r A[r][j] (A n x K): CTA-strided rows summed in the
// storage type, one FP64 atomic per CTA and column.
template <typename T>
__global__ void k_bwd_colsum(const T* __restrict__ A, long long n, int K, double* colsum) {
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    T s = 0;
    for (long long r = blockIdx.x; r < n; r += gridDim.x) s += A[r * K + j];
    atomicAdd(&colsum[j], (double)s);
  }
}

// mean[j] = colsum[j] / n in the storage type.
template <typename T>
__global__ void k_bwd_mean(const double* __restrict__ colsum, long long n, int K, T* mean) {
  for (int j = threadIdx.x; j < K; j += blockDim.x) mean[j] = (T)(colsum[j] / (double)n);
}

// ---------------------------------------------------------------- chain adjoint
//
// The chain adjoints run in the storage type T of the form (FP32 buffers and
// arithmetic for the FP32 form: FP64 runs at 1/64 of the rate on this GPU),
// with the forward's scalars from the same-typed copies of the incidence;
// weight gradients accumulate in FP64.

template <typename T>
struct ChainBwd {
  int n, m, S, k, K, j;
  const double* coef;    // forward coefficients, (k+1) x 2S x 4
  const double* inv_nu;  // forward inverse norms, (k+1) x 2S
  const T* uc;           // forward u_j, clique chains: (k+1) x n x S
  const T* ub;           // forward u_j, star chains: (k+1) x (n+m) x S
  T* xbc0;               // adjoints of x_j (clique, n x S), slot j mod 3
  T* xbc1;
  T* xbc2;
  T* xbb0;               // adjoints of x_j (star, (n+m) x S), slot j mod 3
  T* xbb1;
  T* xbb2;
  T* zc;                 // D^-1 ubar_j, clique rows
  T* zb;                 // D^-1 ubar_j, star rows
  T* sc;                 // m x S: sum over e's pins of x_{j-1} (clique)
  T* zs;                 // m x S: sum over e's pins of zc
  T* yc;                 // n x S: (M x_{j-1}) clique
  T* yb;                 // n x S: (M x_{j-1}) star vertex rows
  const T* Abar;         // n x K adjoint of the mean-free basis
  const T* mean;         // its column means
  double* wbar;          // m, internal order
  ScalView<T> sv;        // expansion scalars in T
};

// Slot q (0..2) of the rotating adjoint buffers without indexing an array in
// the kernel argument at run time.
template <typename T>
__device__ __forceinline__ T* slot_c(const ChainBwd<T>& c, int q) {
  return q == 0 ? c.xbc0 : (q == 1 ? c.xbc1 : c.xbc2);
}
template <typename T>
__device__ __forceinline__ T* slot_b(const ChainBwd<T>& c, int q) {
  return q == 0 ? c.xbb0 : (q == 1 ? c.xbb1 : c.xbb2);
}

// (A) thread per (row, start): the archive adjoint of x_j (vertex rows, with
// the mean removal P), ubar_j = nu_j xbar_j, z = D^-1 ubar_j, and the fixed
// coefficients' terms xbar_{j-1} -= alpha_j ubar_j, xbar_{j-2} -= beta_j ubar_j.
// Rows: [0, n) clique, [n, 2n + m) star.
template <typename T>
__global__ void k_bwd_prep(IncView g, ChainBwd<T> c) {
  if (g.status[0]) return;
  const int S = c.S, j = c.j;
  const long long nrows = 2ll * c.n + c.m;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nrows * S;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long r = idx / S;
    const int s = (int)(idx % S);
    const bool clique = r < c.n;
    const long long rr = clique ? r : r - c.n;
    const int ch = (clique ? 0 : 1) * S + s;
    T* xj = clique ? slot_c(c, j % 3) : slot_b(c, j % 3);
    T* xj1 = clique ? slot_c(c, (j + 2) % 3) : slot_b(c, (j + 2) % 3);
    T* xj2 = clique ? slot_c(c, (j + 1) % 3) : slot_b(c, (j + 1) % 3);
    T xb = xj[rr * S + s];
    if (rr < c.n) {
      const int col = (j - 1) * 2 * S + ch;
      xb += c.Abar[rr * c.K + col] - c.mean[col];
    }
    const T ub = (T)c.inv_nu[(size_t)j * 2 * S + ch] * xb;
    T invd;
    if (clique) invd = c.sv.inv_dc[rr];
    else if (rr < c.n) invd = c.sv.inv_db[rr];
    else invd = c.sv.ew[rr - c.n] > (T)0 ? (T)1 / c.sv.ew[rr - c.n] : (T)0;
    (clique ? c.zc : c.zb)[rr * S + s] = ub * invd;
    const double* cf = c.coef + ((size_t)j * 2 * S + ch) * 4;
    if (j >= 2) xj1[rr * S + s] -= (T)cf[2] * ub;
    if (j >= 3) xj2[rr * S + s] -= (T)cf[3] * ub;
  }
}

// (B) thread per (hyperedge, start): sc = sum_{p in e} x_{j-1}[p] (clique),
// zs = sum_{p in e} zc[p], and the star hyperedge rows' transposed product
// xbar_{j-1}[n+e] += z_e sum_{p in e} zb[p].
template <typename T>
__global__ void k_bwd_edge1(IncView g, ChainBwd<T> c) {
  if (g.status[0]) return;
  const int S = c.S, j = c.j;
  const T* uc = c.uc + (long long)(j - 1) * c.n * S;
  T* xbb1 = slot_b(c, (j + 2) % 3);
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)c.m * S;
       idx += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(idx / S), s = (int)(idx % S);
    const int a = g.ceptr[e], b = g.ceptr[e + 1];
    const T nu = (T)c.inv_nu[(size_t)(j - 1) * 2 * S + s];
    T sx = 0, sz = 0, szb = 0;
    for (int t = a; t < b; ++t) {
      const long long p = dbg_index(g.cpins[t], g.n, g.status);
      sx += uc[p * S + s];
      sz += c.zc[p * S + s];
      szb += c.zb[p * S + s];
    }
    c.sc[idx] = sx * nu;
    c.zs[idx] = sz;
    xbb1[(long long)(c.n + e) * S + s] += c.sv.ez[e] * szb;
  }
}

// (C) thread per (vertex, start): the forward vertex rows y = M x_{j-1} of
// both chains, and the transposed products into xbar_{j-1}:
// clique sum_{e ∋ v} wh_e (zs_e - zc_v), star sum_{e ∋ v} z_e zb[n+e].
template <typename T>
__global__ void k_bwd_node(IncView g, ChainBwd<T> c) {
  if (g.status[0]) return;
  const int S = c.S, j = c.j;
  const T* uc = c.uc + (long long)(j - 1) * c.n * S;
  const T* ub = c.ub + (long long)(j - 1) * (c.n + c.m) * S;
  T* xbc1 = slot_c(c, (j + 2) % 3);
  T* xbb1 = slot_b(c, (j + 2) % 3);
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)c.n * S;
       idx += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(idx / S), s = (int)(idx % S);
    const T nc = (T)c.inv_nu[(size_t)(j - 1) * 2 * S + s];
    const T nb = (T)c.inv_nu[(size_t)(j - 1) * 2 * S + S + s];
    const T zv = c.zc[idx];
    T fc = 0, fb = 0, tc = 0, tb = 0;
    for (int t = g.vptr[v]; t < g.vptr[v + 1]; ++t) {
      const int e = dbg_index(g.vedge[t], g.m, g.status);
      const T wh = c.sv.ewh[e], z = c.sv.ez[e];
      fc += wh * c.sc[(long long)e * S + s];
      fb += z * ub[(long long)(c.n + e) * S + s];
      tc += wh * (c.zs[(long long)e * S + s] - zv);
      tb += z * c.zb[(long long)(c.n + e) * S + s];
    }
    const T xv = uc[idx] * nc;
    c.yc[idx] = c.sv.inv_dc[v] * (fc - c.sv.wsc[v] * xv);
    c.yb[idx] = c.sv.inv_db[v] * fb * nb;
    xbc1[idx] += tc;
    xbb1[idx] += tb;
  }
}

// (D) thread per hyperedge: derivative of M with respect to w_e at step j,
//   clique: sum_s sum_{v in e} zc_v (a_e (s_e - x_v) - b_e y_v),
//           a_e = d wh_e / d w_e = wh_e / w_e, b_e = d dc(v) / d w_e = a_e (|e| - 1)
//   star:   sum_s (1/|e|) sum_{v in e} zb_v (x_{n+e} - yb_v)
template <typename T>
__global__ void k_bwd_edge2(IncView g, ChainBwd<T> c) {
  if (g.status[0]) return;
  const int S = c.S, j = c.j;
  const T* uc = c.uc + (long long)(j - 1) * c.n * S;
  const T* ub = c.ub + (long long)(j - 1) * (c.n + c.m) * S;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < c.m;
       e += (long long)gridDim.x * blockDim.x) {
    const int a = g.ceptr[e], b = g.ceptr[e + 1];
    const int k = b - a;
    if (k < 2) continue;
    const T ae = c.sv.ewh[e] / c.sv.ew[e], be = ae * (T)(k - 1);
    const T ik = (T)1 / (T)k;
    T acc = 0;
    for (int s = 0; s < S; ++s) {
      const T nc = (T)c.inv_nu[(size_t)(j - 1) * 2 * S + s];
      const T nb = (T)c.inv_nu[(size_t)(j - 1) * 2 * S + S + s];
      const T se = c.sc[e * S + s];
      const T xe = ub[(c.n + e) * S + s] * nb;
      T t1 = 0, t2 = 0, t3 = 0, t4 = 0;
      for (int t = a; t < b; ++t) {
        const long long p = dbg_index(g.cpins[t], g.n, g.status);
        const T zc = c.zc[p * S + s];
        const T zb = c.zb[p * S + s];
        t1 += zc * (se - uc[p * S + s] * nc);
        t2 += zc * c.yc[p * S + s];
        t3 += zb;
        t4 += zb * c.yb[p * S + s];
      }
      acc += ae * t1 - be * t2 + (xe * t3 - t4) * ik;
    }
    c.wbar[e] += (double)acc;
  }
}

// Deflation of the start (j = 0): ubar_0 = nu_0 xbar_0 and its sums over the
// rows of each trivial vector t (clique; star vertices; star hyperedges)
// with d > 0: tdot[slot][s] = t^T ubar_0 (FP64).  Sums per thread, then per
// CTA in shared memory, then one atomic per CTA and slot.
template <typename T>
__global__ void k_bwd_defl_dots(IncView g, ChainBwd<T> c, double* tdot) {
  if (g.status[0]) return;
  __shared__ double sacc[3 * 16];
  const int S = c.S;
  for (int q = threadIdx.x; q < 3 * S; q += blockDim.x) sacc[q] = 0.0;
  __syncthreads();
  const long long nrows = 2ll * c.n + c.m;
  double acc[3][16];
  for (int q = 0; q < 3; ++q)
    for (int s = 0; s < S; ++s) acc[q][s] = 0.0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
       r += (long long)gridDim.x * blockDim.x) {
    double d;
    int slot;
    const T* xa;
    long long arow;
    if (r < c.n) {
      d = g.dc[r], slot = 0, xa = c.xbc0, arow = r;
    } else {
      const long long rb = r - c.n;
      const bool vrow = rb < c.n;
      d = vrow ? g.db[rb] : g.ew[rb - c.n];
      slot = vrow ? 1 : 2, xa = c.xbb0, arow = rb;
    }
    if (d > 0.0)
      for (int s = 0; s < S; ++s)
        acc[slot][s] += c.inv_nu[(slot ? S : 0) + s] * (double)xa[arow * S + s];
  }
  for (int q = 0; q < 3; ++q)
    for (int s = 0; s < S; ++s) {
      double v = acc[q][s];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(&sacc[q * S + s], v);
    }
  __syncthreads();
  for (int q = threadIdx.x; q < 3 * S; q += blockDim.x)
    if (sacc[q] != 0.0) atomicAdd(&tdot[q], sacc[q]);
}

// x0 = Pi x0_raw with Pi x = x - sum_t t c_t(x), c_t = (t^T D x) / (t^T D t):
//   dx0_r = ubar_r - d_r (t^T ubar) / T_t            (rows with d_r > 0)
//   dbar_r = -sum_s (t^T ubar) / T_t (x0_r - c_t)    (T_t = sum of d over t)
// dx0 rows are written in the caller's order (FP64).
template <typename T>
__global__ void k_bwd_defl_out(IncView g, ChainBwd<T> c, const double* __restrict__ tdot,
                               const double* __restrict__ x0c, const double* __restrict__ x0b,
                               double* dx0c, double* dx0b, double* dbar) {
  if (g.status[0]) return;
  const int S = c.S;
  const long long nrows = 2ll * c.n + c.m;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
       r += (long long)gridDim.x * blockDim.x) {
    double d, Tt;
    int slot, ch0;
    long long arow, src;
    const T* xa;
    const double* x0;
    double* out;
    if (r < c.n) {
      d = g.dc[r], Tt = g.totals[0], slot = 0, ch0 = 0;
      xa = c.xbc0, arow = r, x0 = x0c, src = r * S, out = dx0c;
    } else if (r < 2ll * c.n) {
      const long long v = r - c.n;
      d = g.db[v], Tt = g.totals[1], slot = 1, ch0 = S;
      xa = c.xbb0, arow = v, x0 = x0b, src = v * S, out = dx0b;
    } else {
      const long long rb = r - c.n;
      const int i = (int)(rb - c.n);
      d = g.ew[i], Tt = g.totals[2], slot = 2, ch0 = S;
      xa = c.xbb0, arow = rb, x0 = x0b, src = (long long)(c.n + g.perm[i]) * S, out = dx0b;
    }
    double db = 0.0;
    for (int s = 0; s < S; ++s) {
      const double u = c.inv_nu[ch0 + s] * (double)xa[arow * S + s];
      const bool on = d > 0.0 && Tt > 0.0;
      const double td = on ? tdot[slot * S + s] / Tt : 0.0;
      if (out) out[src + s] = u - d * td;
      if (on) {
        const double ct = c.coef[(size_t)(ch0 + s) * 4 + (slot == 2 ? 1 : 0)];
        db -= td * (x0[src + s] - ct);
      }
    }
    dbar[r] = db;
  }
}

// wbar_e += b_e sum_{v in e} dbar_c(v) + (1/|e|) sum_{v in e} dbar_b(v) + dbar_b(n+e),
// the derivatives of dc(v), db(v) and d(n+e) = w_e with respect to w_e.
__global__ void k_bwd_defl_w(IncView g, const double* __restrict__ dbar, double* wbar) {
  if (g.status[0]) return;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < g.m;
       e += (long long)gridDim.x * blockDim.x) {
    const int a = g.ceptr[e], b = g.ceptr[e + 1];
    const int k = b - a;
    if (k < 2) continue;
    const double be = g.ewh[e] / g.ew[e] * (double)(k - 1);
    double sc = 0.0, sb = 0.0;
    for (int t = a; t < b; ++t) {
      const int p = dbg_index(g.cpins[t], g.n, g.status);
      sc += dbar[p];
      sb += dbar[(long long)g.n + p];
    }
    wbar[e] += be * sc + sb / (double)k + dbar[2ll * g.n + e];
  }
}

__global__ void k_bwd_out_w(IncView g, const double* __restrict__ wbar, double* dw) {
  if (g.status[0]) return;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < g.m;
       e += (long long)gridDim.x * blockDim.x)
    dw[g.perm[e]] = wbar[e];
}

// ---------------------------------------------------------------- driver

struct BwdWs {
  double* QHbar;   // K
  double* wbar;    // m
  void* Qbar;      // n x K (storage type)
  double* spbar;   // m x K spread adjoints
  int32_t* omax;   // m x K position in e of the arg-max pin of each column
  int32_t* omin;   // m x K position in e of the arg-min pin
  double* part;    // nchunk x K x K
  void* C;         // K x K (storage type)
  double* Rinv;    // K x K
  void* RinvT;     // K x K (storage type)
  void* Z;         // n x K (storage type)
  void* Abar;      // n x K (storage type)
  double* colsum;  // K
  void* mean;      // K (storage type)
  double* tdot;    // 3 x S
  double* dbar;    // 2n + m
  void* xbc[3];  // chain adjoint buffers in the storage type
  void* xbb[3];
  void* zc;
  void* zb;
  void* sc;
  void* zs;
  void* yc;
  void* yb;
  void* tape;  // recompute mode: the forward tape
  void* kws;   // recompute mode: Krylov workspace
  void* Vtmp;  // recompute mode: basis
  int nchunk;
};

inline int bwd_ldv(int K, size_t esz) { return (int)(((size_t)K * esz + 15) / 16 * 16 / esz); }

size_t carve_bwd(void* base, const hef_incidence* inc, int k, int S, int dtype, bool recompute,
                 BwdWs* w) {
  Carver c(base);
  const long long n = inc->n, m = inc->m;
  const long long m1 = m > 0 ? m : 1;
  const int K = 2 * k * S;
  const size_t esz = dtype == HEF_F64 ? 8 : 4;
  // row chunks of the Qbar^T Q partials: about 256 rows each, at most 1024
  // chunks and 32 M partial values
  long long chunks = (n + 255) / 256;
  const long long cap = std::max(1ll, (1ll << 25) / ((long long)K * K));
  chunks = std::min(chunks, std::min(1024ll, cap));
  w->nchunk = (int)(chunks < 1 ? 1 : chunks);
  w->QHbar = c.take<double>(K);
  w->wbar = c.take<double>(m1);
  w->Qbar = c.take<char>((size_t)n * K * esz);
  w->spbar = c.take<double>((size_t)m1 * K);
  w->omax = c.take<int32_t>((size_t)m1 * K);
  w->omin = c.take<int32_t>((size_t)m1 * K);
  w->part = c.take<double>((size_t)w->nchunk * K * K);
  w->C = c.take<char>((size_t)K * K * esz);
  w->Rinv = c.take<double>((size_t)K * K);
  w->RinvT = c.take<char>((size_t)K * K * esz);
  w->Z = c.take<char>((size_t)n * K * esz);
  w->Abar = c.take<char>((size_t)n * K * esz);
  w->colsum = c.take<double>(K);
  w->mean = c.take<char>((size_t)K * esz);
  w->tdot = c.take<double>(3 * S);
  w->dbar = c.take<double>(2 * n + m);
  for (int q = 0; q < 3; ++q) {
    w->xbc[q] = c.take<char>((size_t)n * S * esz);
    w->xbb[q] = c.take<char>((size_t)(n + m) * S * esz);
  }
  w->zc = c.take<char>((size_t)n * S * esz);
  w->zb = c.take<char>((size_t)(n + m) * S * esz);
  w->sc = c.take<char>((size_t)m1 * S * esz);
  w->zs = c.take<char>((size_t)m1 * S * esz);
  w->yc = c.take<char>((size_t)n * S * esz);
  w->yb = c.take<char>((size_t)n * S * esz);
  w->tape = w->kws = w->Vtmp = nullptr;
  if (recompute) {
    TapeLayout tl;
    w->tape = c.take<char>(carve_tape(nullptr, n, m, k, S, esz, &tl));
    w->kws = c.take<char>(hef_krylov_workspace_bytes(inc, k, S, dtype));
    w->Vtmp = c.take<char>((size_t)n * bwd_ldv(K, esz) * esz);
  }
  return c.bytes();
}

template <typename T, int NC>
void launch_bwd_scores(IncView g, const T* Q, long long ldq, int K, const double* dR,
                       const int32_t* argvec, const double* QH, const BwdWs& w, cudaStream_t st) {
  const long long warps = g.m > 0 ? g.m : 1;
  const int grid = stride_grid(warps * 32, 8);
  HEF_LAUNCH("k_bwd_scores", st,
             k_bwd_scores<T, NC><<<grid, 256, 0, st>>>(g, Q, ldq, K, dR, argvec, QH, w.QHbar, w.spbar,
                                                       w.omax, w.omin, w.wbar));
}

template <typename T>
hef_status run_bwd(const hef_incidence* inc, int k, int S, const double* x0c, const double* x0b,
                   const void* tape_in, const T* Q, long long ldq, const double* Rfac,
                   const double* QH, const int32_t* argvec, const double* R, const double* dR,
                   double* dw, double* dx0c, double* dx0b, const BwdWs& w, cudaStream_t st) {
  IncView g = view(inc);
  const long long n = inc->n, m = inc->m;
  const long long m1 = m > 0 ? m : 1;
  const int K = 2 * k * S;
  // forward tape (recomputed when the caller kept none)
  const void* tape = tape_in;
  if (!tape) {
    const int dt = sizeof(T) == 8 ? HEF_F64 : HEF_F32;
    hef_status s = hef_krylov_basis_tape(inc, k, S, dt, x0c, x0b, w.Vtmp, bwd_ldv(K, sizeof(T)),
                                         w.tape, hef_krylov_tape_bytes(inc, k, S, dt), w.kws,
                                         hef_krylov_workspace_bytes(inc, k, S, dt), st);
    if (s) return s;
    tape = w.tape;
  }
  TapeLayout tl;
  carve_tape(const_cast<void*>(tape), n, m, k, S, sizeof(T), &tl);

  // 1. scoring adjoint -> Qbar, wbar (direct Q_H term)
  HEF_CHECK_CUDA(cudaMemsetAsync(w.QHbar, 0, K * sizeof(double), st));
  HEF_CHECK_CUDA(cudaMemsetAsync(w.wbar, 0, m1 * sizeof(double), st));

  HEF_LAUNCH("k_bwd_qhbar", st,
             k_bwd_qhbar<<<stride_grid(m1), kThreads, 0, st>>>(g, dR, R, argvec, QH, w.QHbar));
  const int nc = (K + 31) / 32;
  if (nc <= 1) launch_bwd_scores<T, 1>(g, Q, ldq, K, dR, argvec, QH, w, st);
  else if (nc <= 2) launch_bwd_scores<T, 2>(g, Q, ldq, K, dR, argvec, QH, w, st);
  else if (nc <= 4) launch_bwd_scores<T, 4>(g, Q, ldq, K, dR, argvec, QH, w, st);
  else if (nc <= 8) launch_bwd_scores<T, 8>(g, Q, ldq, K, dR, argvec, QH, w, st);
  else launch_bwd_scores<T, 16>(g, Q, ldq, K, dR, argvec, QH, w, st);
  T* Qbar = static_cast<T*>(w.Qbar);
  T* Ct = static_cast<T*>(w.C);
  T* RinvT = static_cast<T*>(w.RinvT);
  T* Z = static_cast<T*>(w.Z);
  T* Abar = static_cast<T*>(w.Abar);
  T* mean = static_cast<T*>(w.mean);
  HEF_LAUNCH("k_bwd_qbar", st,
             k_bwd_qbar<T><<<stride_grid(n * 32, 8), 256, 0, st>>>(g, K, w.spbar, w.omax, w.omin,
                                                                    Qbar));
  HEF_CHECK_LAUNCH();

  // 2. QR adjoint -> Abar and its column means
  const long long rpc = (n + w.nchunk - 1) / w.nchunk;
  const int kk_blocks = (K * K + 255) / 256;
  HEF_LAUNCH("k_bwd_xgram", st,
             k_bwd_xgram<T><<<dim3(kk_blocks, w.nchunk), 256, 0, st>>>(Qbar, Q, ldq, n, K, rpc,
                                                                         w.part));
  HEF_LAUNCH("k_bwd_copyltu", st,
             k_bwd_copyltu<T><<<kk_blocks, 256, 0, st>>>(w.part, K, w.nchunk, Ct));
  HEF_LAUNCH("k_bwd_rinv", st, k_bwd_rinv<T><<<1, 1024, 0, st>>>(Rfac, K, w.Rinv, RinvT));
  const int eg = stride_grid(n * K, 8);
  HEF_LAUNCH("k_bwd_qr_z", st, k_bwd_qr_z<T><<<eg, kThreads, 0, st>>>(Q, ldq, Qbar, Ct, n, K, Z));
  HEF_LAUNCH("k_bwd_qr_abar", st, k_bwd_qr_abar<T><<<eg, kThreads, 0, st>>>(Z, RinvT, n, K, Abar));
  HEF_CHECK_CUDA(cudaMemsetAsync(w.colsum, 0, K * sizeof(double), st));
  HEF_LAUNCH("k_bwd_colsum", st,
             k_bwd_colsum<T><<<num_sms() * 2, 256, 0, st>>>(Abar, n, K, w.colsum));
  HEF_LAUNCH("k_bwd_mean", st, k_bwd_mean<T><<<1, 256, 0, st>>>(w.colsum, n, K, mean));
  HEF_CHECK_LAUNCH();

  // 3. chains, j = k .. 1
  ChainBwd<T> c;
  c.n = (int)n, c.m = (int)m, c.S = S, c.k = k, c.K = K, c.j = 0;
  c.coef = tl.coef, c.inv_nu = tl.inv_nu;
  c.uc = static_cast<const T*>(tl.uc), c.ub = static_cast<const T*>(tl.ub);
  T* xbc[3];
  T* xbb[3];
  for (int q = 0; q < 3; ++q) {
    xbc[q] = static_cast<T*>(w.xbc[q]), xbb[q] = static_cast<T*>(w.xbb[q]);
    HEF_CHECK_CUDA(cudaMemsetAsync(xbc[q], 0, (size_t)n * S * sizeof(T), st));
    HEF_CHECK_CUDA(cudaMemsetAsync(xbb[q], 0, (size_t)(n + m) * S * sizeof(T), st));
  }
  c.xbc0 = xbc[0], c.xbc1 = xbc[1], c.xbc2 = xbc[2];
  c.xbb0 = xbb[0], c.xbb1 = xbb[1], c.xbb2 = xbb[2];
  c.zc = static_cast<T*>(w.zc), c.zb = static_cast<T*>(w.zb), c.sc = static_cast<T*>(w.sc);
  c.zs = static_cast<T*>(w.zs), c.yc = static_cast<T*>(w.yc), c.yb = static_cast<T*>(w.yb);
  c.Abar = Abar, c.mean = mean, c.wbar = w.wbar;
  c.sv = scal_view<T>(inc);
  const int rg = stride_grid((2 * n + m) * S, 8);
  const int egr = stride_grid(m1 * S, 8);
  const int vg = stride_grid(n * S, 8);
  const int eg1 = stride_grid(m1, 8);
  for (int j = k; j >= 1; --j) {
    c.j = j;
    HEF_LAUNCH("k_bwd_prep", st, k_bwd_prep<T><<<rg, kThreads, 0, st>>>(g, c));
    HEF_LAUNCH("k_bwd_edge1", st, k_bwd_edge1<T><<<egr, kThreads, 0, st>>>(g, c));
    HEF_LAUNCH("k_bwd_node", st, k_bwd_node<T><<<vg, kThreads, 0, st>>>(g, c));
    HEF_LAUNCH("k_bwd_edge2", st, k_bwd_edge2<T><<<eg1, kThreads, 0, st>>>(g, c));
    HEF_CHECK_LAUNCH();
    if (j >= 3) {  // slot j mod 3 next holds xbar_{j-3}, which starts at zero
      HEF_CHECK_CUDA(cudaMemsetAsync(xbc[j % 3], 0, (size_t)n * S * sizeof(T), st));
      HEF_CHECK_CUDA(cudaMemsetAsync(xbb[j % 3], 0, (size_t)(n + m) * S * sizeof(T), st));
    }
  }

  // 4. deflation of the start -> dx0, degree adjoints -> wbar
  HEF_CHECK_CUDA(cudaMemsetAsync(w.tdot, 0, 3 * S * sizeof(double), st));
  HEF_LAUNCH("k_bwd_defl_dots", st, k_bwd_defl_dots<T><<<rg, kThreads, 0, st>>>(g, c, w.tdot));
  HEF_LAUNCH("k_bwd_defl_out", st,
             k_bwd_defl_out<T><<<stride_grid(2 * n + m, 8), kThreads, 0, st>>>(g, c, w.tdot, x0c, x0b,
                                                                               dx0c, dx0b, w.dbar));
  HEF_LAUNCH("k_bwd_defl_w", st, k_bwd_defl_w<<<eg1, kThreads, 0, st>>>(g, w.dbar, w.wbar));
  HEF_LAUNCH("k_bwd_out_w", st, k_bwd_out_w<<<eg1, kThreads, 0, st>>>(g, w.wbar, dw));
  HEF_CHECK_LAUNCH();
  return HEF_OK;
}

hef_status check_bwd_args(const hef_incidence* inc, int k, int S, int dtype, const char* fn) {
  if (!inc) return set_error(HEF_ERR_INVALID_ARG, "%s: NULL incidence", fn);
  if (dtype != HEF_F64 && dtype != HEF_F32)
    return set_error(HEF_ERR_INVALID_ARG, "%s: dtype must be HEF_F64 or HEF_F32", fn);
  if (k < 1) return set_error(HEF_ERR_INVALID_ARG, "%s: k must be >= 1", fn);
  if (S < 1 || S > 16 || (S & (S - 1)))
    return set_error(HEF_ERR_UNSUPPORTED, "%s: S must be 1, 2, 4, 8 or 16", fn);
  if (2ll * k * S > 512) return set_error(HEF_ERR_UNSUPPORTED, "%s: K = 2kS must be <= 512", fn);
  if (inc->n < 1) return set_error(HEF_ERR_INVALID_ARG, "%s: n must be >= 1", fn);
  return HEF_OK;
}

}  // namespace

}  // namespace hef

using namespace hef;

extern "C" size_t hef_edge_resistance_backward_workspace_bytes(const hef_incidence* inc, int32_t k,
                                                               int32_t S, int32_t dtype,
                                                               int32_t recompute) {
  if (check_bwd_args(inc, k, S, dtype, "hef_edge_resistance_backward_workspace_bytes")) return 0;
  BwdWs w;
  return carve_bwd(nullptr, inc, k, S, dtype, recompute != 0, &w);
}

extern "C" hef_status hef_edge_resistance_backward(
    const hef_incidence* inc, int32_t k, int32_t S, int32_t dtype, const double* x0_clique,
    const double* x0_star, const void* tape, size_t tape_bytes, const void* Q, int64_t ldq,
    const double* R_fac, const double* QH, const int32_t* argvec, const double* R,
    const double* dR, double* dw, double* dx0_clique, double* dx0_star, void* workspace,
    size_t workspace_bytes, void* stream) {
  HEF_NVTX("hef_edge_resistance_backward");
  static const char* fn = "hef_edge_resistance_backward";
  hef_status s = check_bwd_args(inc, k, S, dtype, fn);
  if (s) return s;
  const long long K = 2ll * k * S;
  if (!x0_clique || !x0_star || !Q || !R_fac || !QH || !argvec || !R || !dR || !dw)
    return set_error(HEF_ERR_INVALID_ARG, "%s: NULL array", fn);
  const size_t esz = dtype == HEF_F64 ? 8 : 4;
  if (ldq < K || (ldq * esz) % 16 || (reinterpret_cast<uintptr_t>(Q) & 15))
    return set_error(HEF_ERR_INVALID_ARG, "%s: ldq must be >= K = %lld with 16-byte aligned rows",
                     fn, K);
  if (tape) {
    const size_t tneed = hef_krylov_tape_bytes(inc, k, S, dtype);
    if ((reinterpret_cast<uintptr_t>(tape) & 255) || tape_bytes < tneed)
      return set_error(HEF_ERR_WORKSPACE, "%s: tape needs %zu bytes (256-aligned)", fn, tneed);
  }
  const size_t need = hef_edge_resistance_backward_workspace_bytes(inc, k, S, dtype, tape == nullptr);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return set_error(HEF_ERR_WORKSPACE, "%s: workspace needs %zu bytes (256-aligned)", fn, need);
  BwdWs w;
  carve_bwd(workspace, inc, k, S, dtype, tape == nullptr, &w);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == HEF_F64)
    return run_bwd<double>(inc, k, S, x0_clique, x0_star, tape, static_cast<const double*>(Q), ldq,
                           R_fac, QH, argvec, R, dR, dw, dx0_clique, dx0_star, w, st);
  return run_bwd<float>(inc, k, S, x0_clique, x0_star, tape, static_cast<const float*>(Q), ldq,
                        R_fac, QH, argvec, R, dR, dw, dx0_clique, dx0_star, w, st);
}

extern "C" hef_status hef_backward_plan(const hef_incidence* inc, int32_t k, int32_t S,
                                        int32_t dtype, uint64_t budget_bytes, int32_t* use_tape,
                                        uint64_t* tape_bytes) {
  static const char* fn = "hef_backward_plan";
  hef_status s = check_bwd_args(inc, k, S, dtype, fn);
  if (s) return s;
  if (!use_tape) return set_error(HEF_ERR_INVALID_ARG, "%s: NULL use_tape", fn);
  const uint64_t tb = hef_krylov_tape_bytes(inc, k, S, dtype);
  uint64_t budget = budget_bytes;
  if (budget == 0) {
    size_t free_b = 0, total_b = 0;
    HEF_CHECK_CUDA(cudaMemGetInfo(&free_b, &total_b));
    budget = free_b / 2;
  }
  *use_tape = tb <= budget ? 1 : 0;
  if (tape_bytes) *tape_bytes = tb;
  return HEF_OK;
}
