// Krylov basis: Algorithm 1 step 3 (Eq. krylov, Section III-A.3).
//
// For each expansion (clique G_c on n vertices, star G_b on n + m vertices)
// and each of S starts, the chain x_1 .. x_k spans M x, ..., M^k x of the
// random-walk operator M = D^-1 W applied implicitly through the incidence:
//
//   clique:  (M_c x)_v = (1/d_c(v)) sum_{e ∋ v} wh_e (s_e - x_v),
//            s_e = sum_{p in e} x_p,  wh_e = w_e/(|e|-1)  (or w_e/C(|e|,2))
//   star:    (M_b x)_v = (1/d_b(v)) sum_{e ∋ v} (w_e/|e|) x_e
//            (M_b x)_e = (1/|e|)    sum_{p in e} x_p          (d_b(e) = w_e)
//
// Stabilisation is a three-term Lanczos recurrence in the degree-weighted
// inner product <a,b>_D (M is self-adjoint there), with the trivial
// eigenvectors of M deflated every step.  Subtracting multiples of earlier
// vectors of the same chain leaves the nested spans span{M x .. M^j x}
// unchanged, so the basis handed to orthonormalisation spans exactly the
// Krylov spaces of the definition.  Chain vectors are stored unnormalised
// (u_j) with their inverse D-norms in `inv_nu`; kernels scale on the fly.
//
// Layout: a chain block is row-major with the S starts of a row contiguous;
// one thread owns a whole row (S values, vector loads).  Per step: an edge
// pass (thread per hyperedge; hyperedges with more than kBig pins are summed
// by their whole warp), a vertex pass (thread per vertex, same split), which
// also archives x_{j-1} into V and reduces the Lanczos dots, and an update
// pass (thread per row) forming x_j and its D-norm.  Every reduction is a
// per-CTA partial followed by a two-level fixed-order sum (grid_reduce).
#include <algorithm>

#include "internal.h"

namespace hef {

namespace {

constexpr int kMaxS = 16;
constexpr int kBig = 16;     // segments longer than this are summed by a warp
// rows per thread in the update pass
template <typename T, int S>
__host__ __device__ constexpr int upd_rows() {
  return 4;
}
// entries gathered per round by one thread in the segment sums (wider rows
// keep two, for registers)
template <typename T, int S>
__host__ __device__ constexpr int seg_round() {
  return S * sizeof(T) <= 16 ? 4 : 2;
}

// Minimum resident CTAs per SM asked of the compiler for the step kernels:
// the FP32 form with S <= 4 fits one wave of the 200k-row workloads in its
// register budget; wider rows keep the compiler's choice (no spills).
template <typename T, int S>
constexpr int kMinBlocks(int want) {
  return (sizeof(T) == 4 && S <= 4) ? want : (S * sizeof(T) <= 32 ? 2 : 1);
}

template <typename T>
struct KView {
  int n, m;
  T* Yc;  // n x S
  T* Bc[2];
  T* Yb;  // (n+m) x S
  T* Bb[2];
  T* se;  // m x S
  double* inv_nu;  // (k+1) x 2S
  double* coef;    // (k+1) x 2S x 4: [ct, ct2, alpha, beta]
  T* nuT;          // inv_nu in the working type
  T* cfT;          // (k+1) x 2S x 4: [ct, ct2, alpha * nu_{j-1}, beta * nu_{j-2}]
  double* te;      // 3S: star edge-row dots of the current step
  double* itot;    // 3: 1 / the incidence's totals (0 where a total is 0), set by k_start_dots
  GridRed red;     // reduction scratch shared by all kernels (serialised)
  T* tape_c;       // nullable: u_j of the clique chains, (k+1) x n x S
  T* tape_b;       // nullable: u_j of the star chains, (k+1) x (n+m) x S
  double tol;      // breakdown threshold on the D-norm of a new vector
  unsigned int* gen;  // barrier generation of the persistent launch
};

// ---------------------------------------------------------------- row I/O

// a[i] for i in {0, 1} without indexing the array at run time (which would
// copy the kernel argument to local memory)
template <typename P>
__device__ __forceinline__ P pick2(P const (&a)[2], int i) {
  return i ? a[1] : a[0];
}

template <typename T, int S>
__device__ __forceinline__ void ldrow(const T* __restrict__ p, T (&v)[S]) {
  if constexpr (sizeof(T) == 4 && S % 4 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < S / 4; ++i) {
      const float4 f = __ldg(q + i);
      v[4 * i] = f.x, v[4 * i + 1] = f.y, v[4 * i + 2] = f.z, v[4 * i + 3] = f.w;
    }
  } else if constexpr (sizeof(T) == 8 && S % 2 == 0) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int i = 0; i < S / 2; ++i) {
      const double2 f = __ldg(q + i);
      v[2 * i] = f.x, v[2 * i + 1] = f.y;
    }
  } else {
#pragma unroll
    for (int s = 0; s < S; ++s) v[s] = __ldg(p + s);
  }
}

template <typename T, int S>
__device__ __forceinline__ void strow(T* __restrict__ p, const T (&v)[S]) {
  if constexpr (sizeof(T) == 4 && S % 4 == 0) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int i = 0; i < S / 4; ++i) q[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  } else if constexpr (sizeof(T) == 8 && S % 2 == 0) {
    double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
    for (int i = 0; i < S / 2; ++i) q[i] = make_double2(v[2 * i], v[2 * i + 1]);
  } else {
#pragma unroll
    for (int s = 0; s < S; ++s) p[s] = v[s];
  }
}

// Per-CTA partials of NQ*S values (slot q*S + s) written to part[block].
// Within a warp the values are summed by a transposing butterfly: at each
// level a lane keeps half of its values and adds its partner's copy of that
// half, so N values cost about N shuffles instead of 5 N; a lane ends with
// the warp sum of one slot.  Warps then meet in a fixed order, in the
// working type; only the CTA's sums are widened to FP64 (conversions and
// FP64 adds run at 1/64 rate on GB300).
template <int NQ, int S, typename A>
__device__ __forceinline__ void block_partials_qs(const A (&v)[NQ][S], double* part) {
  constexpr int N = NQ * S;
  constexpr int P = N > 16 ? 32 : (N > 8 ? 16 : (N > 4 ? 8 : (N > 2 ? 4 : (N > 1 ? 2 : 1))));
  constexpr int R = 32 / P;  // lanes that end up holding the same slot
  constexpr int NCH = (N + P - 1) / P;
  __shared__ A red[kThreads / 32][NCH * P];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int ch = 0; ch < NCH; ++ch) {
    A x[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
      const int idx = ch * P + i;
      x[i] = idx < N ? v[idx / S][idx % S] : (A)0;
    }
#pragma unroll
    for (int h = P / 2; h >= 1; h >>= 1) {
      const bool up = (lane & (h * R)) != 0;
#pragma unroll
      for (int i = 0; i < h; ++i) {
        const A send = up ? x[i] : x[i + h];
        const A keep = up ? x[i + h] : x[i];
        x[i] = keep + __shfl_xor_sync(0xffffffffu, send, h * R);
      }
    }
#pragma unroll
    for (int o = R / 2; o >= 1; o >>= 1) x[0] += __shfl_xor_sync(0xffffffffu, x[0], o);
    if (lane % R == 0) red[wid][ch * P + lane / R] = x[0];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    A acc = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc += red[w][t];
    part[(size_t)blockIdx.x * N + t] = (double)acc;
  }
}

// Sum of the S-rows of `X` over the entries [a, b) of an index list `idx`
// (X row = base + idx[t] * S) with weights, split between one thread (short
// lists) and its whole warp (lists longer than kBig, handled one at a time).
// W(t) gives the weight of entry t.  Result in acc (the owner thread).
template <typename T, int S, typename RowOf, typename WeightOf>
__device__ __forceinline__ void seg_sum(bool valid, int a, int b, RowOf row_of, WeightOf w_of,
                                        T (&acc)[S]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < S; ++s) acc[s] = 0;
  const bool big = valid && (b - a) > kBig;
  if (valid && !big) {
    int t = a;
    for (; t + 2 <= b; t += 2) {
      T v0[S], v1[S];
      ldrow<T, S>(row_of(t), v0);
      ldrow<T, S>(row_of(t + 1), v1);
      const T w0 = w_of(t), w1 = w_of(t + 1);
#pragma unroll
      for (int s = 0; s < S; ++s) acc[s] += w0 * v0[s] + w1 * v1[s];
    }
    if (t < b) {
      T v0[S];
      ldrow<T, S>(row_of(t), v0);
      const T w0 = w_of(t);
#pragma unroll
      for (int s = 0; s < S; ++s) acc[s] += w0 * v0[s];
    }
  }
  unsigned bigmask = __ballot_sync(0xffffffffu, big);
  while (bigmask) {
    const int src = __ffs(bigmask) - 1;
    bigmask &= bigmask - 1;
    const int ba = __shfl_sync(0xffffffffu, a, src), bb = __shfl_sync(0xffffffffu, b, src);
    T part[S];
#pragma unroll
    for (int s = 0; s < S; ++s) part[s] = 0;
    for (int t = ba + lane; t < bb; t += 32) {
      T v0[S];
      ldrow<T, S>(row_of(t), v0);
      const T w0 = w_of(t);
#pragma unroll
      for (int s = 0; s < S; ++s) part[s] += w0 * v0[s];
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part[s] += __shfl_xor_sync(0xffffffffu, part[s], o);
    }
    if (lane == src) {
#pragma unroll
      for (int s = 0; s < S; ++s) acc[s] = part[s];
    }
  }
}

// Two weighted row sums over one index list at once (the index is loaded
// once and both rows are in flight together): accA = sum_t wA(i) rowA(i),
// accB = sum_t wB(i) rowB(i) with i = idx(t), t in [a, b).  Lists longer than
// kBig are summed by the whole warp.
template <typename T, int S, typename Idx, typename RowA, typename RowB, typename WA, typename WB>
__device__ __forceinline__ void seg_sum2(bool valid, int a, int b, Idx idx, RowA rowA, RowB rowB,
                                         WA wA, WB wB, T (&accA)[S], T (&accB)[S]) {
  const int lane = threadIdx.x & 31;
  constexpr int kSeg = seg_round<T, S>();
#pragma unroll
  for (int s = 0; s < S; ++s) accA[s] = 0, accB[s] = 0;
  const bool big = valid && (b - a) > kBig;
  if (valid && !big) {
    // kSeg entries per round, all index loads then all row loads in flight
    // (indices past the end repeat the last entry and are weighted out)
    for (int t = a; t < b; t += kSeg) {
      int ii[kSeg];
#pragma unroll
      for (int q = 0; q < kSeg; ++q) ii[q] = idx(min(t + q, b - 1));
      T ra[kSeg][S], rb[kSeg][S];
#pragma unroll
      for (int q = 0; q < kSeg; ++q) {
        ldrow<T, S>(rowA(ii[q]), ra[q]);
        ldrow<T, S>(rowB(ii[q]), rb[q]);
      }
#pragma unroll
      for (int q = 0; q < kSeg; ++q) {
        const bool in = t + q < b;
        const T wa = in ? wA(ii[q]) : (T)0, wb = in ? wB(ii[q]) : (T)0;
#pragma unroll
        for (int s = 0; s < S; ++s) accA[s] += wa * ra[q][s], accB[s] += wb * rb[q][s];
      }
    }
  }
  unsigned bigmask = __ballot_sync(0xffffffffu, big);
  while (bigmask) {
    const int src = __ffs(bigmask) - 1;
    bigmask &= bigmask - 1;
    const int ba = __shfl_sync(0xffffffffu, a, src), bb = __shfl_sync(0xffffffffu, b, src);
    T pa[S], pb[S];
#pragma unroll
    for (int s = 0; s < S; ++s) pa[s] = 0, pb[s] = 0;
    for (int t = ba + lane; t < bb; t += 32) {
      const int i0 = idx(t);
      T a0[S], b0[S];
      ldrow<T, S>(rowA(i0), a0);
      ldrow<T, S>(rowB(i0), b0);
      const T wa0 = wA(i0), wb0 = wB(i0);
#pragma unroll
      for (int s = 0; s < S; ++s) pa[s] += wa0 * a0[s], pb[s] += wb0 * b0[s];
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        pa[s] += __shfl_xor_sync(0xffffffffu, pa[s], o);
        pb[s] += __shfl_xor_sync(0xffffffffu, pb[s], o);
      }
    }
    if (lane == src) {
#pragma unroll
      for (int s = 0; s < S; ++s) accA[s] = pa[s], accB[s] = pb[s];
    }
  }
}

// ---------------------------------------------------------------- start vectors

// D-weighted dots of the raw starts with the trivial vectors -> coef[0]; the
// starts, in the working type (and the internal hyperedge order), go to the
// first chain buffers for k_start_write (one FP64 -> working-type conversion).
// Rows: [0, n) clique, [n, 2n) star vertices, [2n, 2n+m) star hyperedges.
template <typename T, int S>
__global__ void __launch_bounds__(kThreads) k_start_dots(IncView g, ScalView<T> sv, KView<T> kv,
                                                         const double* __restrict__ x0c,
                                                         const double* __restrict__ x0b) {
  if (g.status[0]) return;
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  T acc[3][S];
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int s = 0; s < S; ++s) acc[q][s] = 0;
  T u[S];
  if (r < g.n) {
    const T d = sv.dc[r];
#pragma unroll
    for (int s = 0; s < S; ++s) u[s] = (T)x0c[r * S + s], acc[0][s] = d * u[s];
    strow<T, S>(kv.Bc[0] + r * S, u);
  } else if (r < 2ll * g.n) {
    const long long v = r - g.n;
    const T d = sv.db[v];
#pragma unroll
    for (int s = 0; s < S; ++s) u[s] = (T)x0b[v * S + s], acc[1][s] = d * u[s];
    strow<T, S>(kv.Bb[0] + v * S, u);
  } else if (r < 2ll * g.n + g.m) {
    const int i = (int)(r - 2ll * g.n);
    const T d = sv.ew[i];
    const long long src = (long long)(g.n + g.perm[i]) * S;
#pragma unroll
    for (int s = 0; s < S; ++s) u[s] = (T)x0b[src + s], acc[2][s] = d * u[s];
    strow<T, S>(kv.Bb[0] + (long long)(g.n + i) * S, u);
  }
  block_partials_qs<3, S, T>(acc, kv.red.part);
  __shared__ double tot[3 * kMaxS];
  if (grid_reduce(kv.red, 3 * S, tot)) {
    if (threadIdx.x < 3)
      kv.itot[threadIdx.x] = g.totals[threadIdx.x] > 0 ? 1.0 / g.totals[threadIdx.x] : 0.0;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
      double* cc = kv.coef + (size_t)s * 4;
      double* cb = kv.coef + (size_t)(S + s) * 4;
      cc[0] = g.totals[0] > 0 ? tot[0 * S + s] / g.totals[0] : 0.0;
      cc[1] = 0.0;
      cb[0] = g.totals[1] > 0 ? tot[1 * S + s] / g.totals[1] : 0.0;
      cb[1] = g.totals[2] > 0 ? tot[2 * S + s] / g.totals[2] : 0.0;
      T* tc = kv.cfT + (size_t)s * 4;
      T* tb = kv.cfT + (size_t)(S + s) * 4;
      tc[0] = (T)cc[0], tc[1] = (T)0, tb[0] = (T)cb[0], tb[1] = (T)cb[1];
    }
  }
}

// x_0 = start minus its trivial components (in place over the starts that
// k_start_dots stored); D-norm -> inv_nu[0].
template <typename T, int S>
__global__ void __launch_bounds__(kThreads) k_start_write(IncView g, ScalView<T> sv, KView<T> kv) {
  pdl_wait();
  pdl_trigger();
  if (g.status[0]) return;
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  T acc[2][S];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int s = 0; s < S; ++s) acc[q][s] = 0;
  if (r < g.n) {
    const T d = sv.dc[r];
    T u[S];
    ldrow<T, S>(kv.Bc[0] + r * S, u);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      u[s] -= (d > 0 ? kv.cfT[(size_t)s * 4] : (T)0);
      acc[0][s] = d * u[s] * u[s];
    }
    strow<T, S>(kv.Bc[0] + r * S, u);
    if (kv.tape_c) strow<T, S>(kv.tape_c + r * S, u);
  } else if (r < 2ll * g.n + g.m) {
    const long long rb = r - g.n;  // star row
    T d;
    int t;
    if (rb < g.n) {
      d = sv.db[rb], t = 0;
    } else {
      d = sv.ew[rb - g.n], t = 1;
    }
    T u[S];
    ldrow<T, S>(kv.Bb[0] + rb * S, u);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const T c = kv.cfT[(size_t)(S + s) * 4 + t];
      u[s] -= (d > 0 ? c : (T)0);
      acc[1][s] = d * u[s] * u[s];
    }
    strow<T, S>(kv.Bb[0] + rb * S, u);
    if (kv.tape_b) strow<T, S>(kv.tape_b + rb * S, u);
  }
  block_partials_qs<2, S, T>(acc, kv.red.part);
  __shared__ double tot[2 * kMaxS];
  if (grid_reduce(kv.red, 2 * S, tot)) {
    for (int c = threadIdx.x; c < 2 * S; c += blockDim.x) {
      const double nu2 = tot[c];  // slot op * S + s == chain c
      kv.inv_nu[c] = nu2 > 0.0 ? rsqrt(nu2) : 0.0;
      kv.nuT[c] = (T)kv.inv_nu[c];
    }
  }
}

// ---------------------------------------------------------------- one Krylov step
//
// Each pass is a per-item device function (one hyperedge, vertex or group of
// rows per thread, adding to the caller's partial dots) plus a final step
// run by the CTA that completes the grid-wide reduction.  The kernels
// k_edge_pass, k_node_pass and k_update run one item per thread;
// k_krylov_steps runs all k steps in one persistent launch over the same
// functions (grid-stride loops, bounded grid barriers).

// Edge pass item (hyperedge e; past the end it still takes part in its
// warp's collective sums): clique pin sums s_e, star rows (M_b x)_e, and the
// D-weighted dots of the star hyperedge rows, added to acc.
template <typename T, int S>
__device__ __forceinline__ void edge_item(const IncView& g, const ScalView<T>& sv,
                                          const KView<T>& kv, int j, int e, T (&acc)[3][S]) {
  const T* __restrict__ curc = pick2(kv.Bc, (j - 1) & 1);
  const T* __restrict__ curb = pick2(kv.Bb, (j - 1) & 1);
  const T* __restrict__ prvb = j >= 3 ? pick2(kv.Bb, j & 1) : nullptr;
  T ncc[S], ncb[S], npb[S];  // inverse norms of x_{j-1} (clique, star) and x_{j-2} (star)
#pragma unroll
  for (int s = 0; s < S; ++s) {
    ncc[s] = kv.nuT[(size_t)(j - 1) * 2 * S + s];
    ncb[s] = kv.nuT[(size_t)(j - 1) * 2 * S + S + s];
    npb[s] = j >= 2 ? kv.nuT[(size_t)(j - 2) * 2 * S + S + s] : (T)0;
  }
  const bool valid = e < g.m;
  int a = 0, b = 0;
  if (valid) a = g.ceptr[e], b = g.ceptr[e + 1];
  const int32_t* __restrict__ pins = g.cpins;
  T sc[S], sb[S];
  seg_sum2<T, S>(valid, a, b, [&](int t) { return __ldg(pins + t); },
                 [&](int p) { return curc + (long long)p * S; },
                 [&](int p) { return curb + (long long)p * S; }, [&](int) { return (T)1; },
                 [&](int) { return (T)1; }, sc, sb);
  if (valid) {
    const int k = b - a;
    const T invk = k >= 2 ? (T)1 / (T)k : (T)0;
    T ye[S], sev[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      sev[s] = sc[s] * ncc[s];
      ye[s] = sb[s] * ncb[s] * invk;
    }
    strow<T, S>(kv.se + (long long)e * S, sev);
    const long long row = (long long)(g.n + e) * S;
    strow<T, S>(kv.Yb + row, ye);
    if (k >= 2) {
      const T we = sv.ew[e];
      T xc[S], xp[S];
      ldrow<T, S>(curb + row, xc);
      if (prvb) ldrow<T, S>(prvb + row, xp);
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const T wy = we * ye[s];
        acc[0][s] += wy;
        acc[1][s] += wy * xc[s] * ncb[s];
        acc[2][s] += prvb ? wy * xp[s] * npb[s] : (T)0;
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ void edge_final(const KView<T>& kv, int S, const double* tot) {
  for (int t = threadIdx.x; t < 3 * S; t += blockDim.x) kv.te[t] = tot[t];
}

// Vertex pass item (vertex v): (M_c x)_v and (M_b x)_v, archive of x_{j-1}
// into V, and the dots of the Lanczos coefficients, added to acc.
template <typename T, int S>
__device__ __forceinline__ void node_item(const IncView& g, const ScalView<T>& sv,
                                          const KView<T>& kv, int j, int v, T (&acc)[6][S],
                                          T* __restrict__ V, long long ldv) {
  const T* __restrict__ curc = pick2(kv.Bc, (j - 1) & 1);
  const T* __restrict__ curb = pick2(kv.Bb, (j - 1) & 1);
  const T* __restrict__ prvc = j >= 3 ? pick2(kv.Bc, j & 1) : nullptr;
  const T* __restrict__ prvb = j >= 3 ? pick2(kv.Bb, j & 1) : nullptr;
  T ncc[S], ncb[S], npc[S], npb[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    ncc[s] = kv.nuT[(size_t)(j - 1) * 2 * S + s];
    ncb[s] = kv.nuT[(size_t)(j - 1) * 2 * S + S + s];
    npc[s] = j >= 2 ? kv.nuT[(size_t)(j - 2) * 2 * S + s] : (T)0;
    npb[s] = j >= 2 ? kv.nuT[(size_t)(j - 2) * 2 * S + S + s] : (T)0;
  }
  const bool valid = v < g.n;
  int a = 0, b = 0;
  if (valid) a = g.vptr[v], b = g.vptr[v + 1];
  const int32_t* __restrict__ ve = g.vedge;
  const T* __restrict__ se = kv.se;
  const T* __restrict__ ewh = sv.ewh;
  const T* __restrict__ ez = sv.ez;
  // the vertex's own rows and scalars first: their loads overlap the gathers
  T xv[S], xb[S], xpc[S], xpb[S];
  T wsum = 0, idc = 0, idb = 0, dcv = 0, dbv = 0;
  if (valid) {
    ldrow<T, S>(curc + (long long)v * S, xv);
    ldrow<T, S>(curb + (long long)v * S, xb);
    if (prvc) {
      ldrow<T, S>(prvc + (long long)v * S, xpc);
      ldrow<T, S>(prvb + (long long)v * S, xpb);
    }
    wsum = sv.wsc[v], idc = sv.inv_dc[v], idb = sv.inv_db[v], dcv = sv.dc[v], dbv = sv.db[v];
  }
  T accc[S], accb[S];
  seg_sum2<T, S>(valid, a, b, [&](int t) { return __ldg(ve + t); },
                 [&](int e) { return se + (long long)e * S; },
                 [&](int e) { return curb + (long long)(g.n + e) * S; },
                 [&](int e) { return __ldg(ewh + e); }, [&](int e) { return __ldg(ez + e); }, accc,
                 accb);
  if (valid) {
    T yc[S], yb[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      xv[s] *= ncc[s];
      xb[s] *= ncb[s];
      yc[s] = idc * (accc[s] - wsum * xv[s]);
      yb[s] = idb * accb[s] * ncb[s];
      const T pc = prvc ? xpc[s] * npc[s] : (T)0;
      const T pb = prvb ? xpb[s] * npb[s] : (T)0;
      acc[0][s] += dcv * yc[s];
      acc[1][s] += dcv * yc[s] * xv[s];
      acc[2][s] += dcv * yc[s] * pc;
      acc[3][s] += dbv * yb[s];
      acc[4][s] += dbv * yb[s] * xb[s];
      acc[5][s] += dbv * yb[s] * pb;
    }
    strow<T, S>(kv.Yc + (long long)v * S, yc);
    strow<T, S>(kv.Yb + (long long)v * S, yb);
    if (j >= 2) {  // x_{j-1} is basis vector j-1 -> column block j-2
      T* row = V + (long long)v * ldv + (long long)(j - 2) * 2 * S;
      strow<T, S>(row, xv);
      strow<T, S>(row + S, xb);
    }
  }
}

// Lanczos coefficients of step j from the vertex dots tn (6S) and the star
// hyperedge-row dots te (3S).
template <typename T>
__device__ __forceinline__ void node_final(const IncView& g, const KView<T>& kv, int S, int j,
                                           const double* tn) {
  for (int c = threadIdx.x; c < 2 * S; c += blockDim.x) {
    const int op = c / S, s = c % S;
    double* cf = kv.coef + ((size_t)j * 2 * S + c) * 4;
    if (op == 0) {
      cf[0] = tn[0 * S + s] * kv.itot[0];  // products: FP64 division is slow here
      cf[1] = 0.0;
      cf[2] = j >= 2 ? tn[1 * S + s] : 0.0;
      cf[3] = j >= 3 ? tn[2 * S + s] : 0.0;
    } else {
      cf[0] = tn[3 * S + s] * kv.itot[1];
      cf[1] = kv.te[0 * S + s] * kv.itot[2];
      cf[2] = j >= 2 ? tn[4 * S + s] + kv.te[1 * S + s] : 0.0;
      cf[3] = j >= 3 ? tn[5 * S + s] + kv.te[2 * S + s] : 0.0;
    }
    // working-type copies with the inverse norms folded in
    T* ct = kv.cfT + ((size_t)j * 2 * S + c) * 4;
    ct[0] = (T)cf[0];
    ct[1] = (T)cf[1];
    ct[2] = (T)(cf[2] * kv.inv_nu[(size_t)(j - 1) * 2 * S + c]);
    ct[3] = j >= 3 ? (T)(cf[3] * kv.inv_nu[(size_t)(j - 2) * 2 * S + c]) : (T)0;
  }
}

// Update pass item (rows r0 + it * blockDim.x, it < upd_rows): u_j = y -
// trivial part - alpha x_{j-1} - beta x_{j-2} (written over x_{j-2}'s
// buffer) and its D-norm, added to acc.  Rows: [0, n) clique, [n, 2n + m) star.
template <typename T, int S>
__device__ __forceinline__ void update_item(const IncView& g, const ScalView<T>& sv,
                                            const KView<T>& kv, int j, long long r0,
                                            T (&acc)[2][S]) {
  const bool has_prv = j >= 3;
  // coefficients of both expansions in registers: [op][s][ct, ct2, a, b]
  T cf[2][S][4];
#pragma unroll
  for (int op = 0; op < 2; ++op)
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int q = 0; q < 4; ++q) cf[op][s][q] = kv.cfT[((size_t)j * 2 * S + op * S + s) * 4 + q];
  const long long nrows = 2ll * g.n + g.m;
  constexpr int kUpdRows = upd_rows<T, S>();
#pragma unroll
  for (int it = 0; it < kUpdRows; ++it) {
    const long long r = r0 + (long long)it * blockDim.x;
    if (r >= nrows) break;
    const bool clique = r < g.n;
    const long long rr = clique ? r : r - g.n;
    const T* cur = clique ? pick2(kv.Bc, (j - 1) & 1) : pick2(kv.Bb, (j - 1) & 1);
    T* nw = clique ? pick2(kv.Bc, j & 1) : pick2(kv.Bb, j & 1);
    const T* Y = clique ? kv.Yc : kv.Yb;
    T d;
    int tsel;
    if (clique) d = sv.dc[rr], tsel = 0;
    else if (rr < g.n) d = sv.db[rr], tsel = 0;
    else d = sv.ew[rr - g.n], tsel = 1;
    T y[S], xc[S], xp[S], u[S], dsq[S];
    ldrow<T, S>(Y + rr * S, y);
    ldrow<T, S>(cur + rr * S, xc);
    if (has_prv) ldrow<T, S>(nw + rr * S, xp);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const T c0 = clique ? cf[0][s][0] : (tsel ? cf[1][s][1] : cf[1][s][0]);
      const T ca = clique ? cf[0][s][2] : cf[1][s][2];
      const T cb = clique ? cf[0][s][3] : cf[1][s][3];
      const T t = d > 0 ? c0 : (T)0;
      u[s] = y[s] - t - ca * xc[s] - (has_prv ? cb * xp[s] : (T)0);
      dsq[s] = d * u[s] * u[s];
    }
    strow<T, S>(nw + rr * S, u);
    if (clique && kv.tape_c) strow<T, S>(kv.tape_c + ((long long)j * g.n + rr) * S, u);
    if (!clique && kv.tape_b) strow<T, S>(kv.tape_b + ((long long)j * (g.n + g.m) + rr) * S, u);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if (clique) acc[0][s] += dsq[s];
      else acc[1][s] += dsq[s];
    }
  }
}

// Inverse D-norms of step j from the squared norms tot (2S).
template <typename T>
__device__ __forceinline__ void update_final(const KView<T>& kv, int S, int j, const double* tot) {
  const double* nu0 = kv.inv_nu + (size_t)(j - 1) * 2 * S;
  for (int c = threadIdx.x; c < 2 * S; c += blockDim.x) {
    const double nu2 = tot[c];
    const bool alive = nu0[c] > 0.0 && nu2 > kv.tol * kv.tol;
    kv.inv_nu[(size_t)j * 2 * S + c] = alive ? rsqrt(nu2) : 0.0;  // one FP64 rsqrt
    kv.nuT[(size_t)j * 2 * S + c] = (T)kv.inv_nu[(size_t)j * 2 * S + c];
  }
}

// Archive of the last chain vector x_k of vertex v into V.
template <typename T, int S>
__device__ __forceinline__ void archive_item(const IncView& g, const KView<T>& kv, int k, int v,
                                             T* __restrict__ V, long long ldv) {
  if (v >= g.n) return;
  T xc[S], xb[S];
  ldrow<T, S>(pick2(kv.Bc, k & 1) + (long long)v * S, xc);
  ldrow<T, S>(pick2(kv.Bb, k & 1) + (long long)v * S, xb);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    xc[s] *= kv.nuT[(size_t)k * 2 * S + s];
    xb[s] *= kv.nuT[(size_t)k * 2 * S + S + s];
  }
  T* row = V + (long long)v * ldv + (long long)(k - 1) * 2 * S;
  strow<T, S>(row, xc);
  strow<T, S>(row + S, xb);
}

template <int NQ, int S, typename T>
__device__ __forceinline__ void zero_acc(T (&acc)[NQ][S]) {
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int s = 0; s < S; ++s) acc[q][s] = 0;
}

// Edge pass of step j (thread per hyperedge).
template <typename T, int S>
__global__ void __launch_bounds__(kThreads, kMinBlocks<T, S>(6))
    k_edge_pass(IncView g, ScalView<T> sv, KView<T> kv, int j) {
  pdl_wait();
  pdl_trigger();
  if (g.status[0]) return;
  T acc[3][S];
  zero_acc(acc);
  edge_item<T, S>(g, sv, kv, j, blockIdx.x * blockDim.x + threadIdx.x, acc);
  block_partials_qs<3, S, T>(acc, kv.red.part);
  __shared__ double tot[3 * kMaxS];
  if (grid_reduce(kv.red, 3 * S, tot)) edge_final(kv, S, tot);
}

// Vertex pass of step j (thread per vertex); the final CTA forms the
// Lanczos coefficients.
template <typename T, int S>
__global__ void __launch_bounds__(kThreads, kMinBlocks<T, S>(4))
    k_node_pass(IncView g, ScalView<T> sv, KView<T> kv, int j, T* __restrict__ V, long long ldv) {
  pdl_wait();
  pdl_trigger();
  if (g.status[0]) return;
  T acc[6][S];
  zero_acc(acc);
  node_item<T, S>(g, sv, kv, j, blockIdx.x * blockDim.x + threadIdx.x, acc, V, ldv);
  block_partials_qs<6, S, T>(acc, kv.red.part);
  __shared__ double tn[6 * kMaxS];
  if (grid_reduce(kv.red, 6 * S, tn)) node_final(g, kv, S, j, tn);
}

// Update pass of step j (upd_rows rows per thread); the final CTA forms the
// inverse norms.
template <typename T, int S>
__global__ void __launch_bounds__(kThreads, kMinBlocks<T, S>(4))
    k_update(IncView g, ScalView<T> sv, KView<T> kv, int j) {
  pdl_wait();
  pdl_trigger();
  if (g.status[0]) return;
  T acc[2][S];
  zero_acc(acc);
  update_item<T, S>(g, sv, kv, j,
                    (long long)blockIdx.x * blockDim.x * upd_rows<T, S>() + threadIdx.x, acc);
  block_partials_qs<2, S, T>(acc, kv.red.part);
  __shared__ double tot[2 * kMaxS];
  if (grid_reduce(kv.red, 2 * S, tot)) update_final(kv, S, j, tot);
}

// Archive of the last chain vectors x_k into V (thread per vertex).
template <typename T, int S>
__global__ void __launch_bounds__(kThreads) k_archive_last(IncView g, KView<T> kv, int k,
                                                           T* __restrict__ V, long long ldv) {
  pdl_wait();
  if (g.status[0]) return;
  archive_item<T, S>(g, kv, k, blockIdx.x * blockDim.x + threadIdx.x, V, ldv);
}

// ---------------------------------------------------------------- persistent form

constexpr unsigned int kBarIters = 1u << 20;  // bounded barrier wait (about 0.25 s)

// Grid barrier with the pass's reduction: per-CTA partials, the two-level
// reduction of grid_reduce, the final step fin(tot) in the CTA that completes
// it, then a generation counter releases the others.  A wait that runs out
// sets HEF_WAIT_TIMEOUT in the status word; every later pass then stops.
template <int NQ, int S, typename T, typename Fin>
__device__ __forceinline__ void reduce_barrier(const KView<T>& kv, const T (&acc)[NQ][S],
                                               unsigned int* gen, unsigned int* status, Fin fin) {
  __shared__ unsigned int g0;
  __shared__ double tot[6 * kMaxS];
  if (threadIdx.x == 0) g0 = *reinterpret_cast<volatile unsigned int*>(gen);
  // (block_partials_qs begins and grid_reduce ends with a CTA barrier)
  block_partials_qs<NQ, S, T>(acc, kv.red.part);
  if (grid_reduce(kv.red, NQ * S, tot)) {
    fin(tot);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(gen, 1u);
    return;
  }
  if (threadIdx.x == 0) {
    unsigned int it = 0;
    while (*reinterpret_cast<volatile unsigned int*>(gen) == g0) {
      if (++it > kBarIters) {
        atomicOr(status, HEF_WAIT_TIMEOUT);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
}

__device__ __forceinline__ bool stopped(const unsigned int* status) {
  return *reinterpret_cast<const volatile unsigned int*>(status) != 0u;
}

// All k steps in one launch.  Every CTA must be resident at once (the grid is
// sized from the occupancy of this kernel); passes walk their items in
// grid-stride tiles of blockDim.x.
template <typename T, int S>
__global__ void __launch_bounds__(kThreads, kMinBlocks<T, S>(3))
    k_krylov_steps(IncView g, ScalView<T> sv, KView<T> kv, int k, T* __restrict__ V,
                   long long ldv, unsigned int* gen, unsigned int* status) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long base = (long long)blockIdx.x * blockDim.x;
  const long long nrows = 2ll * g.n + g.m;
  for (int j = 1; j <= k; ++j) {
    if (stopped(status)) return;
    {
      T acc[3][S];
      zero_acc(acc);
      for (long long e0 = base; e0 < g.m; e0 += stride)
        edge_item<T, S>(g, sv, kv, j, (int)(e0 + threadIdx.x), acc);
      reduce_barrier<3, S>(kv, acc, gen, status, [&](const double* tot) { edge_final(kv, S, tot); });
    }
    if (stopped(status)) return;
    {
      T acc[6][S];
      zero_acc(acc);
      for (long long v0 = base; v0 < g.n; v0 += stride)
        node_item<T, S>(g, sv, kv, j, (int)(v0 + threadIdx.x), acc, V, ldv);
      reduce_barrier<6, S>(kv, acc, gen, status,
                           [&](const double* tn) { node_final(g, kv, S, j, tn); });
    }
    if (stopped(status)) return;
    {
      T acc[2][S];
      zero_acc(acc);
      for (long long r0 = base * upd_rows<T, S>(); r0 < nrows; r0 += stride * upd_rows<T, S>())
        update_item<T, S>(g, sv, kv, j, r0 + threadIdx.x, acc);
      reduce_barrier<2, S>(kv, acc, gen, status,
                           [&](const double* tot) { update_final(kv, S, j, tot); });
    }
  }
  if (stopped(status)) return;
  for (long long v0 = base; v0 < g.n; v0 += stride)
    archive_item<T, S>(g, kv, k, (int)(v0 + threadIdx.x), V, ldv);
}

inline int blocks_for(long long rows) { return (int)((rows + kThreads - 1) / kThreads); }

template <typename T>
size_t carve_krylov(void* base, long long n, long long m, int k, int S, KView<T>* kv) {
  Carver c(base);
  const long long maxblk = blocks_for(2 * n + m);
  kv->n = (int)n;
  kv->m = (int)m;
  kv->Yc = c.take<T>(n * S);
  kv->Bc[0] = c.take<T>(n * S);
  kv->Bc[1] = c.take<T>(n * S);
  kv->Yb = c.take<T>((n + m) * S);
  kv->Bb[0] = c.take<T>((n + m) * S);
  kv->Bb[1] = c.take<T>((n + m) * S);
  kv->se = c.take<T>((m > 0 ? m : 1) * S);
  kv->inv_nu = c.take<double>((size_t)(k + 1) * 2 * S);
  kv->coef = c.take<double>((size_t)(k + 1) * 2 * S * 4);
  kv->nuT = c.take<T>((size_t)(k + 1) * 2 * S);
  kv->cfT = c.take<T>((size_t)(k + 1) * 2 * S * 4);
  kv->te = c.take<double>((size_t)3 * S);
  kv->itot = c.take<double>(4);
  kv->red.part = c.take<double>((size_t)maxblk * 6 * S);
  kv->red.gpart = c.take<double>((size_t)red_groups((int)maxblk) * 6 * S);
  kv->red.gcnt = c.take<unsigned int>(red_groups((int)maxblk) + 1);
  kv->red.tcnt = c.take<unsigned int>(1);
  kv->gen = c.take<unsigned int>(1);
  return c.bytes();
}

// Whether the one-launch form may be used by calls from this thread (the
// batched form, whose hypergraphs share the GPU, turns it off).
thread_local bool t_persistent = true;
// Test of the timeout path: launch the persistent form with twice the
// resident grid, so that its first barrier cannot complete.
thread_local bool t_force_oversized = false;

template <typename T, int S>
hef_status run_krylov_s(const hef_incidence* inc, int k, const double* x0c, const double* x0b,
                        T* V, long long ldv, KView<T>& kv, bool persistent, cudaStream_t st) {
  IncView g = view(inc);
  const ScalView<T> sv = scal_view<T>(inc);
  const long long n = inc->n, m = inc->m;
  const int grid_all = blocks_for(2 * n + m);
  const int grid_e = blocks_for(m > 0 ? m : 1);
  const int grid_n = blocks_for(n);
  const int grid_upd = blocks_for((2 * n + m + upd_rows<T, S>() - 1) / upd_rows<T, S>());
  HEF_LAUNCH("k_start_dots", st, k_start_dots<T, S><<<grid_all, kThreads, 0, st>>>(g, sv, kv, x0c, x0b));
  // the launches after the first are programmatically dependent on their
  // predecessor (each kernel waits for it before touching shared buffers)
  HEF_LAUNCH("k_start_write", st,
             HEF_CHECK_CUDA(launch_dependent(k_start_write<T, S>, grid_all, kThreads, st, g, sv, kv)));
  HEF_CHECK_LAUNCH();
  // one launch for all steps when every row of a pass has a resident thread
  // of its own (small hypergraphs, where per-step launches cost more than the
  // work); larger ones run faster as three launches per step, whose CTAs each
  // take one item per thread
  const int res = persistent ? num_sms() * resident_ctas(k_krylov_steps<T, S>, kThreads) : 0;
  if (persistent && t_force_oversized) {
    // the timeout test: a plain launch of twice the resident grid, so that
    // the first barrier cannot complete and its bounded wait runs out
    const int grid = std::max(1, std::min(2 * res, grid_all));
    HEF_LAUNCH("k_krylov_steps", st, k_krylov_steps<T, S><<<grid, kThreads, 0, st>>>(
                                         g, sv, kv, k, V, ldv, kv.gen, inc->status));
    HEF_CHECK_LAUNCH();
    return HEF_OK;
  }
  if (persistent && (long long)res * kThreads >= 2 * n + m) {
    // cooperative: the runtime guarantees that all CTAs are resident at once
    // (other work on the GPU delays the start instead of starving a barrier);
    // if it refuses the grid, the per-step form below runs instead
    const int grid = std::max(1, std::min(res, grid_all));
    cudaError_t e = cudaSuccess;
    HEF_LAUNCH("k_krylov_steps", st,
               e = launch_cooperative(k_krylov_steps<T, S>, grid, kThreads, st, g, sv, kv, k, V,
                                      ldv, kv.gen, inc->status));
    if (e == cudaSuccess) return HEF_OK;
    if (e != cudaErrorCooperativeLaunchTooLarge && e != cudaErrorNotSupported)
      return set_error(HEF_ERR_CUDA, "k_krylov_steps: %s", cudaGetErrorString(e));
    (void)cudaGetLastError();
  }
  for (int j = 1; j <= k; ++j) {
    HEF_LAUNCH("k_edge_pass", st,
               HEF_CHECK_CUDA(launch_dependent(k_edge_pass<T, S>, grid_e, kThreads, st, g, sv, kv, j)));
    HEF_LAUNCH("k_node_pass", st,
               HEF_CHECK_CUDA(launch_dependent(k_node_pass<T, S>, grid_n, kThreads, st, g, sv, kv,
                                               j, V, ldv)));
    HEF_LAUNCH("k_update", st,
               HEF_CHECK_CUDA(launch_dependent(k_update<T, S>, grid_upd, kThreads, st, g, sv, kv, j)));
    HEF_CHECK_LAUNCH();
  }
  HEF_LAUNCH("k_archive_last", st,
             HEF_CHECK_CUDA(launch_dependent(k_archive_last<T, S>, grid_n, kThreads, st, g, kv, k,
                                             V, ldv)));
  HEF_CHECK_LAUNCH();
  return HEF_OK;
}

template <typename T>
hef_status run_krylov(const hef_incidence* inc, int k, int S, const double* x0c, const double* x0b,
                      void* Vv, long long ldv, void* ws, cudaStream_t st, void* tape = nullptr) {
  KView<T> kv;
  carve_krylov<T>(ws, inc->n, inc->m, k, S, &kv);
  TapeLayout tl;
  carve_tape(tape, inc->n, inc->m, k, S, sizeof(T), &tl);
  kv.tape_c = static_cast<T*>(tl.uc);
  kv.tape_b = static_cast<T*>(tl.ub);
  kv.tol = sizeof(T) == 8 ? 1e-12 : 1e-5;
  const int ngr = red_groups(blocks_for(2 * inc->n + inc->m));
  HEF_CHECK_CUDA(cudaMemsetAsync(kv.red.gcnt, 0, (ngr + 1) * sizeof(unsigned int), st));
  HEF_CHECK_CUDA(cudaMemsetAsync(kv.red.tcnt, 0, sizeof(unsigned int), st));
  T* V = static_cast<T*>(Vv);
  hef_status s;
  switch (S) {
    case 1: s = run_krylov_s<T, 1>(inc, k, x0c, x0b, V, ldv, kv, t_persistent, st); break;
    case 2: s = run_krylov_s<T, 2>(inc, k, x0c, x0b, V, ldv, kv, t_persistent, st); break;
    case 4: s = run_krylov_s<T, 4>(inc, k, x0c, x0b, V, ldv, kv, t_persistent, st); break;
    case 8: s = run_krylov_s<T, 8>(inc, k, x0c, x0b, V, ldv, kv, t_persistent, st); break;
    case 16: s = run_krylov_s<T, 16>(inc, k, x0c, x0b, V, ldv, kv, t_persistent, st); break;
    default: return set_error(HEF_ERR_UNSUPPORTED, "hef_krylov_basis: S must be 1, 2, 4, 8 or 16");
  }
  if (s || !tape) return s;
  HEF_CHECK_CUDA(cudaMemcpyAsync(tl.coef, kv.coef, (size_t)(k + 1) * 2 * S * 4 * sizeof(double),
                                 cudaMemcpyDeviceToDevice, st));
  HEF_CHECK_CUDA(cudaMemcpyAsync(tl.inv_nu, kv.inv_nu, (size_t)(k + 1) * 2 * S * sizeof(double),
                                 cudaMemcpyDeviceToDevice, st));
  return HEF_OK;
}

hef_status check_krylov_args(const hef_incidence* inc, int k, int S, int dtype, const char* fn) {
  if (!inc) return set_error(HEF_ERR_INVALID_ARG, "%s: NULL incidence", fn);
  if (dtype != HEF_F64 && dtype != HEF_F32)
    return set_error(HEF_ERR_INVALID_ARG, "%s: dtype must be HEF_F64 or HEF_F32", fn);
  if (k < 1) return set_error(HEF_ERR_INVALID_ARG, "%s: k must be >= 1", fn);
  if (S < 1 || S > kMaxS || (S & (S - 1)))
    return set_error(HEF_ERR_UNSUPPORTED, "%s: S must be 1, 2, 4, 8 or 16", fn);
  if (2ll * k * S > 512) return set_error(HEF_ERR_UNSUPPORTED, "%s: K = 2kS must be <= 512", fn);
  return HEF_OK;
}

}  // namespace

void krylov_allow_persistent(bool on) { t_persistent = on; }
void krylov_force_oversized(bool on) { t_force_oversized = on; }

}  // namespace hef

using namespace hef;

extern "C" size_t hef_krylov_workspace_bytes(const hef_incidence* inc, int32_t k, int32_t S,
                                             int32_t dtype) {
  if (check_krylov_args(inc, k, S, dtype, "hef_krylov_workspace_bytes")) return 0;
  if (dtype == HEF_F64) {
    KView<double> kv;
    return carve_krylov<double>(nullptr, inc->n, inc->m, k, S, &kv);
  }
  KView<float> kv;
  return carve_krylov<float>(nullptr, inc->n, inc->m, k, S, &kv);
}

extern "C" hef_status hef_krylov_basis(const hef_incidence* inc, int32_t k, int32_t S,
                                       int32_t dtype, const double* x0_clique,
                                       const double* x0_star, void* V, int64_t ldv,
                                       void* workspace, size_t workspace_bytes, void* stream) {
  hef_status s = check_krylov_args(inc, k, S, dtype, "hef_krylov_basis");
  if (s) return s;
  const long long K = 2ll * k * S;
  if (!x0_clique || !x0_star || !V)
    return set_error(HEF_ERR_INVALID_ARG, "hef_krylov_basis: NULL array");
  const size_t esz = dtype == HEF_F64 ? 8 : 4;
  if (ldv < K || (ldv * esz) % 16 || (reinterpret_cast<uintptr_t>(V) & 15))
    return set_error(HEF_ERR_INVALID_ARG,
                     "hef_krylov_basis: ldv must be >= K = %lld with 16-byte aligned rows", K);
  size_t need = hef_krylov_workspace_bytes(inc, k, S, dtype);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return set_error(HEF_ERR_WORKSPACE, "hef_krylov_basis: workspace needs %zu bytes (256-aligned)",
                     need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == HEF_F64) return run_krylov<double>(inc, k, S, x0_clique, x0_star, V, ldv, workspace, st);
  return run_krylov<float>(inc, k, S, x0_clique, x0_star, V, ldv, workspace, st);
}

extern "C" hef_status hef_set_krylov_persistent(int32_t on) {
  if (on < 0 || on > 2) return set_error(HEF_ERR_INVALID_ARG, "hef_set_krylov_persistent: on must be 0, 1 or 2");
  krylov_allow_persistent(on != 0);
  krylov_force_oversized(on == 2);
  return HEF_OK;
}

extern "C" size_t hef_krylov_tape_bytes(const hef_incidence* inc, int32_t k, int32_t S, int32_t dtype) {
  if (check_krylov_args(inc, k, S, dtype, "hef_krylov_tape_bytes")) return 0;
  TapeLayout tl;
  return carve_tape(nullptr, inc->n, inc->m, k, S, dtype == HEF_F64 ? 8 : 4, &tl);
}

extern "C" hef_status hef_krylov_basis_tape(const hef_incidence* inc, int32_t k, int32_t S,
                                            int32_t dtype, const double* x0_clique,
                                            const double* x0_star, void* V, int64_t ldv,
                                            void* tape, size_t tape_bytes, void* workspace,
                                            size_t workspace_bytes, void* stream) {
  hef_status s = check_krylov_args(inc, k, S, dtype, "hef_krylov_basis_tape");
  if (s) return s;
  const long long K = 2ll * k * S;
  if (!x0_clique || !x0_star || !V || !tape)
    return set_error(HEF_ERR_INVALID_ARG, "hef_krylov_basis_tape: NULL array");
  const size_t esz = dtype == HEF_F64 ? 8 : 4;
  if (ldv < K || (ldv * esz) % 16 || (reinterpret_cast<uintptr_t>(V) & 15))
    return set_error(HEF_ERR_INVALID_ARG,
                     "hef_krylov_basis_tape: ldv must be >= K = %lld with 16-byte aligned rows", K);
  const size_t need = hef_krylov_workspace_bytes(inc, k, S, dtype);
  const size_t tneed = hef_krylov_tape_bytes(inc, k, S, dtype);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return set_error(HEF_ERR_WORKSPACE, "hef_krylov_basis_tape: workspace needs %zu bytes", need);
  if ((reinterpret_cast<uintptr_t>(tape) & 255) || tape_bytes < tneed)
    return set_error(HEF_ERR_WORKSPACE, "hef_krylov_basis_tape: tape needs %zu bytes", tneed);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == HEF_F64)
    return run_krylov<double>(inc, k, S, x0_clique, x0_star, V, ldv, workspace, st, tape);
  return run_krylov<float>(inc, k, S, x0_clique, x0_star, V, ldv, workspace, st, tape);
}
