// Krylov basis: Algorithm 1 step 3 (Eq. krylov, Section III-A.4).
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
// Per step: an edge pass (segmented sums over each hyperedge's pins), a
// vertex pass (segmented sums over each vertex's hyperedges, which also
// archives x_{j-1} into V and reduces the Lanczos dot products), and an update
// pass (x_j = y - projections, with its D-norm).  Every reduction is a
// per-CTA partial followed by a fixed-order sum in the last CTA.
#include "internal.h"

namespace hef {

namespace {

constexpr int kMaxS = 16;
constexpr int kGridPerSm = 4;

template <typename T>
struct KView {
  int n, m, S, lgS;
  T* Yc;  // n x S
  T* Bc[2];
  T* Yb;  // (n+m) x S
  T* Bb[2];
  T* se;  // m x S
  double* inv_nu;  // (k+1) x 2S
  double* coef;    // (k+1) x 2S x 4: [ct, ct2, alpha, beta]
  double* part_e;  // grid x S x 4
  double* part_n;  // grid x S x 8
  double* part_u;  // grid x 2S
  double* part_s;  // grid x 3S (start)
  unsigned int* counter;
  double tol;  // breakdown threshold on the D-norm of a new vector
};

// Per-CTA partials of NQ quantities per column s (thread layout: s = idx mod S).
// part[block][s][q].
template <int NQ, typename A>
__device__ __forceinline__ void partials_per_s(const A (&v)[NQ], int S, double* part) {
  __shared__ double red[NQ][kThreads / 32][kMaxS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    A x = v[q];
    for (int o = 16; o >= S; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane < S) red[q][wid][lane] = (double)x;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NQ * S; t += blockDim.x) {
    const int s = t / NQ, q = t % NQ;
    double acc = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc += red[q][w][s];
    part[(size_t)blockIdx.x * NQ * S + t] = acc;
  }
  __syncthreads();
}

// ----------------------------------------------------------------- start vectors

// D-weighted dots of the raw starts with the trivial vectors.
template <typename T>
__global__ void k_start_dots(IncView g, KView<T> kv, const double* __restrict__ x0c,
                             const double* __restrict__ x0b) {
  if (g.status[0]) return;
  const int S = kv.S, lgS = kv.lgS;
  double acc[3] = {0.0, 0.0, 0.0};  // clique t, star vertex t, star edge t
  const long long nc = (long long)g.n << lgS;
  const long long nb = (long long)(g.n + g.m) << lgS;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nc + nb;
       idx += (long long)gridDim.x * blockDim.x) {
    if (idx < nc) {
      const int v = (int)(idx >> lgS);
      acc[0] += g.dc[v] * x0c[idx];
    } else {
      const long long j = idx - nc;
      const int r = (int)(j >> lgS), s = (int)(j & (S - 1));
      if (r < g.n) {
        acc[1] += g.db[r] * x0b[j];
      } else {
        const int i = r - g.n;
        acc[2] += g.ew[i] * x0b[((long long)(g.n + g.perm[i]) << lgS) + s];
      }
    }
  }
  partials_per_s<3, double>(acc, S, kv.part_s);
  if (last_block_done(kv.counter)) {
    __shared__ double tot[3 * kMaxS];
    reduce_slots(kv.part_s, gridDim.x, 3 * S, tot);
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
      double* cc = kv.coef + (size_t)(0 * 2 * S + s) * 4;
      double* cb = kv.coef + (size_t)(0 * 2 * S + S + s) * 4;
      cc[0] = g.totals[0] > 0 ? tot[s * 3 + 0] / g.totals[0] : 0.0;
      cc[1] = 0.0;
      cb[0] = g.totals[1] > 0 ? tot[s * 3 + 1] / g.totals[1] : 0.0;
      cb[1] = g.totals[2] > 0 ? tot[s * 3 + 2] / g.totals[2] : 0.0;
    }
  }
}

// x_0 = start minus its trivial components; D-norm -> inv_nu[0].
template <typename T>
__global__ void k_start_write(IncView g, KView<T> kv, const double* __restrict__ x0c,
                              const double* __restrict__ x0b) {
  if (g.status[0]) return;
  const int S = kv.S, lgS = kv.lgS;
  double acc[2] = {0.0, 0.0};
  const long long nc = (long long)g.n << lgS;
  const long long nb = (long long)(g.n + g.m) << lgS;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nc + nb;
       idx += (long long)gridDim.x * blockDim.x) {
    if (idx < nc) {
      const int v = (int)(idx >> lgS), s = (int)(idx & (S - 1));
      const double d = g.dc[v];
      const double u = x0c[idx] - (d > 0 ? kv.coef[(size_t)s * 4 + 0] : 0.0);
      kv.Bc[0][idx] = (T)u;
      acc[0] += d * u * u;
    } else {
      const long long j = idx - nc;
      const int r = (int)(j >> lgS), s = (int)(j & (S - 1));
      const double* cb = kv.coef + (size_t)(S + s) * 4;
      double d, u;
      if (r < g.n) {
        d = g.db[r];
        u = x0b[j] - (d > 0 ? cb[0] : 0.0);
      } else {
        const int i = r - g.n;
        d = g.ew[i];
        u = x0b[((long long)(g.n + g.perm[i]) << lgS) + s] - (d > 0 ? cb[1] : 0.0);
      }
      kv.Bb[0][j] = (T)u;
      acc[1] += d * u * u;
    }
  }
  partials_per_s<2, double>(acc, S, kv.part_s);
  if (last_block_done(kv.counter)) {
    __shared__ double tot[2 * kMaxS];
    reduce_slots(kv.part_s, gridDim.x, 2 * S, tot);
    for (int c = threadIdx.x; c < 2 * S; c += blockDim.x) {
      const int op = c / S, s = c % S;
      const double nu2 = tot[s * 2 + op];
      kv.inv_nu[c] = nu2 > 0.0 ? 1.0 / sqrt(nu2) : 0.0;
    }
  }
}

// ----------------------------------------------------------------- one Krylov step

// Edge pass of step j: clique pin sums s_e, star rows (M_b x)_e and the
// D-weighted dots of the star edge rows.
template <typename T>
__global__ void k_edge_pass(IncView g, KView<T> kv, int j) {
  if (g.status[0]) return;
  const int S = kv.S, lgS = kv.lgS;
  const T* __restrict__ curc = kv.Bc[(j - 1) & 1];
  const T* __restrict__ curb = kv.Bb[(j - 1) & 1];
  const T* __restrict__ prvb = j >= 3 ? kv.Bb[j & 1] : nullptr;
  const double* nu0 = kv.inv_nu + (size_t)(j - 1) * 2 * S;
  const double* nup = j >= 2 ? kv.inv_nu + (size_t)(j - 2) * 2 * S : nullptr;
  T acc[4] = {0, 0, 0, 0};  // sum w y, sum w y x_cur, sum w y x_prv, sum w y^2
  const long long work = (long long)g.m << lgS;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < work;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx >> lgS), s = (int)(idx & (S - 1));
    const int a = g.ceptr[i], b = g.ceptr[i + 1];
    T sc = 0, sb = 0;
    int t = a;
    for (; t + 4 <= b; t += 4) {  // four independent gathers in flight
      const long long p0 = g.cpins[t], p1 = g.cpins[t + 1], p2 = g.cpins[t + 2],
                      p3 = g.cpins[t + 3];
      const T c0 = curc[(p0 << lgS) + s], c1 = curc[(p1 << lgS) + s];
      const T c2 = curc[(p2 << lgS) + s], c3 = curc[(p3 << lgS) + s];
      const T b0 = curb[(p0 << lgS) + s], b1 = curb[(p1 << lgS) + s];
      const T b2 = curb[(p2 << lgS) + s], b3 = curb[(p3 << lgS) + s];
      sc += (c0 + c1) + (c2 + c3);
      sb += (b0 + b1) + (b2 + b3);
    }
    for (; t < b; ++t) {
      const long long p = g.cpins[t];
      sc += curc[(p << lgS) + s];
      sb += curb[(p << lgS) + s];
    }
    const T ic = (T)nu0[s], ib = (T)nu0[S + s];
    kv.se[idx] = sc * ic;
    const int k = b - a;
    const long long row = ((long long)(g.n + i) << lgS) + s;
    T ye = 0;
    if (k >= 2) {
      ye = sb * ib / (T)k;
      const T we = (T)g.ew[i];
      const T xc = curb[row] * ib;
      const T xp = prvb ? prvb[row] * (T)nup[S + s] : (T)0;
      acc[0] += we * ye;
      acc[1] += we * ye * xc;
      acc[2] += we * ye * xp;
      acc[3] += we * ye * ye;
    }
    kv.Yb[row] = ye;
  }
  partials_per_s<4, T>(acc, S, kv.part_e);
}

// Vertex pass of step j: (M_c x)_v and (M_b x)_v, archive of x_{j-1} into V,
// and the Lanczos coefficients (last CTA, with the edge pass partials).
template <typename T>
__global__ void k_node_pass(IncView g, KView<T> kv, int j, int grid_e, T* __restrict__ V,
                            long long ldv) {
  if (g.status[0]) return;
  const int S = kv.S, lgS = kv.lgS;
  const T* __restrict__ curc = kv.Bc[(j - 1) & 1];
  const T* __restrict__ curb = kv.Bb[(j - 1) & 1];
  const T* __restrict__ prvc = j >= 3 ? kv.Bc[j & 1] : nullptr;
  const T* __restrict__ prvb = j >= 3 ? kv.Bb[j & 1] : nullptr;
  const double* nu0 = kv.inv_nu + (size_t)(j - 1) * 2 * S;
  const double* nup = j >= 2 ? kv.inv_nu + (size_t)(j - 2) * 2 * S : nullptr;
  T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const long long work = (long long)g.n << lgS;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < work;
       idx += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(idx >> lgS), s = (int)(idx & (S - 1));
    T accc = 0, wsum = 0, accb = 0;
    for (int t = g.vptr[v]; t < g.vptr[v + 1]; ++t) {
      const int e = g.vedge[t];
      const T wh = (T)g.ewh[e];
      accc += wh * kv.se[((long long)e << lgS) + s];
      wsum += wh;
      accb += (T)g.ez[e] * curb[((long long)(g.n + e) << lgS) + s];
    }
    const T ic = (T)nu0[s], ib = (T)nu0[S + s];
    const T xv = curc[idx] * ic;
    const T xb = curb[idx] * ib;
    const T yc = (T)g.inv_dc[v] * (accc - wsum * xv);
    const T yb = (T)g.inv_db[v] * accb * ib;
    kv.Yc[idx] = yc;
    kv.Yb[idx] = yb;
    if (j >= 2) {  // x_{j-1} is basis vector j-1 -> column block j-2
      T* row = V + (long long)v * ldv + (long long)(j - 2) * 2 * S;
      row[s] = xv;
      row[S + s] = xb;
    }
    const T dcv = (T)g.dc[v], dbv = (T)g.db[v];
    const T xpc = prvc ? prvc[idx] * (T)nup[s] : (T)0;
    const T xpb = prvb ? prvb[idx] * (T)nup[S + s] : (T)0;
    acc[0] += dcv * yc;
    acc[1] += dcv * yc * xv;
    acc[2] += dcv * yc * xpc;
    acc[3] += dcv * yc * yc;
    acc[4] += dbv * yb;
    acc[5] += dbv * yb * xb;
    acc[6] += dbv * yb * xpb;
    acc[7] += dbv * yb * yb;
  }
  partials_per_s<8, T>(acc, S, kv.part_n);
  if (last_block_done(kv.counter)) {
    __shared__ double tn[8 * kMaxS];
    __shared__ double te[4 * kMaxS];
    reduce_slots(kv.part_n, gridDim.x, 8 * S, tn);
    reduce_slots(kv.part_e, grid_e, 4 * S, te);
    for (int c = threadIdx.x; c < 2 * S; c += blockDim.x) {
      const int op = c / S, s = c % S;
      double* cf = kv.coef + ((size_t)j * 2 * S + c) * 4;
      if (op == 0) {
        cf[0] = g.totals[0] > 0 ? tn[s * 8 + 0] / g.totals[0] : 0.0;
        cf[1] = 0.0;
        cf[2] = j >= 2 ? tn[s * 8 + 1] : 0.0;
        cf[3] = j >= 3 ? tn[s * 8 + 2] : 0.0;
      } else {
        cf[0] = g.totals[1] > 0 ? tn[s * 8 + 4] / g.totals[1] : 0.0;
        cf[1] = g.totals[2] > 0 ? te[s * 4 + 0] / g.totals[2] : 0.0;
        cf[2] = j >= 2 ? tn[s * 8 + 5] + te[s * 4 + 1] : 0.0;
        cf[3] = j >= 3 ? tn[s * 8 + 6] + te[s * 4 + 2] : 0.0;
      }
    }
  }
}

// Update pass of step j: u_j = y - trivial part - alpha x_{j-1} - beta x_{j-2}
// (written over x_{j-2}'s buffer) and its D-norm -> inv_nu[j].
template <typename T>
__global__ void k_update(IncView g, KView<T> kv, int j) {
  if (g.status[0]) return;
  const int S = kv.S, lgS = kv.lgS;
  const T* __restrict__ curc = kv.Bc[(j - 1) & 1];
  const T* __restrict__ curb = kv.Bb[(j - 1) & 1];
  T* newc = kv.Bc[j & 1];  // holds x_{j-2} (read first when j >= 3)
  T* newb = kv.Bb[j & 1];
  const bool has_prv = j >= 3;
  const double* nu0 = kv.inv_nu + (size_t)(j - 1) * 2 * S;
  const double* nup = has_prv ? kv.inv_nu + (size_t)(j - 2) * 2 * S : nullptr;
  const double* cf = kv.coef + (size_t)j * 2 * S * 4;
  T acc[2] = {0, 0};
  const long long nc = (long long)g.n << lgS;
  const long long nb = (long long)(g.n + g.m) << lgS;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nc + nb;
       idx += (long long)gridDim.x * blockDim.x) {
    if (idx < nc) {
      const int v = (int)(idx >> lgS), s = (int)(idx & (S - 1));
      const double* c = cf + (size_t)s * 4;
      const T d = (T)g.dc[v];
      const T xc = curc[idx] * (T)nu0[s];
      const T xp = has_prv ? newc[idx] * (T)nup[s] : (T)0;
      const T u = kv.Yc[idx] - (d > 0 ? (T)c[0] : (T)0) - (T)c[2] * xc - (T)c[3] * xp;
      newc[idx] = u;
      acc[0] += d * u * u;
    } else {
      const long long jj = idx - nc;
      const int r = (int)(jj >> lgS), s = (int)(jj & (S - 1));
      const double* c = cf + (size_t)(S + s) * 4;
      T d, t;
      if (r < g.n) {
        d = (T)g.db[r];
        t = d > 0 ? (T)c[0] : (T)0;
      } else {
        d = (T)g.ew[r - g.n];
        t = d > 0 ? (T)c[1] : (T)0;
      }
      const T xc = curb[jj] * (T)nu0[S + s];
      const T xp = has_prv ? newb[jj] * (T)nup[S + s] : (T)0;
      const T u = kv.Yb[jj] - t - (T)c[2] * xc - (T)c[3] * xp;
      newb[jj] = u;
      acc[1] += d * u * u;
    }
  }
  partials_per_s<2, T>(acc, S, kv.part_u);
  if (last_block_done(kv.counter)) {
    __shared__ double tot[2 * kMaxS];
    reduce_slots(kv.part_u, gridDim.x, 2 * S, tot);
    for (int c = threadIdx.x; c < 2 * S; c += blockDim.x) {
      const int op = c / S, s = c % S;
      const double nu2 = tot[s * 2 + op];
      const bool alive = nu0[c] > 0.0 && nu2 > kv.tol * kv.tol;
      kv.inv_nu[(size_t)j * 2 * S + c] = alive ? 1.0 / sqrt(nu2) : 0.0;
    }
  }
}

// Archive of the last chain vectors x_k into V.
template <typename T>
__global__ void k_archive_last(IncView g, KView<T> kv, int k, T* __restrict__ V, long long ldv) {
  if (g.status[0]) return;
  const int S = kv.S, lgS = kv.lgS;
  const T* curc = kv.Bc[k & 1];
  const T* curb = kv.Bb[k & 1];
  const double* nu = kv.inv_nu + (size_t)k * 2 * S;
  const long long work = (long long)g.n << lgS;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < work;
       idx += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(idx >> lgS), s = (int)(idx & (S - 1));
    T* row = V + (long long)v * ldv + (long long)(k - 1) * 2 * S;
    row[s] = curc[idx] * (T)nu[s];
    row[S + s] = curb[idx] * (T)nu[S + s];
  }
}

template <typename T>
size_t carve_krylov(void* base, long long n, long long m, int k, int S, KView<T>* kv) {
  Carver c(base);
  const int grid = num_sms() * kGridPerSm;
  kv->n = (int)n;
  kv->m = (int)m;
  kv->S = S;
  kv->Yc = c.take<T>(n * S);
  kv->Bc[0] = c.take<T>(n * S);
  kv->Bc[1] = c.take<T>(n * S);
  kv->Yb = c.take<T>((n + m) * S);
  kv->Bb[0] = c.take<T>((n + m) * S);
  kv->Bb[1] = c.take<T>((n + m) * S);
  kv->se = c.take<T>((m > 0 ? m : 1) * S);
  kv->inv_nu = c.take<double>((size_t)(k + 1) * 2 * S);
  kv->coef = c.take<double>((size_t)(k + 1) * 2 * S * 4);
  kv->part_e = c.take<double>((size_t)grid * S * 4);
  kv->part_n = c.take<double>((size_t)grid * S * 8);
  kv->part_u = c.take<double>((size_t)grid * S * 2);
  kv->part_s = c.take<double>((size_t)grid * S * 3);
  kv->counter = c.take<unsigned int>(64);
  return c.bytes();
}

template <typename T>
hef_status run_krylov(const hef_incidence* inc, int k, int S, const double* x0c, const double* x0b,
                      void* Vv, long long ldv, void* ws, cudaStream_t st) {
  KView<T> kv;
  carve_krylov<T>(ws, inc->n, inc->m, k, S, &kv);
  int lgS = 0;
  while ((1 << lgS) < S) ++lgS;
  kv.lgS = lgS;
  kv.tol = sizeof(T) == 8 ? 1e-12 : 1e-5;
  T* V = static_cast<T*>(Vv);
  IncView g = view(inc);
  const long long n = inc->n, m = inc->m;
  HEF_CHECK_CUDA(cudaMemsetAsync(kv.counter, 0, 64 * sizeof(unsigned int), st));
  const int grid_s = stride_grid((2 * n + m) * S, kGridPerSm);
  HEF_LAUNCH("k_start_dots", st, k_start_dots<T><<<grid_s, kThreads, 0, st>>>(g, kv, x0c, x0b));
  HEF_LAUNCH("k_start_write", st, k_start_write<T><<<grid_s, kThreads, 0, st>>>(g, kv, x0c, x0b));
  HEF_CHECK_LAUNCH();
  const int grid_e = stride_grid((m > 0 ? m : 1) * S, kGridPerSm);
  const int grid_n = stride_grid(n * S, kGridPerSm);
  const int grid_u = stride_grid((2 * n + m) * S, kGridPerSm);
  for (int j = 1; j <= k; ++j) {
    HEF_LAUNCH("k_edge_pass", st, k_edge_pass<T><<<grid_e, kThreads, 0, st>>>(g, kv, j));
    HEF_LAUNCH("k_node_pass", st, k_node_pass<T><<<grid_n, kThreads, 0, st>>>(g, kv, j, grid_e, V, ldv));
    HEF_LAUNCH("k_update", st, k_update<T><<<grid_u, kThreads, 0, st>>>(g, kv, j));
    HEF_CHECK_LAUNCH();
  }
  HEF_LAUNCH("k_archive_last", st, k_archive_last<T><<<grid_n, kThreads, 0, st>>>(g, kv, k, V, ldv));
  HEF_CHECK_LAUNCH();
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
