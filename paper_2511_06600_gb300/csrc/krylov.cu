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
// Layout.  Both expansions' chain values of vertex v form one record
// [x_c(v) | x_b(v)] of 2S values (S starts each), so one gather per pin in
// the edge pass fetches the rows of both operators; the star rows of the
// hyperedges are a separate m x S block.  The edge pass leaves per hyperedge
// the record [wh_e s_e | z_e x_b(e)] (weighted and scaled), so the vertex pass
// sums one record per incidence.  Per step: an edge pass (thread per
// hyperedge; hyperedges with more than kBig pins are summed by their whole
// warp), a vertex pass (thread per vertex, same split), which also archives
// x_{j-1} into V (the vertex's record is the contiguous column block of the
// step) and reduces the Lanczos dots, and an update pass (thread per vertex
// record or star hyperedge row) forming x_j and its D-norm.  Every reduction
// is a per-CTA partial followed by a two-level fixed-order sum (grid_reduce).
#include <cuda_bf16.h>

#include <algorithm>
#include <memory>
#include <type_traits>
#include <utility>
#include <vector>

#include "internal.h"

namespace hef {

namespace {

constexpr int kMaxS = 16;
constexpr int kBig = 16;     // segments longer than this are summed by a warp
// rows per thread in the update pass (vertex records of 32 bytes or more
// take two, for registers)
template <typename T, int S>
__host__ __device__ constexpr int upd_rows() {
  return 2 * S * sizeof(T) >= 32 ? 2 : 4;
}
// records gathered per round by one thread in the segment sums (wider
// records keep two, for registers)
template <typename T, int N>
__host__ __device__ constexpr int gather_round() {
  return N * sizeof(T) <= 32 ? 4 : 2;
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
  T* Yv;     // n x 2S: [(M_c x)_v | (M_b x)_v]
  T* Bv[2];  // n x 2S: [u_c(v) | u_b(v)] of alternate steps
  T* Ye;     // m x S: (M_b x)_e
  T* Be[2];  // m x S: u_b(e) of alternate steps
  T* Er;     // m x 2S: [wh_e s_e | z_e x_b(e)] of the current step (scaled)
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
  double* ppart;   // persistent launch: partial sums (2 x grid x 9S; the timeout
                   // test's grid is 2 num_sms)
  unsigned int* pcount;  // persistent launch: kRelCopies arrival counters (4 KB apart)
  int capi, capl;  // persistent launch: vertices / hyperedges (capi) and incidences /
                   // pins (capl) whose offsets and index lists a CTA keeps in shared
                   // memory
  int capv;        // persistent launch: own vertices whose chain records (two steps)
                   // and Y rows a CTA keeps in shared memory (0: none)
};

// ---------------------------------------------------------------- row I/O

// a[i] for i in {0, 1} without indexing the array at run time (which would
// copy the kernel argument to local memory)
template <typename P>
__device__ __forceinline__ P pick2(P const (&a)[2], int i) {
  return i ? a[1] : a[0];
}

// Load through the read-only path (data written by earlier launches), or,
// with CG, through L2 only: coherent with writes of other CTAs of the same
// launch that a grid barrier has ordered before the load.
template <bool CG, typename V>
__device__ __forceinline__ V ld1(const V* p) {
  if constexpr (CG) return __ldcg(p);
  else return __ldg(p);
}

// One 32-byte access (the 256-bit loads and stores of sm_100 and later): a
// record that fills an L2 sector costs one request instead of two 16-byte
// ones.  p is 32-byte aligned.  The coherent (CG) loads and the stores are
// ordered with the grid barriers' memory operations like the plain accesses
// they replace.
template <bool CG>
__device__ __forceinline__ void ld32B(const float* p, float* v) {
  if constexpr (CG)
    asm volatile("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
                   "=f"(v[6]), "=f"(v[7])
                 : "l"(p)
                 : "memory");
  else
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
          "=f"(v[7])
        : "l"(p));
}
template <bool CG>
__device__ __forceinline__ void ld32B(const double* p, double* v) {
  if constexpr (CG)
    asm volatile("ld.global.cg.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
                 : "l"(p)
                 : "memory");
  else
    asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
        : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
        : "l"(p));
}
__device__ __forceinline__ void st32B(float* p, const float* v) {
  asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]), "f"(v[1]),
               "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}
__device__ __forceinline__ void st32B(double* p, const double* v) {
  asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(v[0]), "d"(v[1]), "d"(v[2]),
               "d"(v[3])
               : "memory");
}

__device__ __forceinline__ void st32B_cs(float* p, const float* v) {
  asm volatile("st.global.cs.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]),
               "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}
__device__ __forceinline__ void st32B_cs(double* p, const double* v) {
  asm volatile("st.global.cs.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(v[0]), "d"(v[1]),
               "d"(v[2]), "d"(v[3])
               : "memory");
}

// N contiguous values with the widest vector access the row size allows.
// Rows and records start at multiples of their own size from 256-byte aligned
// buffers, so a row of a multiple of 32 bytes is 32-byte aligned.
template <typename T, int N, bool CG = false>
__device__ __forceinline__ void ldrow(const T* __restrict__ p, T (&v)[N]) {
  if constexpr ((N * sizeof(T)) % 32 == 0) {
    constexpr int E = 32 / sizeof(T);
#pragma unroll
    for (int i = 0; i < N / E; ++i) ld32B<CG>(p + E * i, v + E * i);
  } else if constexpr (sizeof(T) == 4 && N % 4 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
      const float4 f = ld1<CG>(q + i);
      v[4 * i] = f.x, v[4 * i + 1] = f.y, v[4 * i + 2] = f.z, v[4 * i + 3] = f.w;
    }
  } else if constexpr (sizeof(T) == 4 && N % 2 == 0) {
    const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const float2 f = ld1<CG>(q + i);
      v[2 * i] = f.x, v[2 * i + 1] = f.y;
    }
  } else if constexpr (sizeof(T) == 8 && N % 2 == 0) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const double2 f = ld1<CG>(q + i);
      v[2 * i] = f.x, v[2 * i + 1] = f.y;
    }
  } else {
#pragma unroll
    for (int s = 0; s < N; ++s) v[s] = ld1<CG>(p + s);
  }
}

template <typename T, int N>
__device__ __forceinline__ void strow(T* __restrict__ p, const T (&v)[N]) {
  if constexpr ((N * sizeof(T)) % 32 == 0) {
    constexpr int E = 32 / sizeof(T);
#pragma unroll
    for (int i = 0; i < N / E; ++i) st32B(p + E * i, v + E * i);
  } else if constexpr (sizeof(T) == 4 && N % 4 == 0) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int i = 0; i < N / 4; ++i) q[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  } else if constexpr (sizeof(T) == 4 && N % 2 == 0) {
    float2* q = reinterpret_cast<float2*>(p);
#pragma unroll
    for (int i = 0; i < N / 2; ++i) q[i] = make_float2(v[2 * i], v[2 * i + 1]);
  } else if constexpr (sizeof(T) == 8 && N % 2 == 0) {
    double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
    for (int i = 0; i < N / 2; ++i) q[i] = make_double2(v[2 * i], v[2 * i + 1]);
  } else {
#pragma unroll
    for (int s = 0; s < N; ++s) p[s] = v[s];
  }
}

// Store with the streaming (evict-first) hint: the basis archive is written
// once per step and read only by the orthonormalisation, so it should not
// push the chain blocks out of L2.
template <typename T, int N>
__device__ __forceinline__ void strow_cs(T* __restrict__ p, const T (&v)[N]) {
  if constexpr (sizeof(T) == 4 && N % 4 == 0) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int i = 0; i < N / 4; ++i)
      __stcs(q + i, make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]));
  } else if constexpr (sizeof(T) == 4 && N % 2 == 0) {
    float2* q = reinterpret_cast<float2*>(p);
#pragma unroll
    for (int i = 0; i < N / 2; ++i) __stcs(q + i, make_float2(v[2 * i], v[2 * i + 1]));
  } else if constexpr (sizeof(T) == 8 && N % 2 == 0) {
    double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
    for (int i = 0; i < N / 2; ++i) __stcs(q + i, make_double2(v[2 * i], v[2 * i + 1]));
  } else {
#pragma unroll
    for (int s = 0; s < N; ++s) __stcs(p + s, v[s]);
  }
}

// Archive store of a record into a basis of storage type TV (the working
// type, or BF16 rounded to nearest).
template <typename T, int N, typename TV>
__device__ __forceinline__ void store_basis(TV* __restrict__ p, const T (&v)[N]) {
  if constexpr (std::is_same<T, TV>::value && (N * sizeof(T)) % 32 == 0) {
    // the caller's basis rows need only 16-byte alignment: 32-byte stores
    // where the record happens to be 32-byte aligned
    if ((reinterpret_cast<uintptr_t>(p) & 31) == 0) {
      constexpr int E = 32 / sizeof(T);
#pragma unroll
      for (int i = 0; i < N / E; ++i) st32B_cs(p + E * i, v + E * i);
    } else {
      strow_cs<T, N>(p, v);
    }
  } else if constexpr (std::is_same<T, TV>::value) {
    strow_cs<T, N>(p, v);
  } else if constexpr (N % 8 == 0) {
#pragma unroll
    for (int i = 0; i < N / 8; ++i) {
      __nv_bfloat162 h[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) h[q] = __floats2bfloat162_rn((float)v[8 * i + 2 * q], (float)v[8 * i + 2 * q + 1]);
      __stcs(reinterpret_cast<uint4*>(p) + i, *reinterpret_cast<const uint4*>(h));
    }
  } else if constexpr (N % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N / 2; ++i)
      reinterpret_cast<__nv_bfloat162*>(p)[i] = __floats2bfloat162_rn((float)v[2 * i], (float)v[2 * i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) p[i] = __float2bfloat16_rn((float)v[i]);
  }
}

// The halves of a record.
template <typename T, int S>
__device__ __forceinline__ void split2(const T (&r)[2 * S], T (&lo)[S], T (&hi)[S]) {
#pragma unroll
  for (int s = 0; s < S; ++s) lo[s] = r[s], hi[s] = r[S + s];
}

// Per-CTA partials of NQ*S values (slot q*S + s) written to part[block].
// Within a warp the values are summed by a transposing butterfly: at each
// level a lane keeps half of its values and adds its partner's copy of that
// half, so N values cost about N shuffles instead of 5 N; a lane ends with
// the warp sum of one slot.  Warps then meet in a fixed order, in the
// working type; only the CTA's sums are widened to FP64 (conversions and
// FP64 adds run at 1/64 rate on GB300).
// PMAX caps the butterfly width (values held at once) for register-tight callers.
// row: the partial's row in part (default: the CTA's index); with
// col_stride > 0 the partials are stored slot-major instead, value t at
// part[t * col_stride + row].
template <int NQ, int S, typename A, int NT = kThreads, int PMAX = 32, typename PT = double>
__device__ __forceinline__ void block_partials_qs(const A (&v)[NQ][S], PT* part, int row = -1,
                                                  int col_stride = 0) {
  constexpr int N = NQ * S;
  constexpr int P0 = N > 16 ? 32 : (N > 8 ? 16 : (N > 4 ? 8 : (N > 2 ? 4 : (N > 1 ? 2 : 1))));
  constexpr int P = P0 < PMAX ? P0 : PMAX;
  constexpr int R = 32 / P;  // lanes that end up holding the same slot
  constexpr int NCH = (N + P - 1) / P;
  __shared__ A red[NT / 32][NCH * P];
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
    const size_t r = (size_t)(row < 0 ? (int)blockIdx.x : row);
    part[col_stride > 0 ? (size_t)t * col_stride + r : r * N + t] = (PT)acc;
  }
}


// Sum of the N-value records row(idx(t)) over the entries t in [a, b) of an
// index list, split between one thread (short lists) and its whole warp
// (lists longer than kBig, handled one at a time).  A short list is gathered
// gather_round records per round, all index loads and then all record loads
// in flight (entries past the end repeat the last one and are not added).
// Each thread adds in entry order, so the sum does not depend on scheduling.
// Result in acc (the owner thread).
// idx values lie in [0, lim) (checked in the bounds-checked build, which
// reports a violation in `status`).
template <typename T, int N, bool CG, typename Idx, typename Row>
__device__ __forceinline__ void seg_gather(bool valid, int a, int b, Idx idx, Row row,
                                           T (&acc)[N], int lim, const unsigned int* status) {
  const int lane = threadIdx.x & 31;
  constexpr int kSeg = gather_round<T, N>();
#pragma unroll
  for (int i = 0; i < N; ++i) acc[i] = 0;
  const bool big = valid && (b - a) > kBig;
  if (valid && !big) {
    for (int t = a; t < b; t += kSeg) {
      int ii[kSeg];
#pragma unroll
      for (int q = 0; q < kSeg; ++q) ii[q] = dbg_index(idx(min(t + q, b - 1)), lim, status);
      T r[kSeg][N];
#pragma unroll
      for (int q = 0; q < kSeg; ++q) ldrow<T, N, CG>(row(ii[q]), r[q]);
#pragma unroll
      for (int q = 0; q < kSeg; ++q) {
        const bool in = t + q < b;
#pragma unroll
        for (int i = 0; i < N; ++i) acc[i] += in ? r[q][i] : (T)0;
      }
    }
  }
  unsigned bigmask = __ballot_sync(0xffffffffu, big);
  while (bigmask) {
    const int src = __ffs(bigmask) - 1;
    bigmask &= bigmask - 1;
    const int ba = __shfl_sync(0xffffffffu, a, src), bb = __shfl_sync(0xffffffffu, b, src);
    T part[N];
#pragma unroll
    for (int i = 0; i < N; ++i) part[i] = 0;
    // kSeg records per lane in flight: a 400-pin hyperedge takes 4 dependent
    // rounds instead of 13 (each lane still adds in entry order)
    for (int t0 = ba + lane; t0 < bb; t0 += 32 * kSeg) {
      T r[kSeg][N];
#pragma unroll
      for (int q = 0; q < kSeg; ++q) {
        const int t = min(t0 + 32 * q, bb - 1);
        ldrow<T, N, CG>(row(dbg_index(idx(t), lim, status)), r[q]);
      }
#pragma unroll
      for (int q = 0; q < kSeg; ++q) {
        const bool in = t0 + 32 * q < bb;
#pragma unroll
        for (int i = 0; i < N; ++i) part[i] += in ? r[q][i] : (T)0;
      }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part[i] += __shfl_xor_sync(0xffffffffu, part[i], o);
    }
    if (lane == src) {
#pragma unroll
      for (int i = 0; i < N; ++i) acc[i] = part[i];
    }
  }
}

// Records of the persistent kernel's own vertices in shared memory: the
// chain records u_{j-1}, u_{j-2} (x[0], x[1], alternating like Bv) and the Y
// rows of vertices [0, cap) of a CTA's range, so that the vertex and update
// passes read and write them without going through L2 (only u_j still goes
// to Bv, for the gathers).  Each record of N values is stored as 16-byte
// planes (plane p of record i at p * cap + i), so a warp's access to 32
// consecutive records of one plane reads 512 contiguous bytes.
template <typename T, int N>
struct OwnRows {
  T* x[2];
  T* y;
  int cap;
  static constexpr int kPlaneBytes = (N * sizeof(T)) % 16 == 0 ? 16 : (int)(N * sizeof(T));
  static constexpr int E = kPlaneBytes / (int)sizeof(T);  // values per plane
  __device__ __forceinline__ void ld(const T* base, int i, T (&v)[N]) const {
#pragma unroll
    for (int p = 0; p < N / E; ++p) {
      const T* q = base + ((size_t)p * cap + i) * E;
      if constexpr (kPlaneBytes == 16 && sizeof(T) == 4) {
        const float4 f = *reinterpret_cast<const float4*>(q);
        v[E * p] = f.x, v[E * p + 1] = f.y, v[E * p + 2] = f.z, v[E * p + 3] = f.w;
      } else if constexpr (kPlaneBytes == 16) {
        const double2 f = *reinterpret_cast<const double2*>(q);
        v[E * p] = f.x, v[E * p + 1] = f.y;
      } else {
#pragma unroll
        for (int t = 0; t < E; ++t) v[E * p + t] = q[t];
      }
    }
  }
  __device__ __forceinline__ void st(T* base, int i, const T (&v)[N]) const {
#pragma unroll
    for (int p = 0; p < N / E; ++p) {
      T* q = base + ((size_t)p * cap + i) * E;
      if constexpr (kPlaneBytes == 16 && sizeof(T) == 4) {
        *reinterpret_cast<float4*>(q) = make_float4(v[E * p], v[E * p + 1], v[E * p + 2], v[E * p + 3]);
      } else if constexpr (kPlaneBytes == 16) {
        *reinterpret_cast<double2*>(q) = make_double2(v[E * p], v[E * p + 1]);
      } else {
#pragma unroll
        for (int t = 0; t < E; ++t) q[t] = v[E * p + t];
      }
    }
  }
};

// ---------------------------------------------------------------- start vectors

// D-weighted dots of the raw starts with the trivial vectors -> coef[0]; the
// starts, in the working type (and the internal hyperedge order), go to the
// first chain buffers for k_start_write (one FP64 -> working-type conversion).
// Rows: [0, n) vertex records (clique and star), [n, n+m) star hyperedges.
template <typename T, int S>
__global__ void __launch_bounds__(kThreads) k_start_dots(IncView g, ScalView<T> sv, KView<T> kv,
                                                         const double* __restrict__ x0c,
                                                         const double* __restrict__ x0b) {
  if (g.status[0]) return;
  T acc[3][S];
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int s = 0; s < S; ++s) acc[q][s] = 0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < (long long)g.n + g.m;
       r += (long long)gridDim.x * blockDim.x) {
    if (r < g.n) {
      const T dc = sv.dc[r], db = sv.db[r];
      T u[2 * S];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        u[s] = (T)x0c[r * S + s], acc[0][s] += dc * u[s];
        u[S + s] = (T)x0b[r * S + s], acc[1][s] += db * u[S + s];
      }
      strow<T, 2 * S>(kv.Bv[0] + r * 2 * S, u);
    } else {
      const int i = (int)(r - g.n);
      const T d = sv.ew[i];
      const long long src = (long long)(g.n + g.perm[i]) * S;
      T u[S];
#pragma unroll
      for (int s = 0; s < S; ++s) u[s] = (T)x0b[src + s], acc[2][s] += d * u[s];
      strow<T, S>(kv.Be[0] + (long long)i * S, u);
    }
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
  T acc[2][S];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int s = 0; s < S; ++s) acc[q][s] = 0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < (long long)g.n + g.m;
       r += (long long)gridDim.x * blockDim.x) {
    if (r < g.n) {
      const T dc = sv.dc[r], db = sv.db[r];
      T u[2 * S];
      ldrow<T, 2 * S>(kv.Bv[0] + r * 2 * S, u);
#pragma unroll
      for (int s = 0; s < S; ++s) {
        u[s] -= (dc > 0 ? kv.cfT[(size_t)s * 4] : (T)0);
        acc[0][s] += dc * u[s] * u[s];
        u[S + s] -= (db > 0 ? kv.cfT[(size_t)(S + s) * 4] : (T)0);
        acc[1][s] += db * u[S + s] * u[S + s];
      }
      strow<T, 2 * S>(kv.Bv[0] + r * 2 * S, u);
      if (kv.tape_c) {
        T uc[S], ub[S];
        split2<T, S>(u, uc, ub);
        strow<T, S>(kv.tape_c + r * S, uc);
        strow<T, S>(kv.tape_b + r * S, ub);
      }
    } else {
      const long long i = r - g.n;  // star hyperedge row
      const T d = sv.ew[i];
      T u[S];
      ldrow<T, S>(kv.Be[0] + i * S, u);
#pragma unroll
      for (int s = 0; s < S; ++s) {
        u[s] -= (d > 0 ? kv.cfT[(size_t)(S + s) * 4 + 1] : (T)0);
        acc[1][s] += d * u[s] * u[s];
      }
      strow<T, S>(kv.Be[0] + i * S, u);
      if (kv.tape_b) strow<T, S>(kv.tape_b + (g.n + i) * S, u);
    }
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
// warp's collective sums): the clique pin sum s_e and star pin sum from one
// record gather per pin, the star row (M_b x)_e, the record
// [wh_e s_e | z_e x_b(e)] for the vertex pass, and the D-weighted dots of the
// star hyperedge rows, added to acc.
// ofs(e) gives the CSC offset of hyperedge e and pin(t) the vertex of CSC
// slot t; CG selects coherent loads of the chain data (see ldrow).
template <typename T, int S, bool CG, typename Ofs, typename Pin>
__device__ __forceinline__ void edge_item(const IncView& g, const ScalView<T>& sv,
                                          const KView<T>& kv, const T* nuT, int j, int e,
                                          T (&acc)[3][S], Ofs ofs, Pin pin) {
  const T* __restrict__ curv = pick2(kv.Bv, (j - 1) & 1);
  const T* __restrict__ cure = pick2(kv.Be, (j - 1) & 1);
  const T* __restrict__ prve = j >= 3 ? pick2(kv.Be, j & 1) : nullptr;
  const bool valid = e < g.m;
  int a = 0, b = 0;
  // the hyperedge's own rows and scalars first: their loads overlap the gathers
  T xc[S], xp[S];
  T we = 0, wh = 0, z = 0;
  if (valid) {
    a = ofs(e), b = ofs(e + 1);
    ldrow<T, S, CG>(cure + (long long)e * S, xc);
    if (prve) ldrow<T, S, CG>(prve + (long long)e * S, xp);
    we = sv.ew[e], wh = sv.ewh[e], z = sv.ez[e];
  }
  T sum[2 * S];
  seg_gather<T, 2 * S, CG>(valid, a, b, pin,
                           [&](int p) { return curv + (long long)p * 2 * S; }, sum, g.n, g.status);
  if (valid) {
    const int k = b - a;
    const T invk = k >= 2 ? (T)1 / (T)k : (T)0;
    // inverse norms of x_{j-1} (clique, star) and x_{j-2} (star)
    const T* __restrict__ n1 = nuT + (size_t)(j - 1) * 2 * S;
    const T* __restrict__ n2 = nuT + (size_t)(j >= 2 ? j - 2 : 0) * 2 * S;
    T ye[S], er[2 * S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const T ncc = n1[s], ncb = n1[S + s];
      ye[s] = sum[S + s] * ncb * invk;
      er[s] = wh * (sum[s] * ncc);
      er[S + s] = z * (xc[s] * ncb);
      if (k >= 2) {
        const T wy = we * ye[s];
        acc[0][s] += wy;
        acc[1][s] += wy * xc[s] * ncb;
        acc[2][s] += prve ? wy * xp[s] * n2[S + s] : (T)0;
      }
    }
    strow<T, S>(kv.Ye + (long long)e * S, ye);
    strow<T, 2 * S>(kv.Er + (long long)e * 2 * S, er);
  }
}

template <typename T>
__device__ __forceinline__ void edge_final(const KView<T>& kv, int S, const double* tot) {
  for (int t = threadIdx.x; t < 3 * S; t += blockDim.x) kv.te[t] = tot[t];
}

// Vertex pass item (vertex v): (M_c x)_v and (M_b x)_v from one record per
// incidence, archive of x_{j-1} into V (one contiguous record), and the dots
// of the Lanczos coefficients, added to acc.
// ofs(v) gives the offset of vertex v's incidences and edge(t) the hyperedge
// of incidence t; CG as in edge_item.
template <typename T, int S, bool CG, typename TV, typename Ofs, typename Edge>
__device__ __forceinline__ void node_item(const IncView& g, const ScalView<T>& sv,
                                          const KView<T>& kv, const T* nuT, int j, int v,
                                          T (&acc)[6][S], TV* __restrict__ V, long long ldv,
                                          Ofs ofs, Edge edge,
                                          OwnRows<T, 2 * S> own = {}, int si = -1) {
  const T* __restrict__ curv = pick2(kv.Bv, (j - 1) & 1);
  const T* __restrict__ prvv = j >= 3 ? pick2(kv.Bv, j & 1) : nullptr;
  const bool valid = v < g.n;
  int a = 0, b = 0;
  if (valid) a = ofs(v), b = ofs(v + 1);
  const T* __restrict__ er = kv.Er;
  // the vertex's own records and scalars first: their loads overlap the gathers
  T xr[2 * S], pr[2 * S];
  T wsum = 0, idc = 0, idb = 0, dcv = 0, dbv = 0;
  if (valid) {
    if (si >= 0) {
      own.ld(pick2(own.x, (j - 1) & 1), si, xr);
      if (prvv) own.ld(pick2(own.x, j & 1), si, pr);
    } else {
      ldrow<T, 2 * S, CG>(curv + (long long)v * 2 * S, xr);
      if (prvv) ldrow<T, 2 * S, CG>(prvv + (long long)v * 2 * S, pr);
    }
    wsum = sv.wsc[v], idc = sv.inv_dc[v], idb = sv.inv_db[v], dcv = sv.dc[v], dbv = sv.db[v];
  }
  T sum[2 * S];
  seg_gather<T, 2 * S, CG>(valid, a, b, edge,
                           [&](int e) { return er + (long long)e * 2 * S; }, sum, g.m, g.status);
  if (valid) {
    // inverse norms of x_{j-1} and x_{j-2} (both expansions)
    const T* __restrict__ n1 = nuT + (size_t)(j - 1) * 2 * S;
    const T* __restrict__ n2 = nuT + (size_t)(j >= 2 ? j - 2 : 0) * 2 * S;
    T y[2 * S], xo[2 * S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const T xv = xr[s] * n1[s];
      const T xb = xr[S + s] * n1[S + s];
      const T yc = idc * (sum[s] - wsum * xv);
      const T yb = idb * sum[S + s];
      const T pc = prvv ? pr[s] * n2[s] : (T)0;
      const T pb = prvv ? pr[S + s] * n2[S + s] : (T)0;
      acc[0][s] += dcv * yc;
      acc[1][s] += dcv * yc * xv;
      acc[2][s] += dcv * yc * pc;
      acc[3][s] += dbv * yb;
      acc[4][s] += dbv * yb * xb;
      acc[5][s] += dbv * yb * pb;
      y[s] = yc, y[S + s] = yb;
      xo[s] = xv, xo[S + s] = xb;
    }
    if (si >= 0) own.st(own.y, si, y);
    else strow<T, 2 * S>(kv.Yv + (long long)v * 2 * S, y);
    if (j >= 2)  // x_{j-1} is basis vector j-1 -> column block j-2
      store_basis<T, 2 * S, TV>(V + (long long)v * ldv + (long long)(j - 2) * 2 * S, xo);
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

// Update of one vertex record (both expansions) and of one star hyperedge
// row: u_j = y - trivial part - alpha x_{j-1} - beta x_{j-2} (written over
// x_{j-2}'s buffer) and its D-norm, added to acc.  cf[op][s][q] = [ct, ct2,
// alpha nu_{j-1}, beta nu_{j-2}] of step j (a register array, or a view of
// shared memory).
template <typename T, int S, bool CG, typename CF>
__device__ __forceinline__ void update_vertex(const IncView& g, const ScalView<T>& sv,
                                              const KView<T>& kv, int j, long long r,
                                              const CF& cf, T (&acc)[2][S],
                                              OwnRows<T, 2 * S> own = {}, int si = -1) {
  const bool has_prv = j >= 3;
  const T* cur = pick2(kv.Bv, (j - 1) & 1) + r * 2 * S;
  T* nw = pick2(kv.Bv, j & 1) + r * 2 * S;
  const T dc = sv.dc[r], db = sv.db[r];
  T y[2 * S], xc[2 * S], xp[2 * S], u[2 * S];
  if (si >= 0) {
    own.ld(own.y, si, y);
    own.ld(pick2(own.x, (j - 1) & 1), si, xc);
    if (has_prv) own.ld(pick2(own.x, j & 1), si, xp);
  } else {
    ldrow<T, 2 * S, CG>(kv.Yv + r * 2 * S, y);
    ldrow<T, 2 * S, CG>(cur, xc);
    if (has_prv) ldrow<T, 2 * S, CG>(nw, xp);
  }
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const T tc = dc > 0 ? cf[0][s][0] : (T)0;
    u[s] = y[s] - tc - cf[0][s][2] * xc[s] - (has_prv ? cf[0][s][3] * xp[s] : (T)0);
    acc[0][s] += dc * u[s] * u[s];
    const T tb = db > 0 ? cf[1][s][0] : (T)0;
    u[S + s] = y[S + s] - tb - cf[1][s][2] * xc[S + s] -
               (has_prv ? cf[1][s][3] * xp[S + s] : (T)0);
    acc[1][s] += db * u[S + s] * u[S + s];
  }
  strow<T, 2 * S>(nw, u);
  if (si >= 0) own.st(pick2(own.x, j & 1), si, u);
  if (kv.tape_c) {
    T uc[S], ub[S];
    split2<T, S>(u, uc, ub);
    strow<T, S>(kv.tape_c + ((long long)j * g.n + r) * S, uc);
    strow<T, S>(kv.tape_b + ((long long)j * (g.n + g.m) + r) * S, ub);
  }
}

template <typename T, int S, bool CG, typename CF>
__device__ __forceinline__ void update_edge(const IncView& g, const ScalView<T>& sv,
                                            const KView<T>& kv, int j, long long i,
                                            const CF& cf, T (&acc)[2][S]) {
  const bool has_prv = j >= 3;
  const T* cur = pick2(kv.Be, (j - 1) & 1) + i * S;
  T* nw = pick2(kv.Be, j & 1) + i * S;
  const T d = sv.ew[i];
  T y[S], xc[S], xp[S], u[S];
  ldrow<T, S, CG>(kv.Ye + i * S, y);
  ldrow<T, S, CG>(cur, xc);
  if (has_prv) ldrow<T, S, CG>(nw, xp);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const T t = d > 0 ? cf[1][s][1] : (T)0;
    u[s] = y[s] - t - cf[1][s][2] * xc[s] - (has_prv ? cf[1][s][3] * xp[s] : (T)0);
    acc[1][s] += d * u[s] * u[s];
  }
  strow<T, S>(nw, u);
  if (kv.tape_b) strow<T, S>(kv.tape_b + ((long long)j * (g.n + g.m) + g.n + i) * S, u);
}

// cf[op][s][q] read from coefficients in (shared) memory, the same indexing
// as a register array T[2][S][4].
template <typename T, int S>
struct CoefView {
  const T* p;  // cfT + j * 2S * 4
  struct Row {
    const T* p;
    __device__ T operator[](int q) const { return p[q]; }
  };
  struct Op {
    const T* p;
    __device__ Row operator[](int s) const { return Row{p + s * 4}; }
  };
  __device__ Op operator[](int op) const { return Op{p + op * S * 4}; }
};

template <typename T, int S>
__device__ __forceinline__ void load_coefs(const T* cfT, int j, T (&cf)[2][S][4]) {
#pragma unroll
  for (int op = 0; op < 2; ++op)
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int q = 0; q < 4; ++q) cf[op][s][q] = cfT[((size_t)j * 2 * S + op * S + s) * 4 + q];
}

// Update pass item (rows r0 + it * blockDim.x, it < upd_rows).  Rows: [0, n)
// vertex records, [n, n + m) star hyperedge rows.
template <typename T, int S>
__device__ __forceinline__ void update_item(const IncView& g, const ScalView<T>& sv,
                                            const KView<T>& kv, int j, long long r0,
                                            T (&acc)[2][S]) {
  T cf[2][S][4];
  load_coefs<T, S>(kv.cfT, j, cf);
  const long long nrows = (long long)g.n + g.m;
  constexpr int kUpdRows = upd_rows<T, S>();
#pragma unroll
  for (int it = 0; it < kUpdRows; ++it) {
    const long long r = r0 + (long long)it * blockDim.x;
    if (r >= nrows) break;
    if (r < g.n) update_vertex<T, S, false>(g, sv, kv, j, r, cf, acc);
    else update_edge<T, S, false>(g, sv, kv, j, r - g.n, cf, acc);
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
template <typename T, int S, bool CG, typename TV>
__device__ __forceinline__ void archive_item(const IncView& g, const KView<T>& kv, const T* nuT,
                                             int k, int v, TV* __restrict__ V, long long ldv) {
  if (v >= g.n) return;
  T x[2 * S];
  ldrow<T, 2 * S, CG>(pick2(kv.Bv, k & 1) + (long long)v * 2 * S, x);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    x[s] *= nuT[(size_t)k * 2 * S + s];
    x[S + s] *= nuT[(size_t)k * 2 * S + S + s];
  }
  store_basis<T, 2 * S, TV>(V + (long long)v * ldv + (long long)(k - 1) * 2 * S, x);
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
  edge_item<T, S, false>(g, sv, kv, kv.nuT, j, blockIdx.x * blockDim.x + threadIdx.x, acc,
                         [&](int e) { return g.ceptr[e]; },
                         [&](int t) { return __ldg(g.cpins + t); });
  block_partials_qs<3, S, T>(acc, kv.red.part);
  __shared__ double tot[3 * kMaxS];
  if (grid_reduce(kv.red, 3 * S, tot)) edge_final(kv, S, tot);
}

// Vertex pass of step j (thread per vertex); the final CTA forms the
// Lanczos coefficients.
template <typename T, int S, typename TV>
__global__ void __launch_bounds__(kThreads, kMinBlocks<T, S>(4))
    k_node_pass(IncView g, ScalView<T> sv, KView<T> kv, int j, TV* __restrict__ V, long long ldv) {
  pdl_wait();
  pdl_trigger();
  if (g.status[0]) return;
  T acc[6][S];
  zero_acc(acc);
  node_item<T, S, false, TV>(g, sv, kv, kv.nuT, j, blockIdx.x * blockDim.x + threadIdx.x, acc, V,
                             ldv,
                         [&](int v) { return g.vptr[v]; },
                         [&](int t) { return __ldg(g.vedge + t); });
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
template <typename T, int S, typename TV>
__global__ void __launch_bounds__(kThreads) k_archive_last(IncView g, KView<T> kv, int k,
                                                           TV* __restrict__ V, long long ldv) {
  pdl_wait();
  if (g.status[0]) return;
  archive_item<T, S, false, TV>(g, kv, kv.nuT, k, blockIdx.x * blockDim.x + threadIdx.x, V, ldv);
}

// ---------------------------------------------------------------- persistent form
//
// All k steps in one cooperative launch of one CTA per SM.  CTA b owns a
// contiguous range of vertices and one of hyperedges (internal order),
// balanced on incidences plus items, and keeps their offsets and index lists
// in shared memory for all k steps (entries past the capacity are read from
// global memory): after the first step a gather costs one dependent load
// instead of three.  The three phases of a step (edge, vertex, update) meet
// at grid barriers, each carrying its phase's reduction: every CTA writes its
// partial sums, and after the barrier every CTA sums all partials in the
// same fixed order (reduce_slots), so every CTA holds the same coefficients
// and no CTA runs a serial final step.  Chain data written during the launch
// is read through L2 only (ldrow with CG), which the barriers order.

constexpr unsigned int kBarIters = 1u << 21;  // bounded barrier wait (polls of an L2 line: about 1 s)
constexpr int kCapItems = 4096;               // vertices / hyperedges cached per CTA
constexpr long long kPersistentMinRows = 32768;  // n + m from which the persistent form runs
constexpr int kCapList = 12288;               // incidences / pins cached per CTA
constexpr int kPartSlots = 9;                 // reduction slots per start (see part_buffer)

// Threads of the persistent CTA: 128 registers a thread (the fused phases
// spill at 64) for records of up to 32 bytes, 255 for wider records.
template <typename T, int S>
__host__ __device__ constexpr int pers_threads() {
  return 2 * S * sizeof(T) <= 32 ? 512 : 256;
}

// In one CTA of NT threads: out[slot] = sum over b < nb of part[slot * nb + b]
// (slot-major partials) for slot < N.  Warp w takes slots w, w + NT / 32,
// ... (up to four at a time): lane l loads partials l, l + 32, ... of each
// (every load issued before the adds: one round trip to L2 for up to 256
// partials and 4 NT / 32 slots), adds its eight in a fixed pairwise tree,
// then the lanes combine by a butterfly and lane 0's sum is kept: a fixed
// order for given nb.  DF (FP32 partials, P = float): the sums run in
// double-float arithmetic, since FP64 operations and conversions are slow on
// this part (a warp-wide FP64 add costs tens of issue cycles); otherwise in
// FP64 (P = double).
// Ends with __syncthreads (out may be shared memory).
// reduce_slot_range: the same sums for slots [s_begin, s_end) by the nw warps
// from warp w_first (the others return at once); each slot's result depends
// only on its partials, not on which warp sums it.  No barrier at the end.
template <int NT, bool DF, typename P>
__device__ __forceinline__ void reduce_slot_range(const P* part, int nb, int s_begin, int s_end,
                                                  double* out, int w_first, int nw) {
  constexpr int kI = DF ? 4 : 1;  // slots of a warp per round
  const int lane = threadIdx.x & 31, w = (int)(threadIdx.x >> 5) - w_first;
  if (w < 0 || w >= nw) return;
  const int kW = nw;
  const int N = s_end;
  for (int s0 = s_begin + w; s0 < N; s0 += kI * kW) {
    P x[kI][8];
    DFloat da[kI];
    double acc[kI];
#pragma unroll
    for (int i = 0; i < kI; ++i) da[i] = {0.f, 0.f}, acc[i] = 0.0;
    for (int b0 = 0; b0 < nb; b0 += 256) {
#pragma unroll
      for (int i = 0; i < kI; ++i)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int bb = b0 + lane + 32 * q, slot = s0 + i * kW;
          x[i][q] = bb < nb && slot < N ? __ldcg(part + (size_t)slot * nb + bb) : (P)0;
        }
#pragma unroll
      for (int i = 0; i < kI; ++i) {
        if (DF) {
          DFloat y[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) y[q] = {(float)x[i][q], 0.f};  // exact: P is float
          da[i] = df_add(da[i], df_add(df_add(df_add(y[0], y[1]), df_add(y[2], y[3])),
                                       df_add(df_add(y[4], y[5]), df_add(y[6], y[7]))));
        } else {
          acc[i] += ((x[i][0] + x[i][1]) + (x[i][2] + x[i][3])) + ((x[i][4] + x[i][5]) + (x[i][6] + x[i][7]));
        }
      }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
      for (int i = 0; i < kI; ++i) {
        if (DF) {
          const DFloat p{__shfl_xor_sync(0xffffffffu, da[i].hi, o), __shfl_xor_sync(0xffffffffu, da[i].lo, o)};
          da[i] = df_add(da[i], p);
        } else {
          acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
        }
      }
#pragma unroll
    for (int i = 0; i < kI; ++i)
      if (lane == 0 && s0 + i * kW < N) out[s0 + i * kW] = DF ? (double)da[i].hi + (double)da[i].lo : acc[i];
  }
}
template <int NT, bool DF, typename P>
__device__ __forceinline__ void reduce_slots_wide(const P* part, int nb, int N, double* out) {
  reduce_slot_range<NT, DF, P>(part, nb, 0, N, out, 0, NT / 32);
  __syncthreads();
}

// Dynamic shared memory of the persistent kernel.
// Layout: the vertex and edge lists (capi + 1 offsets and capl entries each),
// then inv_nu, the reduction results, itot (FP64), cfT and nuT (working
// type).  The lists take what the balanced ranges need (the rest of the SM's
// storage stays L1); entries past their capacity are read from global memory.
__host__ __device__ inline size_t list_bytes(int capi, int capl) {
  return ((size_t)2 * (capi + 1 + capl) * sizeof(int) + 15) / 16 * 16;
}
template <typename T>
__host__ __device__ inline size_t pers_smem(int k, int S, int capi, int capl) {
  const size_t nc = (size_t)(k + 1) * 2 * S;
  size_t b = list_bytes(capi, capl);
  b += nc * sizeof(double);                                            // inv_nu
  b += (size_t)(kPartSlots + 1) * S * sizeof(double) + 4 * sizeof(double);  // red, spare, itot
  b += nc * 4 * sizeof(T) + nc * sizeof(T);                            // cfT, nuT
  return (b + 15) / 16 * 16;
}

// Smallest x in [0, hi] with key(x) >= t (key non-decreasing, key(hi) >= t),
// by one warp: 32 probes per round.
template <typename Key>
__device__ __forceinline__ int warp_lower_bound(int hi, long long t, Key key) {
  const int lane = threadIdx.x & 31;
  int lo = 0;
  while (hi - lo > 32) {
    const int step = (hi - lo + 31) / 32;
    const int x = min(lo + step * (lane + 1), hi);
    const unsigned mask = __ballot_sync(0xffffffffu, key(x) >= t);
    const int f = __ffs(mask) - 1;  // lane 31 probes hi, so f >= 0
    const int nhi = min(lo + step * (f + 1), hi);
    lo = f == 0 ? lo : lo + step * f + 1;
    hi = nhi;
  }
  const int x = lo + lane;
  const unsigned mask = __ballot_sync(0xffffffffu, x <= hi && key(min(x, hi)) >= t);
  return lo + __ffs(mask) - 1;
}

__device__ __forceinline__ bool stopped(const unsigned int* status) {
  return *reinterpret_cast<const volatile unsigned int*>(status) != 0u;
}

// Barrier scratch layout.  The time of a grid barrier depended on where its
// few hot lines landed (about 2 us per barrier between two placements 4 KB
// apart), so the arrival counter exists in kRelCopies copies 4 KB apart:
// every CTA adds to all of them and CTA c polls copy c mod kRelCopies.
constexpr int kRelCopies = 4;
constexpr int kRelStride = 1024;  // uint32 words between copies (4 KB)
__host__ __device__ inline size_t flag_words(int /*Gmax*/) { return (size_t)kRelCopies * kRelStride; }

// Grid barrier number `ph`.  Every CTA, after its partial sums are written,
// adds 1 with release semantics to each of the kRelCopies arrival counters
// (4 KB apart); thread 0 of CTA b polls copy b mod kRelCopies with relaxed
// loads until all G CTAs of barrier ph have arrived (G (ph + 1) arrivals),
// then an acquire fence orders the partials' reads after the arrivals.  The
// counters rise monotonically within a launch (zeroed before it), and a copy
// first reaches G (ph + 1) only when every CTA has arrived at barrier ph (no
// CTA adds for ph + 1 before it has passed ph).  Every wait is bounded; on
// expiry HEF_WAIT_TIMEOUT is set in the status word.  Returns false when the
// launch must stop.
__device__ __forceinline__ void red_release_add(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned int ld_relaxed(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// `work` runs in warps 1.. while thread 0 waits (work that needs no result of
// this barrier).
template <typename Work>
__device__ __forceinline__ bool grid_arrive_wait(int ph, unsigned int* flags, unsigned int* status,
                                                 int b, int G, Work work) {
  __shared__ int go;
  __syncthreads();
  const unsigned int want = (unsigned int)G * (unsigned int)(ph + 1);
  if (threadIdx.x < kRelCopies) red_release_add(flags + (size_t)threadIdx.x * kRelStride, 1u);
  if (threadIdx.x == 0) {
    const unsigned int* mine = flags + (size_t)(b % kRelCopies) * kRelStride;
    unsigned int it = 0;
    int ok = 1;
    while (ld_relaxed(mine) < want) {
      if (++it > kBarIters) {
        atomicOr(status, HEF_WAIT_TIMEOUT);
        ok = 0;
        break;
      }
      if ((it & 255u) == 0u && stopped(status)) {
        ok = 0;
        break;
      }
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    go = ok;
  } else if (threadIdx.x >= 32) {
    work();
  }
  __syncthreads();
  return go != 0;
}
__device__ __forceinline__ bool grid_arrive_wait(int ph, unsigned int* flags, unsigned int* status,
                                                 int b, int G) {
  return grid_arrive_wait(ph, flags, status, b, G, [] {});
}

// Partial-sum buffers of the persistent kernel: two buffers (barriers
// alternate) of kPartSlots S slots by G CTAs, slot-major.  The vertex
// barrier's buffer holds the vertex dots in slots [0, 6S) and the edge
// pass's star-row dots in [6S, 9S): the edge barrier only synchronises, and
// the vertex barrier reduces both (kPartSlots is defined with the
// persistent kernel's shared-memory layout).
template <typename T>
__device__ __forceinline__ T* part_buffer(double* part, int ph, int G, int S) {
  return reinterpret_cast<T*>(part + (size_t)(ph & 1) * G * kPartSlots * S);
}

// Grid barrier `ph` carrying a reduction: the CTA's partial sums of acc go to
// slots [0, NQ S) of barrier ph's buffer, and after the barrier every CTA
// sums slots [0, nred) of all CTAs in the same fixed order
// (reduce_slots_wide) into `out` (shared memory): every CTA obtains the same
// bits, and no CTA publishes results for the others (one L2 round trip fewer
// on the critical path).  Two buffers suffice: a buffer's slots are written
// again only for barrier ph + 2, and no CTA writes them before every CTA has
// arrived at barrier ph + 1, that is, has finished reading barrier ph's
// partials (the edge pass's early writes to slots [6S, 9S) of barrier ph + 2's
// buffer do not overlap the slots [0, 2S) that the update barrier ph reads).
template <int NQ, int S, int NT, typename T>
__device__ __forceinline__ bool pbarrier(const T (&acc)[NQ][S], double* part, int ph, int nred,
                                         unsigned int* flags, unsigned int* status, double* out,
                                         int b, int G) {
  // FP32 forms: FP32 partials (their values are FP32 sums), reduced in
  // double-float arithmetic
  T* pbuf = part_buffer<T>(part, ph, G, S);
  block_partials_qs<NQ, S, T, NT, 8, T>(acc, pbuf, b, G);
  if (!grid_arrive_wait(ph, flags, status, b, G)) return false;
  reduce_slots_wide<NT, sizeof(T) == 4, T>(pbuf, G, nred, out);
  return true;
}

template <typename T, int S, typename TV>
__device__ __forceinline__ void krylov_body(const IncView& g, const ScalView<T>& sv,
                                            const KView<T>& kv, int k, TV* __restrict__ V,
                                            long long ldv, double* part, unsigned int* cnt,
                                            unsigned int* status, const int b, const int G) {
  constexpr int NT = pers_threads<T, S>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nc = (k + 1) * 2 * S;
  int* lv_ofs = reinterpret_cast<int*>(smem_raw);
  const int capi = kv.capi, capl = kv.capl;
  int* lv_edge = lv_ofs + capi + 1;
  int* le_ofs = lv_edge + capl;
  int* le_pin = le_ofs + capi + 1;
  double* s_inv_nu = reinterpret_cast<double*>(smem_raw + list_bytes(capi, capl));
  double* s_red = s_inv_nu + nc;    // reduction results (kPartSlots S)
  double* s_te = s_red + 6 * S;     // the star hyperedge-row dots of the step
  double* s_itot = s_red + (kPartSlots + 1) * S;
  T* s_cfT = reinterpret_cast<T*>(s_itot + 4);
  T* s_nuT = s_cfT + (size_t)nc * 4;
  __shared__ int rng[4];

  if (stopped(status)) return;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // this CTA's ranges: boundaries at b/G of the weights (incidences + items)
  if (wid < 4) {
    const bool vtx = wid < 2;
    const int bb = b + (wid & 1);
    const long long W = vtx ? (long long)g.vptr[g.n] + g.n : (long long)g.ceptr[g.m] + g.m;
    const long long t = bb >= G ? W : W * bb / G;
    const int x = vtx ? warp_lower_bound(g.n, t, [&](int v) { return (long long)__ldg(g.vptr + v) + v; })
                      : warp_lower_bound(g.m, t, [&](int e) { return (long long)__ldg(g.ceptr + e) + e; });
    if (lane == 0) rng[wid] = x;
  }
  for (int c = tid; c < nc; c += NT) {
    s_inv_nu[c] = kv.inv_nu[c];
    s_nuT[c] = kv.nuT[c];
  }
  if (tid < 3) s_itot[tid] = kv.itot[tid];
  __syncthreads();
  const int v0 = rng[0], v1 = rng[1], e0 = rng[2], e1 = rng[3];
  const int i0 = g.vptr[v0], p0 = g.ceptr[e0];
  const int nv = min(v1 - v0, capi), ne = min(e1 - e0, capi);
  const int ni = min(g.vptr[v1] - i0, capl), np = min(g.ceptr[e1] - p0, capl);
  for (int i = tid; i <= nv; i += NT) lv_ofs[i] = __ldg(g.vptr + v0 + i);
  for (int i = tid; i < ni; i += NT) lv_edge[i] = __ldg(g.vedge + i0 + i);
  for (int i = tid; i <= ne; i += NT) le_ofs[i] = __ldg(g.ceptr + e0 + i);
  for (int i = tid; i < np; i += NT) le_pin[i] = __ldg(g.cpins + p0 + i);
  // own vertices [v0, v0 + nown): chain records and Y rows in shared memory,
  // starting from x_0 (written by the start kernels)
  OwnRows<T, 2 * S> own;
  own.cap = kv.capv;
  own.x[0] = reinterpret_cast<T*>(smem_raw + pers_smem<T>(k, S, capi, capl));
  own.x[1] = own.x[0] + (size_t)own.cap * 2 * S;
  own.y = own.x[1] + (size_t)own.cap * 2 * S;
  const int nown = min(v1 - v0, own.cap);
  for (int i = tid; i < nown; i += NT) {
    T r[2 * S];
    ldrow<T, 2 * S, true>(kv.Bv[0] + (long long)(v0 + i) * 2 * S, r);
    own.st(own.x[0], i, r);
  }
  __syncthreads();
  auto vofs = [&](int v) { const int i = v - v0; return i <= nv ? lv_ofs[i] : __ldg(g.vptr + v); };
  auto vedg = [&](int t) { const int i = t - i0; return i < ni ? lv_edge[i] : __ldg(g.vedge + t); };
  auto eofs = [&](int e) { const int i = e - e0; return i <= ne ? le_ofs[i] : __ldg(g.ceptr + e); };
  auto epin = [&](int t) { const int i = t - p0; return i < np ? le_pin[i] : __ldg(g.cpins + t); };

  int ph = 0;
  for (int j = 1; j <= k; ++j) {
    {  // edge phase; its star-row dots are reduced at the vertex barrier
      T acc[3][S];
      zero_acc(acc);
      for (int base = e0 + wid * 32; base < e1; base += NT) {
        const int e = base + lane;
        edge_item<T, S, true>(g, sv, kv, s_nuT, j, e < e1 ? e : g.m, acc, eofs, epin);
      }
      block_partials_qs<3, S, T, NT, 8, T>(acc, part_buffer<T>(part, ph + 1, G, S) + (size_t)6 * S * G,
                                           b, G);
      if (!grid_arrive_wait(ph++, cnt, status, b, G)) return;
    }
    {  // vertex phase; then the Lanczos coefficients of step j
      T acc[6][S];
      zero_acc(acc);
      for (int base = v0 + wid * 32; base < v1; base += NT) {
        const int v = base + lane;
        node_item<T, S, true, TV>(g, sv, kv, s_nuT, j, v < v1 ? v : g.n, acc, V, ldv, vofs, vedg,
                                  own, v < v1 && v - v0 < nown ? v - v0 : -1);
      }
      // the vertex barrier: while thread 0 waits, warps 1.. sum the edge
      // pass's slots [6S, 9S) (complete since the edge barrier); then all
      // warps sum the vertex slots [0, 6S)
      T* pbuf = part_buffer<T>(part, ph, G, S);
      block_partials_qs<6, S, T, NT, 8, T>(acc, pbuf, b, G);
      if (!grid_arrive_wait(ph++, cnt, status, b, G, [&] {
            reduce_slot_range<NT, sizeof(T) == 4, T>(pbuf, G, 6 * S, kPartSlots * S, s_red, 1,
                                                    NT / 32 - 1);
          }))
        return;
      reduce_slots_wide<NT, sizeof(T) == 4, T>(pbuf, G, 6 * S, s_red);
      for (int c = tid; c < 2 * S; c += NT) {
        const int op = c / S, q = c % S;
        double cf[4];
        if (op == 0) {
          cf[0] = s_red[0 * S + q] * s_itot[0];
          cf[1] = 0.0;
          cf[2] = j >= 2 ? s_red[1 * S + q] : 0.0;
          cf[3] = j >= 3 ? s_red[2 * S + q] : 0.0;
        } else {
          cf[0] = s_red[3 * S + q] * s_itot[1];
          cf[1] = s_te[0 * S + q] * s_itot[2];
          cf[2] = j >= 2 ? s_red[4 * S + q] + s_te[1 * S + q] : 0.0;
          cf[3] = j >= 3 ? s_red[5 * S + q] + s_te[2 * S + q] : 0.0;
        }
        T* ct = s_cfT + ((size_t)j * 2 * S + c) * 4;
        ct[0] = (T)cf[0];
        ct[1] = (T)cf[1];
        ct[2] = (T)(cf[2] * s_inv_nu[(size_t)(j - 1) * 2 * S + c]);
        ct[3] = j >= 3 ? (T)(cf[3] * s_inv_nu[(size_t)(j - 2) * 2 * S + c]) : (T)0;
        if (b == 0) {  // one copy in global memory for the tape and the backward
          double* gc = kv.coef + ((size_t)j * 2 * S + c) * 4;
          T* gt = kv.cfT + ((size_t)j * 2 * S + c) * 4;
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) gc[q4] = cf[q4], gt[q4] = ct[q4];
        }
      }
      __syncthreads();
    }
    {  // update phase; then the inverse norms of step j
      const CoefView<T, S> cf{s_cfT + (size_t)j * 2 * S * 4};
      T acc[2][S];
      zero_acc(acc);
      for (int v = v0 + tid; v < v1; v += NT)
        update_vertex<T, S, true>(g, sv, kv, j, v, cf, acc, own, v - v0 < nown ? v - v0 : -1);
      for (int e = e0 + tid; e < e1; e += NT) update_edge<T, S, true>(g, sv, kv, j, e, cf, acc);
      if (!pbarrier<2, S, NT>(acc, part, ph++, 2 * S, cnt, status, s_red, b, G)) return;
      for (int c = tid; c < 2 * S; c += NT) {
        const double nu2 = s_red[c];
        const bool alive = s_inv_nu[(size_t)(j - 1) * 2 * S + c] > 0.0 && nu2 > kv.tol * kv.tol;
        const double inu = alive ? rsqrt(nu2) : 0.0;
        s_inv_nu[(size_t)j * 2 * S + c] = inu;
        s_nuT[(size_t)j * 2 * S + c] = (T)inu;
        if (b == 0) kv.inv_nu[(size_t)j * 2 * S + c] = inu, kv.nuT[(size_t)j * 2 * S + c] = (T)inu;
      }
      __syncthreads();
    }
  }
  for (int v = v0 + tid; v < v1; v += NT) archive_item<T, S, true, TV>(g, kv, s_nuT, k, v, V, ldv);
}

template <typename T, int S, typename TV>
__global__ void __launch_bounds__(pers_threads<T, S>(), 1)
    k_krylov_steps(IncView g, ScalView<T> sv, KView<T> kv, int k, TV* __restrict__ V,
                   long long ldv, double* part, unsigned int* cnt, unsigned int* status) {
  krylov_body<T, S, TV>(g, sv, kv, k, V, ldv, part, cnt, status, (int)blockIdx.x, (int)gridDim.x);
}

// Many hypergraphs in one cooperative launch (the batched form): hypergraph
// i owns CTAs [cta0[i], cta0[i+1]) and runs the persistent form on them with
// its own barriers and partials; the table travels as the kernel parameter.
constexpr int kBatchItems = 64;  // hypergraphs per launch (parameter space)
template <typename T, typename TV>
struct KBatchItem {
  IncView g;
  ScalView<T> sv;
  KView<T> kv;
  TV* V;
  long long ldv;
  unsigned int* status;
};
template <typename T, typename TV>
struct KBatch {
  int nitems, k;
  int cta0[kBatchItems + 1];
  KBatchItem<T, TV> it[kBatchItems];
};

template <typename T, int S, typename TV>
__global__ void __launch_bounds__(pers_threads<T, S>(), 1)
    k_krylov_batched(const __grid_constant__ KBatch<T, TV> bt) {
  int i = 0;
  while (i + 1 < bt.nitems && (int)blockIdx.x >= bt.cta0[i + 1]) ++i;
  const KBatchItem<T, TV>& it = bt.it[i];
  krylov_body<T, S, TV>(it.g, it.sv, it.kv, bt.k, it.V, it.ldv, it.kv.ppart, it.kv.pcount,
                        it.status, (int)blockIdx.x - bt.cta0[i], bt.cta0[i + 1] - bt.cta0[i]);
}

inline int blocks_for(long long rows) { return (int)((rows + kThreads - 1) / kThreads); }

template <typename T>
size_t carve_krylov(void* base, long long n, long long m, int k, int S, KView<T>* kv) {
  Carver c(base);
  const long long maxblk = blocks_for(2 * n + m);
  const long long me = m > 0 ? m : 1;
  kv->n = (int)n;
  kv->m = (int)m;
  kv->Yv = c.take<T>(n * 2 * S);
  kv->Bv[0] = c.take<T>(n * 2 * S);
  kv->Bv[1] = c.take<T>(n * 2 * S);
  kv->Ye = c.take<T>(me * S);
  kv->Be[0] = c.take<T>(me * S);
  kv->Be[1] = c.take<T>(me * S);
  kv->Er = c.take<T>(me * 2 * S);
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
  kv->ppart = c.take<double>((size_t)2 * num_sms() * 2 * kPartSlots * S);
  kv->pcount = c.take<unsigned int>(flag_words(2 * num_sms()));
  kv->capi = kCapItems;
  kv->capl = kCapList;
  kv->capv = 0;
  return c.bytes();
}

// Whether the one-launch form may be used by calls from this thread (the
// batched form, whose hypergraphs share the GPU, turns it off).
thread_local bool t_persistent = true;
// Test of the timeout path: launch the persistent form with twice the
// resident grid, so that its first barrier cannot complete.
thread_local bool t_force_oversized = false;

// The deflated starts x_0 and their norms (the first two launches of every form).
template <typename T, int S>
hef_status krylov_start_s(const hef_incidence* inc, const double* x0c, const double* x0b,
                          const KView<T>& kv, cudaStream_t st) {
  IncView g = view(inc);
  const ScalView<T> sv = scal_view<T>(inc);
  // grid-stride rows: few CTAs, so few partials and grid-reduction arrivals
  const int grid_all = std::min(blocks_for(inc->n + inc->m), 4 * num_sms());
  HEF_LAUNCH("k_start_dots", st, k_start_dots<T, S><<<grid_all, kThreads, 0, st>>>(g, sv, kv, x0c, x0b));
  // the launches after the first are programmatically dependent on their
  // predecessor (each kernel waits for it before touching shared buffers)
  HEF_LAUNCH("k_start_write", st,
             HEF_CHECK_CUDA(launch_dependent(k_start_write<T, S>, grid_all, kThreads, st, g, sv, kv)));
  HEF_CHECK_LAUNCH();
  return HEF_OK;
}

template <typename T, int S, typename TV>
hef_status run_krylov_s(const hef_incidence* inc, int k, const double* x0c, const double* x0b,
                        TV* V, long long ldv, KView<T>& kv, bool persistent, cudaStream_t st) {
  IncView g = view(inc);
  const ScalView<T> sv = scal_view<T>(inc);
  const long long n = inc->n, m = inc->m;
  const int grid_e = blocks_for(m > 0 ? m : 1);
  const int grid_n = blocks_for(n);
  const int grid_upd = blocks_for((n + m + upd_rows<T, S>() - 1) / upd_rows<T, S>());
  if (hef_status s0 = krylov_start_s<T, S>(inc, x0c, x0b, kv, st)) return s0;
  // all steps as one cooperative launch of one CTA per SM (see
  // k_krylov_steps) unless this thread's calls share the GPU with other work
  // (the batched form); if the runtime refuses the grid, three launches per
  // step run instead
  // (small hypergraphs: the per-step launches are as fast as the barriers)
  if (persistent && (n + m >= kPersistentMinRows || t_force_oversized)) {
    constexpr int NT = pers_threads<T, S>();
    constexpr size_t kSmemLimit = 227 * 1024;  // per-CTA opt-in limit of the sm_100 family
    // list capacities: 1.25 times the average range (the balanced ranges
    // stay within a few per cent of it), at most kCapItems / kCapList
    const double G = (double)num_sms();
    kv.capi = (int)std::min<double>(kCapItems, 1.25 * (double)std::max(n, m) / G + 64.0);
    kv.capl = (int)std::min<double>(kCapList, 1.25 * (double)inc->P / G + 256.0);
    size_t smem = pers_smem<T>(k, S, kv.capi, kv.capl);
    kv.capv = 0;
    if (smem <= kSmemLimit) {
      // own vertices' chain records (two steps) and Y rows in shared memory:
      // room for 1.1 times the average vertex range, within the limit
      static thread_local int stat = -1;  // static shared bytes of this instantiation
      if (stat < 0) {
        cudaFuncAttributes fa;
        HEF_CHECK_CUDA(cudaFuncGetAttributes(&fa, k_krylov_steps<T, S, TV>));
        stat = (int)fa.sharedSizeBytes;
      }
      const size_t used = smem + (size_t)stat + 1024;
      const size_t per_v = (size_t)3 * 2 * S * sizeof(T);
      const size_t fit = used < kSmemLimit ? (kSmemLimit - used) / per_v : 0;
      kv.capv = (int)std::min<double>((double)fit, 1.1 * (double)n / G + 64.0) & ~1;
      smem += (size_t)kv.capv * per_v;
      HEF_ENSURE_SMEM((k_krylov_steps<T, S, TV>), smem);
    }
    int occ = 0;
    if (smem <= kSmemLimit &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_krylov_steps<T, S, TV>, NT, smem) ==
            cudaSuccess &&
        occ >= 1) {
      HEF_CHECK_CUDA(cudaMemsetAsync(kv.pcount, 0, flag_words(2 * num_sms()) * sizeof(unsigned int), st));
      // the timeout test launches twice the resident grid as a plain launch,
      // so that the first barrier cannot complete and its bounded wait runs out
      const int grid = num_sms() * (t_force_oversized ? 2 : 1);
      cudaError_t e = cudaSuccess;
      if (t_force_oversized) {
        HEF_LAUNCH("k_krylov_steps", st,
                   k_krylov_steps<T, S, TV><<<grid, NT, smem, st>>>(g, sv, kv, k, V, ldv, kv.ppart,
                                                               kv.pcount, inc->status));
        e = cudaGetLastError();
      } else {
        HEF_LAUNCH("k_krylov_steps", st,
                   e = launch_cooperative_smem(k_krylov_steps<T, S, TV>, grid, NT, smem, st, g, sv,
                                               kv, k, V, ldv, kv.ppart, kv.pcount, inc->status));
      }
      if (e == cudaSuccess) return HEF_OK;
      if (e != cudaErrorCooperativeLaunchTooLarge && e != cudaErrorNotSupported)
        return set_error(HEF_ERR_CUDA, "k_krylov_steps: %s", cudaGetErrorString(e));
      (void)cudaGetLastError();
    } else {
      (void)cudaGetLastError();
    }
  }
  for (int j = 1; j <= k; ++j) {
    HEF_LAUNCH("k_edge_pass", st,
               HEF_CHECK_CUDA(launch_dependent(k_edge_pass<T, S>, grid_e, kThreads, st, g, sv, kv, j)));
    HEF_LAUNCH("k_node_pass", st,
               HEF_CHECK_CUDA(launch_dependent(k_node_pass<T, S, TV>, grid_n, kThreads, st, g, sv, kv,
                                               j, V, ldv)));
    HEF_LAUNCH("k_update", st,
               HEF_CHECK_CUDA(launch_dependent(k_update<T, S>, grid_upd, kThreads, st, g, sv, kv, j)));
    HEF_CHECK_LAUNCH();
  }
  HEF_LAUNCH("k_archive_last", st,
             HEF_CHECK_CUDA(launch_dependent(k_archive_last<T, S, TV>, grid_n, kThreads, st, g, kv, k,
                                             V, ldv)));
  HEF_CHECK_LAUNCH();
  return HEF_OK;
}

// The Krylov workspace's view (no tape) with its reduction counters zeroed.
template <typename T>
hef_status krylov_view(const hef_incidence* inc, int k, int S, void* ws, void* tape, KView<T>* kv,
                       TapeLayout* tl, cudaStream_t st) {
  carve_krylov<T>(ws, inc->n, inc->m, k, S, kv);
  carve_tape(tape, inc->n, inc->m, k, S, sizeof(T), tl);
  kv->tape_c = static_cast<T*>(tl->uc);
  kv->tape_b = static_cast<T*>(tl->ub);
  kv->tol = sizeof(T) == 8 ? 1e-12 : 1e-5;
  const int ngr = red_groups(blocks_for(2 * inc->n + inc->m));
  HEF_CHECK_CUDA(cudaMemsetAsync(kv->red.gcnt, 0, (ngr + 1) * sizeof(unsigned int), st));
  HEF_CHECK_CUDA(cudaMemsetAsync(kv->red.tcnt, 0, sizeof(unsigned int), st));
  return HEF_OK;
}

template <typename T, typename TV = T>
hef_status run_krylov(const hef_incidence* inc, int k, int S, const double* x0c, const double* x0b,
                      void* Vv, long long ldv, void* ws, cudaStream_t st, void* tape = nullptr) {
  KView<T> kv;
  TapeLayout tl;
  if (hef_status s0 = krylov_view<T>(inc, k, S, ws, tape, &kv, &tl, st)) return s0;
  TV* V = static_cast<TV*>(Vv);
  hef_status s;
  switch (S) {
    case 1: s = run_krylov_s<T, 1, TV>(inc, k, x0c, x0b, V, ldv, kv, t_persistent, st); break;
    case 2: s = run_krylov_s<T, 2, TV>(inc, k, x0c, x0b, V, ldv, kv, t_persistent, st); break;
    case 4: s = run_krylov_s<T, 4, TV>(inc, k, x0c, x0b, V, ldv, kv, t_persistent, st); break;
    case 8: s = run_krylov_s<T, 8, TV>(inc, k, x0c, x0b, V, ldv, kv, t_persistent, st); break;
    case 16: s = run_krylov_s<T, 16, TV>(inc, k, x0c, x0b, V, ldv, kv, t_persistent, st); break;
    default: return set_error(HEF_ERR_UNSUPPORTED, "hef_krylov_basis: S must be 1, 2, 4, 8 or 16");
  }
  if (s || !tape) return s;
  HEF_CHECK_CUDA(cudaMemcpyAsync(tl.coef, kv.coef, (size_t)(k + 1) * 2 * S * 4 * sizeof(double),
                                 cudaMemcpyDeviceToDevice, st));
  HEF_CHECK_CUDA(cudaMemcpyAsync(tl.inv_nu, kv.inv_nu, (size_t)(k + 1) * 2 * S * sizeof(double),
                                 cudaMemcpyDeviceToDevice, st));
  return HEF_OK;
}

// Columns of one expansion from the mixed basis W (n x ldw): V[v, (j-1) S +
// s] = W[v, (j-1) 2S + op S + s].
template <typename T>
__global__ void k_select_op(long long n, int k, int S, int op, const T* __restrict__ W,
                            long long ldw, T* __restrict__ V, long long ldv) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long KS = (long long)k * S;
  if (t >= n * KS) return;
  const long long v = t / KS;
  const int c = (int)(t % KS), j = c / S, s = c % S;
  V[v * ldv + c] = W[v * ldw + (long long)j * 2 * S + op * S + s];
}

inline long long mixed_ld(int k, int S, size_t esz) {
  const long long K = 2ll * k * S, per = 16 / (long long)esz;
  return (K + per - 1) / per * per;
}

// Bytes of a basis element of `dtype` (FP64, FP32, or BF16: FP32 chains
// archived in BF16).
inline size_t basis_esz(int dtype) { return dtype == HEF_F64 ? 8 : (dtype == HEF_BF16 ? 2 : 4); }

hef_status check_krylov_args(const hef_incidence* inc, int k, int S, int dtype, const char* fn) {
  if (!inc) return set_error(HEF_ERR_INVALID_ARG, "%s: NULL incidence", fn);
  if (dtype != HEF_F64 && dtype != HEF_F32 && dtype != HEF_BF16)
    return set_error(HEF_ERR_INVALID_ARG, "%s: dtype must be HEF_F64, HEF_F32 or HEF_BF16", fn);
  if (k < 1) return set_error(HEF_ERR_INVALID_ARG, "%s: k must be >= 1", fn);
  if (S < 1 || S > kMaxS || (S & (S - 1)))
    return set_error(HEF_ERR_UNSUPPORTED, "%s: S must be 1, 2, 4, 8 or 16", fn);
  if (2ll * k * S > 512) return set_error(HEF_ERR_UNSUPPORTED, "%s: K = 2kS must be <= 512", fn);
  return HEF_OK;
}

// Starts of one hypergraph of a batch (the Krylov call up to its steps).
template <typename T>
hef_status batch_start(const hef_incidence* inc, int k, int S, const double* x0c,
                       const double* x0b, void* ws, cudaStream_t st) {
  KView<T> kv;
  TapeLayout tl;
  if (hef_status s0 = krylov_view<T>(inc, k, S, ws, nullptr, &kv, &tl, st)) return s0;
  switch (S) {
    case 1: return krylov_start_s<T, 1>(inc, x0c, x0b, kv, st);
    case 2: return krylov_start_s<T, 2>(inc, x0c, x0b, kv, st);
    case 4: return krylov_start_s<T, 4>(inc, x0c, x0b, kv, st);
    case 8: return krylov_start_s<T, 8>(inc, x0c, x0b, kv, st);
    case 16: return krylov_start_s<T, 16>(inc, x0c, x0b, kv, st);
    default: return set_error(HEF_ERR_UNSUPPORTED, "batched Krylov: S must be 1, 2, 4, 8 or 16");
  }
}

// CTA shares of a launch: at least one per hypergraph, the rest in proportion
// to the cost (largest remainders first); the shares sum to `total`.
void cta_shares(const double* cost, int n, int total, int* share) {
  double sum = 0.0;
  for (int i = 0; i < n; ++i) sum += cost[i] > 0 ? cost[i] : 0.0;
  const int spare = total - n;
  std::vector<std::pair<double, int>> rem;
  int used = 0;
  for (int i = 0; i < n; ++i) {
    const double want = sum > 0 ? spare * (cost[i] > 0 ? cost[i] : 0.0) / sum : 0.0;
    share[i] = 1 + (int)want;
    used += share[i];
    rem.push_back({want - (int)want, i});
  }
  std::stable_sort(rem.begin(), rem.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  for (size_t q = 0; q < rem.size() && used < total; ++q, ++used) ++share[rem[q].second];
}

template <typename T, int S, typename TV>
hef_status batch_steps_s(const KrylovBatchArg* items, int G, int k, cudaStream_t st) {
  constexpr int NT = pers_threads<T, S>();
  const size_t smem = pers_smem<T>(k, S, kCapItems, kCapList);
  constexpr size_t kSmemLimit = 227 * 1024;
  if (smem > kSmemLimit) return set_error(HEF_ERR_UNSUPPORTED, "batched Krylov: k too large");
  HEF_ENSURE_SMEM((k_krylov_batched<T, S, TV>), smem);
  int occ = 0;
  HEF_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_krylov_batched<T, S, TV>, NT,
                                                               smem));
  // one CTA per SM at most (the partial-sum buffers hold up to num_sms rows)
  const int total = num_sms() * std::min(std::max(occ, 1), 1);
  static_assert(sizeof(KBatch<T, TV>) < 32000, "kernel parameter space");
  auto bt = std::make_unique<KBatch<T, TV>>();
  for (int g0 = 0; g0 < G; g0 += kBatchItems) {
    const int nb = std::min(kBatchItems, G - g0);
    if (nb > total) return set_error(HEF_ERR_UNSUPPORTED, "batched Krylov: more items than CTAs");
    std::vector<double> cost(nb);
    std::vector<int> share(nb);
    for (int i = 0; i < nb; ++i) cost[i] = items[g0 + i].cost;
    cta_shares(cost.data(), nb, total, share.data());
    bt->nitems = nb;
    bt->k = k;
    bt->cta0[0] = 0;
    for (int i = 0; i < nb; ++i) {
      const KrylovBatchArg& a = items[g0 + i];
      KBatchItem<T, TV>& it = bt->it[i];
      it.g = view(a.inc);
      it.sv = scal_view<T>(a.inc);
      carve_krylov<T>(a.ws, a.inc->n, a.inc->m, k, S, &it.kv);
      it.kv.tape_c = it.kv.tape_b = nullptr;
      it.kv.tol = sizeof(T) == 8 ? 1e-12 : 1e-5;
      it.V = static_cast<TV*>(a.V);
      it.ldv = a.ldv;
      it.status = a.inc->status;
      bt->cta0[i + 1] = bt->cta0[i] + share[i];
      HEF_CHECK_CUDA(cudaMemsetAsync(it.kv.pcount, 0, flag_words(2 * num_sms()) * sizeof(unsigned int), st));
    }
    const KBatch<T, TV>& arg = *bt;
    cudaError_t e = cudaSuccess;
    HEF_LAUNCH("k_krylov_batched", st,
               e = launch_cooperative_smem(k_krylov_batched<T, S, TV>, bt->cta0[nb], NT, smem, st,
                                           arg));
    if (e != cudaSuccess) return set_error(HEF_ERR_CUDA, "k_krylov_batched: %s", cudaGetErrorString(e));
  }
  return HEF_OK;
}

template <typename T, typename TV>
hef_status batch_steps(const KrylovBatchArg* items, int G, int k, int S, cudaStream_t st) {
  switch (S) {
    case 1: return batch_steps_s<T, 1, TV>(items, G, k, st);
    case 2: return batch_steps_s<T, 2, TV>(items, G, k, st);
    case 4: return batch_steps_s<T, 4, TV>(items, G, k, st);
    case 8: return batch_steps_s<T, 8, TV>(items, G, k, st);
    case 16: return batch_steps_s<T, 16, TV>(items, G, k, st);
    default: return set_error(HEF_ERR_UNSUPPORTED, "batched Krylov: S must be 1, 2, 4, 8 or 16");
  }
}

}  // namespace

hef_status krylov_batch_start(const hef_incidence* inc, int k, int S, int dtype, const double* x0c,
                              const double* x0b, void* ws, cudaStream_t st) {
  if (dtype == HEF_F64) return batch_start<double>(inc, k, S, x0c, x0b, ws, st);
  return batch_start<float>(inc, k, S, x0c, x0b, ws, st);
}

hef_status krylov_batch_steps(const KrylovBatchArg* items, int G, int k, int S, int dtype,
                              cudaStream_t st) {
  if (dtype == HEF_F64) return batch_steps<double, double>(items, G, k, S, st);
  if (dtype == HEF_BF16) return batch_steps<float, __nv_bfloat16>(items, G, k, S, st);
  return batch_steps<float, float>(items, G, k, S, st);
}

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
  HEF_NVTX("hef_krylov_basis (Algorithm 1 step 3)");
  hef_status s = check_krylov_args(inc, k, S, dtype, "hef_krylov_basis");
  if (s) return s;
  const long long K = 2ll * k * S;
  if (!x0_clique || !x0_star || !V)
    return set_error(HEF_ERR_INVALID_ARG, "hef_krylov_basis: NULL array");
  const size_t esz = basis_esz(dtype);
  if (ldv < K || (ldv * esz) % 16 || (reinterpret_cast<uintptr_t>(V) & 15))
    return set_error(HEF_ERR_INVALID_ARG,
                     "hef_krylov_basis: ldv must be >= K = %lld with 16-byte aligned rows", K);
  size_t need = hef_krylov_workspace_bytes(inc, k, S, dtype);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return set_error(HEF_ERR_WORKSPACE, "hef_krylov_basis: workspace needs %zu bytes (256-aligned)",
                     need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == HEF_F64) return run_krylov<double>(inc, k, S, x0_clique, x0_star, V, ldv, workspace, st);
  if (dtype == HEF_BF16)
    return run_krylov<float, __nv_bfloat16>(inc, k, S, x0_clique, x0_star, V, ldv, workspace, st);
  return run_krylov<float>(inc, k, S, x0_clique, x0_star, V, ldv, workspace, st);
}

extern "C" hef_status hef_set_krylov_persistent(int32_t on) {
  if (on < 0 || on > 2) return set_error(HEF_ERR_INVALID_ARG, "hef_set_krylov_persistent: on must be 0, 1 or 2");
  krylov_allow_persistent(on != 0);
  krylov_force_oversized(on == 2);
  return HEF_OK;
}

extern "C" size_t hef_krylov_tape_bytes(const hef_incidence* inc, int32_t k, int32_t S, int32_t dtype) {
  if (check_krylov_args(inc, k, S, dtype, "hef_krylov_tape_bytes") || dtype == HEF_BF16) return 0;
  TapeLayout tl;
  return carve_tape(nullptr, inc->n, inc->m, k, S, dtype == HEF_F64 ? 8 : 4, &tl);
}

extern "C" hef_status hef_krylov_basis_tape(const hef_incidence* inc, int32_t k, int32_t S,
                                            int32_t dtype, const double* x0_clique,
                                            const double* x0_star, void* V, int64_t ldv,
                                            void* tape, size_t tape_bytes, void* workspace,
                                            size_t workspace_bytes, void* stream) {
  HEF_NVTX("hef_krylov_basis_tape (Algorithm 1 step 3, taped)");
  hef_status s = check_krylov_args(inc, k, S, dtype, "hef_krylov_basis_tape");
  if (s) return s;
  if (dtype == HEF_BF16)
    return set_error(HEF_ERR_UNSUPPORTED, "hef_krylov_basis_tape: the backward has no BF16 form");
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

extern "C" size_t hef_krylov_ops_workspace_bytes(const hef_incidence* inc, int32_t k, int32_t S,
                                                 int32_t dtype, int32_t ops) {
  const size_t base = hef_krylov_workspace_bytes(inc, k, S, dtype);
  if (!base || (ops != HEF_OPS_CLIQUE && ops != HEF_OPS_STAR && ops != HEF_OPS_BOTH)) return 0;
  if (ops == HEF_OPS_BOTH) return base;
  const size_t esz = basis_esz(dtype);
  return (base + 255) / 256 * 256 + (size_t)inc->n * mixed_ld(k, S, esz) * esz + 256;
}

extern "C" hef_status hef_krylov_basis_ops(const hef_incidence* inc, int32_t k, int32_t S,
                                           int32_t dtype, int32_t ops, const double* x0_clique,
                                           const double* x0_star, void* V, int64_t ldv,
                                           void* workspace, size_t workspace_bytes,
                                           void* stream) {
  HEF_NVTX("hef_krylov_basis_ops (Algorithm 1 step 3, one expansion)");
  if (ops == HEF_OPS_BOTH)
    return hef_krylov_basis(inc, k, S, dtype, x0_clique, x0_star, V, ldv, workspace,
                            workspace_bytes, stream);
  if (ops != HEF_OPS_CLIQUE && ops != HEF_OPS_STAR)
    return set_error(HEF_ERR_INVALID_ARG, "hef_krylov_basis_ops: unknown ops %d", ops);
  hef_status s = check_krylov_args(inc, k, S, dtype, "hef_krylov_basis_ops");
  if (s) return s;
  if (!x0_clique || !x0_star || !V) return set_error(HEF_ERR_INVALID_ARG, "hef_krylov_basis_ops: NULL array");
  const size_t esz = basis_esz(dtype);
  if (ldv < (long long)k * S || (ldv * esz) % 16 || (reinterpret_cast<uintptr_t>(V) & 15))
    return set_error(HEF_ERR_INVALID_ARG,
                     "hef_krylov_basis_ops: ldv must be >= k S with 16-byte aligned rows");
  const size_t base = hef_krylov_workspace_bytes(inc, k, S, dtype);
  const size_t need = hef_krylov_ops_workspace_bytes(inc, k, S, dtype, ops);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return set_error(HEF_ERR_WORKSPACE, "hef_krylov_basis_ops: workspace needs %zu bytes", need);
  // the kernels fuse both expansions: run them into a mixed basis in the
  // workspace, then keep the chosen expansion's columns
  char* W = static_cast<char*>(workspace) + (base + 255) / 256 * 256;
  const long long ldw = mixed_ld(k, S, esz);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s = dtype == HEF_F64    ? run_krylov<double>(inc, k, S, x0_clique, x0_star, W, ldw, workspace, st)
      : dtype == HEF_BF16 ? run_krylov<float, __nv_bfloat16>(inc, k, S, x0_clique, x0_star, W,
                                                             ldw, workspace, st)
                          : run_krylov<float>(inc, k, S, x0_clique, x0_star, W, ldw, workspace, st);
  if (s) return s;
  const long long total = inc->n * (long long)k * S;
  if (total == 0) return HEF_OK;
  const int op = ops == HEF_OPS_CLIQUE ? 0 : 1;
  const int grid = (int)((total + kThreads - 1) / kThreads);
  if (dtype == HEF_F64)
    HEF_LAUNCH("k_select_op", st, k_select_op<double><<<grid, kThreads, 0, st>>>(
                                      inc->n, k, S, op, reinterpret_cast<const double*>(W), ldw,
                                      static_cast<double*>(V), ldv));
  else if (dtype == HEF_BF16)
    HEF_LAUNCH("k_select_op", st, k_select_op<__nv_bfloat16><<<grid, kThreads, 0, st>>>(
                                      inc->n, k, S, op, reinterpret_cast<const __nv_bfloat16*>(W),
                                      ldw, static_cast<__nv_bfloat16*>(V), ldv));
  else
    HEF_LAUNCH("k_select_op", st, k_select_op<float><<<grid, kThreads, 0, st>>>(
                                      inc->n, k, S, op, reinterpret_cast<const float*>(W), ldw,
                                      static_cast<float*>(V), ldv));
  HEF_CHECK_LAUNCH();
  return HEF_OK;
}
