// Consumers of the hyperedge resistances: Algorithm 1 step 6 (sort) and one
// coarsening level of Algorithm 2 (Section III-B, steps 4-10), with Eq.
// R_W_update of Section III-A.3.  Readings of the paper (it fixes neither the
// threshold nor any tie rule), as stated in include/hef.h:
//  - Eq. R_W_update sums eta over a hyperedge's pins in pin order from 0.0,
//    then adds R_e (FP64).
//  - the sort is by ascending updated resistance, ties by ascending id;
//  - delta is given, or the q-quantile (position floor(q (c - 1)) of the c
//    hyperedges with >= 2 pins in sorted order); contraction needs R_e < delta;
//  - contraction is greedy in sorted order: a hyperedge is contracted when
//    none of its pins belongs to an earlier contracted hyperedge;
//  - supernodes are numbered by their smallest vertex, weighted by the
//    resistance of the hyperedge that formed them;
//  - isolated vertices (seeds) join the neighbouring supernode at the smallest
//    distance max_i (Q[p,i] - mu_c[i])^2 / Q_H[i] (mu_c = mean row of the
//    supernode's members, summed in pin order), ties to the smallest id, and
//    add eta(p) + d to its weight in ascending p order;
//  - final ids are compact in the order of each cluster's smallest vertex; the
//    coarse hypergraph keeps each hyperedge's first occurrence of every
//    cluster and drops hyperedges left with fewer than 2 pins.
// Every result is a deterministic function of the inputs: integer atomics
// only, FP64 sums in the stated orders with explicit round-to-nearest
// operations (no contraction into fused multiply-adds), so the results equal
// a sequential CPU statement of the same rules bit for bit.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "internal.h"

namespace hef {

namespace {

#define HEF_PASS(x)              \
  do {                           \
    hef_status s_ = (x);         \
    if (s_ != HEF_OK) return s_; \
  } while (0)

constexpr int kStateLive = 0, kStateIn = 1, kStateOut = 2;
constexpr unsigned int kSpinIters = 1u << 21;  // bounded barrier wait

// FP64 keys as order-preserving unsigned integers (-0.0 taken as +0.0).
__device__ __forceinline__ unsigned long long ordered_bits(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x == 0.0 ? 0.0 : x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Eq. R_W_update per hyperedge (thread per hyperedge, pins in order) and the
// low words of the sort keys.
__global__ void k_update_r(int m, const int64_t* __restrict__ eptr, const int32_t* __restrict__ pins,
                           const double* __restrict__ R, const double* __restrict__ eta,
                           double* __restrict__ Ru, uint32_t* __restrict__ keys,
                           int32_t* __restrict__ vals) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  double acc = 0.0;
  if (eta) {
    for (int64_t t = eptr[e]; t < eptr[e + 1]; ++t) acc = __dadd_rn(acc, eta[pins[t]]);
  }
  const double r = __dadd_rn(acc, R[e]);
  if (Ru) Ru[e] = r;
  keys[e] = (uint32_t)(ordered_bits(r) & 0xffffffffull);
  vals[e] = e;
}

__global__ void k_high_keys(int m, const double* __restrict__ Ru, const int32_t* __restrict__ vals,
                            uint32_t* __restrict__ keys) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) keys[i] = (uint32_t)(ordered_bits(Ru[vals[i]]) >> 32);
}

// rank[order[i]] = i; flags of the hyperedges with >= 2 pins in sorted order.
__global__ void k_rank(int m, const int32_t* __restrict__ order, const int64_t* __restrict__ eptr,
                       int32_t* __restrict__ rank, int* __restrict__ big) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int e = order[i];
  rank[e] = i;
  big[i] = (eptr[e + 1] - eptr[e]) >= 2 ? 1 : 0;
}

// delta: the given value, or the q-quantile of the resistances of the
// hyperedges with >= 2 pins (pos = their exclusive scan in sorted order).
__global__ void k_delta(int m, double given, double q, const int32_t* __restrict__ order,
                        const double* __restrict__ Ru, const int* __restrict__ big,
                        const int* __restrict__ pos, double* __restrict__ delta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (given >= 0.0) {
    if (i == 0) *delta = given;
    return;
  }
  const int c = pos[m];
  if (c == 0) {
    if (i == 0) *delta = INFINITY;
    return;
  }
  const int want = (int)floor(__dmul_rn(q, (double)(c - 1)));
  if (i < m && big[i] && pos[i] == want) *delta = Ru[order[i]];
}

__global__ void k_contract_init(int n, int m, const int64_t* __restrict__ eptr,
                                const double* __restrict__ Ru, const double* __restrict__ delta,
                                int* __restrict__ state, int* __restrict__ best,
                                int32_t* __restrict__ owner) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double d = *delta;
  if (i < m) state[i] = ((eptr[i + 1] - eptr[i]) >= 2 && Ru[i] < d) ? kStateLive : kStateOut;
  if (i < n) best[i] = 0x7fffffff, owner[i] = -1;
}

// Grid barrier of the contraction kernel: arrivals on a monotonic counter,
// bounded wait.  Returns false when the wait ran out (status set).
__device__ __forceinline__ bool grid_sync(unsigned int* count, unsigned int target,
                                          int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    unsigned int it = 0;
    int good = 1;
    while (*reinterpret_cast<volatile unsigned int*>(count) < target) {
      if (++it > kSpinIters || *reinterpret_cast<volatile int*>(status)) {
        atomicOr(status, 1);
        good = 0;
        break;
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok;
}

// The greedy contraction as rounds (one cooperative launch): in each round a
// live candidate whose rank is the smallest among the live candidates at
// every one of its pins is contracted (such hyperedges are pin-disjoint),
// and a live candidate with a pin taken by a contracted hyperedge drops out.
// A live candidate is contracted exactly when every earlier candidate that
// shares a pin with it has dropped out, which is the sequential greedy rule;
// every round decides at least the smallest live rank, so at most
// (candidates + 1) rounds run.  round_live[r] counts the live candidates left
// after round r.
__global__ void k_contract(int m, const int64_t* __restrict__ eptr, const int32_t* __restrict__ pins,
                           const int32_t* __restrict__ rank, int* state, int* best, int32_t* owner,
                           int* last, int* round_live, unsigned int* count, int* status) {
  const int stride = gridDim.x * blockDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned int ph = 0;
  for (int r = 0; r <= m; ++r) {
    // 1: every live candidate marks its rank at its pins
    for (int e = tid; e < m; e += stride) {
      if (__ldcg(state + e) != kStateLive) continue;
      last[e] = r;
      const int rk = rank[e];
      for (int64_t t = eptr[e]; t < eptr[e + 1]; ++t) atomicMin(best + pins[t], rk);
    }
    if (!grid_sync(count, (++ph) * gridDim.x, status)) return;
    // 2: the smallest live rank at all of its pins is contracted
    for (int e = tid; e < m; e += stride) {
      if (__ldcg(state + e) != kStateLive) continue;
      const int rk = rank[e];
      bool mine = true;
      for (int64_t t = eptr[e]; t < eptr[e + 1] && mine; ++t) mine = __ldcg(best + pins[t]) == rk;
      if (mine) {
        state[e] = kStateIn;
        for (int64_t t = eptr[e]; t < eptr[e + 1]; ++t) owner[pins[t]] = e;
      }
    }
    if (!grid_sync(count, (++ph) * gridDim.x, status)) return;
    // 3: live candidates with a taken pin drop out; the round's marks are cleared
    for (int e = tid; e < m; e += stride) {
      if (__ldcg(last + e) != r) continue;
      const int st = __ldcg(state + e);
      bool taken = false;
      for (int64_t t = eptr[e]; t < eptr[e + 1]; ++t) {
        best[pins[t]] = 0x7fffffff;
        taken = taken || __ldcg(owner + pins[t]) >= 0;
      }
      if (st == kStateLive) {
        if (taken) state[e] = kStateOut;
        else atomicAdd(round_live + r, 1);
      }
    }
    if (!grid_sync(count, (++ph) * gridDim.x, status)) return;
    if (__ldcg(round_live + r) == 0) return;
  }
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(status, 2);  // more rounds than possible
}

// Smallest pin of every contracted hyperedge.
__global__ void k_minpin(int m, const int64_t* __restrict__ eptr, const int32_t* __restrict__ pins,
                         const int* __restrict__ state, int32_t* __restrict__ minpin) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m || state[e] != kStateIn) return;
  int mn = 0x7fffffff;
  for (int64_t t = eptr[e]; t < eptr[e + 1]; ++t) mn = min(mn, pins[t]);
  minpin[e] = mn;
}

__global__ void k_cluster_flags(int n, const int32_t* __restrict__ owner,
                                const int32_t* __restrict__ minpin, int* __restrict__ flag) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int o = owner[v];
  flag[v] = (o < 0 || minpin[o] == v) ? 1 : 0;
}

__global__ void k_clusters(int n, const int32_t* __restrict__ owner, const int32_t* __restrict__ minpin,
                           const int* __restrict__ cid, const double* __restrict__ Ru,
                           const double* __restrict__ eta, int32_t* __restrict__ cluster,
                           double* __restrict__ eta_next, int32_t* __restrict__ formed_by,
                           int* __restrict__ contracted_flag) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int o = owner[v];
  const int c = o < 0 ? cid[v] : cid[minpin[o]];
  cluster[v] = c;
  if (o < 0) {
    eta_next[c] = eta ? eta[v] : 0.0;
    formed_by[c] = -1;
    contracted_flag[c] = 0;
  } else if (minpin[o] == v) {
    eta_next[c] = Ru[o];
    formed_by[c] = o;
    contracted_flag[c] = 1;
  }
}

template <typename T>
__device__ __forceinline__ double qval(const T* Q, long long ldq, long long row, int i) {
  if constexpr (std::is_same<T, __nv_bfloat16>::value) return (double)__bfloat162float(Q[row * ldq + i]);
  else return (double)Q[row * ldq + i];
}

// Centroid rows of the contracted supernodes: one warp per supernode, lanes
// over columns, members summed in the forming hyperedge's pin order.
template <typename T>
__global__ void k_centroids(int nc, const int32_t* __restrict__ formed_by,
                            const int* __restrict__ mrow, const int64_t* __restrict__ eptr,
                            const int32_t* __restrict__ pins, const T* __restrict__ Q, long long ldq,
                            int K, double* __restrict__ mu) {
  const int lane = threadIdx.x & 31;
  const int c = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (c >= nc) return;
  const int e = formed_by[c];
  if (e < 0) return;
  const int64_t a = eptr[e], b = eptr[e + 1];
  const double k = (double)(b - a);
  double* row = mu + (size_t)mrow[c] * K;
  for (int i = lane; i < K; i += 32) {
    double acc = 0.0;
    for (int64_t t = a; t < b; ++t) acc = __dadd_rn(acc, qval(Q, ldq, pins[t], i));
    row[i] = __ddiv_rn(acc, k);
  }
}

// Local clustering of the isolated vertices: one warp per vertex; every
// candidate supernode (of a co-pin in a hyperedge containing the vertex) is
// scored by max over columns of (Q[p,i] - mu_c[i])^2 / Q_H[i]; the smallest
// score wins, ties to the smallest cluster id.
template <typename T>
__global__ void k_seeds(int n, const int32_t* __restrict__ owner, const int32_t* __restrict__ vptr,
                        const int32_t* __restrict__ vedge, const int32_t* __restrict__ perm,
                        const int64_t* __restrict__ eptr, const int32_t* __restrict__ pins,
                        const int32_t* __restrict__ cluster, const int32_t* __restrict__ formed_by,
                        const int* __restrict__ mrow, const double* __restrict__ mu,
                        const T* __restrict__ Q, long long ldq, int K,
                        const double* __restrict__ QH, int32_t* __restrict__ target,
                        double* __restrict__ dist) {
  const int lane = threadIdx.x & 31;
  const int p = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (p >= n) return;
  if (owner[p] >= 0) {
    if (lane == 0) target[p] = -1, dist[p] = 0.0;
    return;
  }
  int best = -1;
  double bd = INFINITY;
  for (int t = vptr[p]; t < vptr[p + 1]; ++t) {
    const int e = perm[vedge[t]];
    for (int64_t s = eptr[e]; s < eptr[e + 1]; ++s) {
      const int u = pins[s];
      const int c = cluster[u];
      if (u == p || formed_by[c] < 0) continue;
      const double* row = mu + (size_t)mrow[c] * K;
      double d = 0.0;
      for (int i = lane; i < K; i += 32) {
        const double qh = QH[i];
        if (qh > 1e-300) {
          const double diff = __dsub_rn(qval(Q, ldq, p, i), row[i]);
          const double r = __ddiv_rn(__dmul_rn(diff, diff), qh);
          d = r > d ? r : d;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double x = __shfl_xor_sync(0xffffffffu, d, o);
        d = x > d ? x : d;
      }
      if (d < bd || (d == bd && c < best)) best = c, bd = d;
    }
  }
  if (lane == 0) {
    target[p] = best;
    dist[p] = best >= 0 ? bd : 0.0;
  }
}

// Sort keys of the merges: target + 1 for seeds that join, 0 otherwise.
__global__ void k_merge_keys(int n, const int32_t* __restrict__ target, uint32_t* __restrict__ keys,
                             int32_t* __restrict__ vals) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  keys[v] = (uint32_t)(target[v] + 1);
  vals[v] = v;
}

// Weight of each supernode that seeds join: its own weight, then eta(p) +
// d(p) for the seeds in ascending p (a sorted segment, summed by one thread).
__global__ void k_merge_sums(int n, const uint32_t* __restrict__ keys, const int32_t* __restrict__ vals,
                             const double* __restrict__ eta, const double* __restrict__ dist,
                             double* __restrict__ eta2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || keys[i] == 0u || (i > 0 && keys[i - 1] == keys[i])) return;
  const int c = (int)keys[i] - 1;
  double acc = eta2[c];
  for (int j = i; j < n && keys[j] == keys[i]; ++j) {
    const int p = vals[j];
    acc = __dadd_rn(acc, __dadd_rn(eta ? eta[p] : 0.0, dist[p]));
  }
  eta2[c] = acc;
}

__global__ void k_final_min(int n, const int32_t* __restrict__ cluster, const int32_t* __restrict__ target,
                            int* __restrict__ minv) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int c = target[v] >= 0 ? target[v] : cluster[v];
  atomicMin(minv + c, v);
}

__global__ void k_final_flags(int n, const int32_t* __restrict__ cluster,
                              const int32_t* __restrict__ target, const int* __restrict__ minv,
                              int* __restrict__ flag) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int c = target[v] >= 0 ? target[v] : cluster[v];
  flag[v] = minv[c] == v ? 1 : 0;
}

__global__ void k_final_ids(int n, const int32_t* __restrict__ cluster, const int32_t* __restrict__ target,
                            const int* __restrict__ minv, const int* __restrict__ fid,
                            const double* __restrict__ eta2, int32_t* __restrict__ final_id,
                            double* __restrict__ eta_out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int c = target[v] >= 0 ? target[v] : cluster[v];
  const int f = fid[minv[c]];
  final_id[v] = f;
  if (minv[c] == v) eta_out[f] = eta2[c];
}

// Distinct clusters of a hyperedge, first occurrences in pin order: with
// `out`, written there; returns their count.
__device__ __forceinline__ int distinct_clusters(const int32_t* pins, int64_t a, int64_t b,
                                                 const int32_t* fid, int32_t* out) {
  int k = 0;
  for (int64_t t = a; t < b; ++t) {
    const int c = fid[pins[t]];
    bool seen = false;
    for (int64_t u = a; u < t && !seen; ++u) seen = fid[pins[u]] == c;
    if (!seen) {
      if (out) out[k] = c;
      ++k;
    }
  }
  return k;
}

__global__ void k_coarse_count(int m, const int64_t* __restrict__ eptr, const int32_t* __restrict__ pins,
                               const int32_t* __restrict__ fid, int* __restrict__ keep,
                               int* __restrict__ cnt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  const int k = distinct_clusters(pins, eptr[e], eptr[e + 1], fid, nullptr);
  keep[e] = k >= 2 ? 1 : 0;
  cnt[e] = k >= 2 ? k : 0;
}

__global__ void k_coarse_fill(int m, const int64_t* __restrict__ eptr, const int32_t* __restrict__ pins,
                              const double* __restrict__ w, const int32_t* __restrict__ fid,
                              const int* __restrict__ keep, const int* __restrict__ ne,
                              const int* __restrict__ po, int64_t* __restrict__ ceptr,
                              int32_t* __restrict__ cpins, double* __restrict__ cw,
                              int32_t* __restrict__ emap) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e > m) return;
  if (e == m) {
    ceptr[ne[m]] = po[m];
    return;
  }
  if (!keep[e]) return;
  const int i = ne[e];
  ceptr[i] = po[e];
  cw[i] = w[e];
  emap[i] = e;
  distinct_clusters(pins, eptr[e], eptr[e + 1], fid, cpins + po[e]);
}

__global__ void k_counts(const int* __restrict__ nc, const int* __restrict__ nf,
                         const int* __restrict__ mc, const int* __restrict__ pc,
                         const int* __restrict__ status, int32_t* __restrict__ counts) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    counts[0] = *nc, counts[1] = *nf, counts[2] = *mc, counts[3] = *pc, counts[4] = *status;
}

inline int grid_of(long long N) { return (int)((N + kThreads - 1) / kThreads); }

struct LevelWs {
  uint32_t* keys;
  int32_t* vals;
  SortBufs sb;
  unsigned int* counter;  // [0] scans and sorts, [1] contraction barrier
  int* status;            // [0] contraction wait / round overflow
  int32_t* rank;
  int* state;
  int* last;
  int* round_live;
  int* best;
  int32_t* minpin;
  int* flag;     // max(n, m) + 1
  int* scan;     // max(n, m) + 1
  int* bsum;
  int* cflag;    // n + 1: contracted-cluster flags, scanned into row indices
  int32_t* formed_by;
  double* eta_next;
  double* eta2;
  double* mu;
  int* minv;
  int* keep;     // m + 1
  int* ne;       // m + 1
  int* po;       // m + 1
};

size_t carve_level(void* base, long long n, long long m, int K, LevelWs* w) {
  Carver c(base);
  const long long N = (n > m ? n : m) + 1;
  w->keys = c.take<uint32_t>(N);
  w->vals = c.take<int32_t>(N);
  carve_sort_bufs(c, N, &w->sb);
  w->counter = c.take<unsigned int>(4);
  w->sb.counter = w->counter;
  w->status = c.take<int>(2);
  w->rank = c.take<int32_t>(m + 1);
  w->state = c.take<int>(m + 1);
  w->last = c.take<int>(m + 1);
  w->round_live = c.take<int>(m + 2);
  w->best = c.take<int>(n + 1);
  w->minpin = c.take<int32_t>(m + 1);
  w->flag = c.take<int>(N + 1);
  w->scan = c.take<int>(N + 1);
  w->bsum = c.take<int>(scan_tiles(N + 1) + 1);
  w->cflag = c.take<int>(n + 1);
  w->formed_by = c.take<int32_t>(n + 1);
  w->eta_next = c.take<double>(n + 1);
  w->eta2 = c.take<double>(n + 1);
  w->mu = c.take<double>((size_t)(n / 2 + 1) * (K > 0 ? K : 1));
  w->minv = c.take<int>(n + 1);
  w->keep = c.take<int>(m + 1);
  w->ne = c.take<int>(m + 1);
  w->po = c.take<int>(m + 1);
  return c.bytes();
}

// Sorted order of R (ascending, ties by id) into `order`: a stable sort on the
// low key words, then on the high words.
hef_status sort_by_value(int m, const double* Ru, int32_t* order, LevelWs& w, cudaStream_t st) {
  if (m <= 0) return HEF_OK;
  HEF_PASS(radix_sort(w.keys, w.vals, m, 32, w.sb, st));
  HEF_LAUNCH("k_high_keys", st, k_high_keys<<<grid_of(m), kThreads, 0, st>>>(m, Ru, w.vals, w.keys));
  HEF_CHECK_LAUNCH();
  HEF_PASS(radix_sort(w.keys, w.vals, m, 32, w.sb, st));
  HEF_CHECK_CUDA(cudaMemcpyAsync(order, w.vals, (size_t)m * sizeof(int32_t),
                                 cudaMemcpyDeviceToDevice, st));
  return HEF_OK;
}

}  // namespace

}  // namespace hef

using namespace hef;

extern "C" size_t hef_level_workspace_bytes(int64_t n, int64_t m, int32_t K) {
  if (n < 0 || m < 0 || K < 0 || K > 512) return 0;
  LevelWs w;
  return carve_level(nullptr, n, m, K, &w);
}

extern "C" hef_status hef_sort_resistance(int64_t m, const double* R, int32_t* order,
                                          void* workspace, size_t workspace_bytes, void* stream) {
  HEF_NVTX("hef_sort_resistance (Algorithm 1 step 6)");
  if (m < 0 || m > 0x7fffffffll) return set_error(HEF_ERR_INVALID_ARG, "hef_sort_resistance: bad m");
  if (m > 0 && (!R || !order)) return set_error(HEF_ERR_INVALID_ARG, "hef_sort_resistance: NULL array");
  LevelWs w;
  const size_t need = carve_level(workspace, 0, m, 0, &w);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return set_error(HEF_ERR_WORKSPACE, "hef_sort_resistance: workspace needs %zu bytes", need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (m == 0) return HEF_OK;
  HEF_CHECK_CUDA(cudaMemsetAsync(w.counter, 0, 4 * sizeof(unsigned int), st));
  // keys of R itself (no eta): Eq. R_W_update with eta = 0 is R
  HEF_LAUNCH("k_update_r", st, k_update_r<<<grid_of(m), kThreads, 0, st>>>(
                                   (int)m, nullptr, nullptr, R, nullptr, nullptr, w.keys, w.vals));
  HEF_CHECK_LAUNCH();
  return sort_by_value((int)m, R, order, w, st);
}

extern "C" hef_status hef_coarsen_level(const hef_incidence* inc, const int64_t* eptr,
                                        const int32_t* pins, const double* w, const double* R,
                                        const double* eta, const void* Q, int64_t ldq, int32_t K,
                                        int32_t dtype, const double* QH, double delta,
                                        double quantile, const hef_level_out* out,
                                        void* workspace, size_t workspace_bytes, void* stream) {
  HEF_NVTX("hef_coarsen_level (Algorithm 2 steps 4-10)");
  if (!inc || !out) return set_error(HEF_ERR_INVALID_ARG, "hef_coarsen_level: NULL incidence or out");
  const long long n = inc->n, m = inc->m;
  if (m > 0 && (!eptr || !pins || !w || !R))
    return set_error(HEF_ERR_INVALID_ARG, "hef_coarsen_level: NULL input array");
  if (!out->R_upd || !out->order || !out->delta || !out->owner || !out->cluster || !out->target ||
      !out->dist || !out->final_cluster || !out->eta_out || !out->counts || !out->ceptr ||
      !out->cpins || !out->cw || !out->emap)
    return set_error(HEF_ERR_INVALID_ARG, "hef_coarsen_level: NULL output array");
  if (Q) {
    if (K < 1 || K > 512 || ldq < K || !QH)
      return set_error(HEF_ERR_INVALID_ARG, "hef_coarsen_level: need 1 <= K <= 512, ldq >= K and QH");
    if (dtype != HEF_F64 && dtype != HEF_F32 && dtype != HEF_BF16)
      return set_error(HEF_ERR_INVALID_ARG,
                       "hef_coarsen_level: dtype must be HEF_F64, HEF_F32 or HEF_BF16");
  }
  if (!(delta >= 0.0) && !(quantile >= 0.0 && quantile <= 1.0))
    return set_error(HEF_ERR_INVALID_ARG,
                     "hef_coarsen_level: give delta >= 0, or delta < 0 and 0 <= quantile <= 1");
  LevelWs ws;
  const size_t need = carve_level(workspace, n, m, Q ? K : 0, &ws);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return set_error(HEF_ERR_WORKSPACE, "hef_coarsen_level: workspace needs %zu bytes", need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nn = (int)n, mm = (int)m;
  const long long N = (n > m ? n : m);
  HEF_CHECK_CUDA(cudaMemsetAsync(ws.counter, 0, 4 * sizeof(unsigned int), st));
  HEF_CHECK_CUDA(cudaMemsetAsync(ws.status, 0, 2 * sizeof(int), st));
  HEF_CHECK_CUDA(cudaMemsetAsync(ws.round_live, 0, (m + 2) * sizeof(int), st));
  HEF_CHECK_CUDA(cudaMemsetAsync(out->counts, 0, 5 * sizeof(int32_t), st));
  // cluster tables: entries at or past the cluster count stay "not contracted"
  HEF_CHECK_CUDA(cudaMemsetAsync(ws.formed_by, 0xff, (size_t)(n + 1) * sizeof(int32_t), st));
  HEF_CHECK_CUDA(cudaMemsetAsync(ws.cflag, 0, (size_t)(n + 1) * sizeof(int), st));
  // Eq. R_W_update and Algorithm 1 step 6
  if (m > 0) {
    HEF_LAUNCH("k_update_r", st, k_update_r<<<grid_of(m), kThreads, 0, st>>>(
                                     mm, eptr, pins, R, eta, out->R_upd, ws.keys, ws.vals));
    HEF_CHECK_LAUNCH();
    HEF_PASS(sort_by_value(mm, out->R_upd, out->order, ws, st));
    HEF_LAUNCH("k_rank", st, k_rank<<<grid_of(m), kThreads, 0, st>>>(mm, out->order, eptr, ws.rank,
                                                                     ws.flag));
    HEF_CHECK_LAUNCH();
    HEF_PASS(exclusive_scan(ws.flag, ws.scan, m, ws.bsum, ws.counter, st));
  } else {
    HEF_CHECK_CUDA(cudaMemsetAsync(ws.scan, 0, sizeof(int), st));
  }
  HEF_LAUNCH("k_delta", st, k_delta<<<grid_of(m > 0 ? m : 1), kThreads, 0, st>>>(
                                mm, delta >= 0.0 ? delta : -1.0, quantile, out->order, out->R_upd,
                                ws.flag, ws.scan, out->delta));
  HEF_CHECK_LAUNCH();
  // Algorithm 2 step 5: greedy contraction
  HEF_LAUNCH("k_contract_init", st, k_contract_init<<<grid_of(N > 0 ? N : 1), kThreads, 0, st>>>(
                                        nn, mm, eptr, out->R_upd, out->delta, ws.state, ws.best,
                                        out->owner));
  HEF_CHECK_LAUNCH();
  if (m > 0) {
    int occ = 0;
    HEF_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_contract, kThreads, 0));
    const int grid = std::max(1, std::min(num_sms() * std::max(occ, 1), grid_of(m)));
    cudaError_t e = cudaSuccess;
    HEF_LAUNCH("k_contract", st,
               e = launch_cooperative_smem(k_contract, grid, kThreads, 0, st, mm, eptr, pins,
                                           (const int32_t*)ws.rank, ws.state, ws.best, out->owner,
                                           ws.last, ws.round_live, ws.counter + 1, ws.status));
    if (e != cudaSuccess) return set_error(HEF_ERR_CUDA, "k_contract: %s", cudaGetErrorString(e));
    HEF_LAUNCH("k_minpin", st, k_minpin<<<grid_of(m), kThreads, 0, st>>>(mm, eptr, pins, ws.state,
                                                                         ws.minpin));
    HEF_CHECK_LAUNCH();
  }
  // supernodes (numbered by their smallest vertex) and their weights
  int* cid = ws.scan;
  if (n > 0) {
    HEF_LAUNCH("k_cluster_flags", st, k_cluster_flags<<<grid_of(n), kThreads, 0, st>>>(
                                          nn, out->owner, ws.minpin, ws.flag));
    HEF_CHECK_LAUNCH();
  }
  HEF_PASS(exclusive_scan(ws.flag, cid, n, ws.bsum, ws.counter, st));
  if (n > 0) {
    HEF_LAUNCH("k_clusters", st, k_clusters<<<grid_of(n), kThreads, 0, st>>>(
                                     nn, out->owner, ws.minpin, cid, out->R_upd, eta, out->cluster,
                                     ws.eta_next, ws.formed_by, ws.cflag));
    HEF_CHECK_LAUNCH();
  }
  // nc is cid[n]; the clusters' arrays are indexed below it.  Algorithm 2
  // steps 7-10: local clustering of the isolated vertices
  HEF_CHECK_CUDA(cudaMemcpyAsync(ws.eta2, ws.eta_next, (size_t)(n > 0 ? n : 1) * sizeof(double),
                                 cudaMemcpyDeviceToDevice, st));
  if (n > 0) HEF_CHECK_CUDA(cudaMemsetAsync(out->target, 0xff, (size_t)n * sizeof(int32_t), st));
  if (n > 0) HEF_CHECK_CUDA(cudaMemsetAsync(out->dist, 0, (size_t)n * sizeof(double), st));
  int* nc_dev = cid + n;
  if (Q && n > 0 && m > 0) {
    // row of each contracted supernode in the centroid table (cflag is
    // defined for cluster ids below nc; the rest are never read)
    HEF_PASS(exclusive_scan(ws.cflag, ws.cflag, n, ws.bsum, ws.counter, st));
    const IncView g = view(inc);
    const int wgrid = (int)((n * 32 + kThreads - 1) / kThreads);
    auto run = [&](auto tag) -> hef_status {
      using QT = decltype(tag);
      HEF_LAUNCH("k_centroids", st, k_centroids<QT><<<wgrid, kThreads, 0, st>>>(
                                        nn, ws.formed_by, ws.cflag, eptr, pins,
                                        static_cast<const QT*>(Q), ldq, K, ws.mu));
      HEF_LAUNCH("k_seeds", st, k_seeds<QT><<<wgrid, kThreads, 0, st>>>(
                                    nn, out->owner, g.vptr, g.vedge, g.perm, eptr, pins,
                                    out->cluster, ws.formed_by, ws.cflag, ws.mu,
                                    static_cast<const QT*>(Q), ldq, K, QH, out->target,
                                    out->dist));
      return HEF_OK;
    };
    if (dtype == HEF_F64) HEF_PASS(run(double{}));
    else if (dtype == HEF_BF16) HEF_PASS(run(__nv_bfloat16{}));
    else HEF_PASS(run(float{}));
    HEF_CHECK_LAUNCH();
    HEF_LAUNCH("k_merge_keys", st, k_merge_keys<<<grid_of(n), kThreads, 0, st>>>(
                                       nn, out->target, ws.keys, ws.vals));
    HEF_CHECK_LAUNCH();
    HEF_PASS(radix_sort(ws.keys, ws.vals, n, bits_for(n + 1), ws.sb, st));
    HEF_LAUNCH("k_merge_sums", st, k_merge_sums<<<grid_of(n), kThreads, 0, st>>>(
                                       nn, ws.keys, ws.vals, eta, out->dist, ws.eta2));
    HEF_CHECK_LAUNCH();
  }
  // final compact ids, their weights
  if (n > 0) {
    HEF_CHECK_CUDA(cudaMemsetAsync(ws.minv, 0x7f, (size_t)n * sizeof(int), st));
    HEF_LAUNCH("k_final_min", st, k_final_min<<<grid_of(n), kThreads, 0, st>>>(
                                      nn, out->cluster, out->target, ws.minv));
    HEF_LAUNCH("k_final_flags", st, k_final_flags<<<grid_of(n), kThreads, 0, st>>>(
                                        nn, out->cluster, out->target, ws.minv, ws.flag));
    HEF_CHECK_LAUNCH();
  }
  int* fid = ws.cflag;  // reuse: the centroid rows are no longer needed
  HEF_PASS(exclusive_scan(ws.flag, fid, n, ws.bsum, ws.counter, st));
  if (n > 0) {
    HEF_LAUNCH("k_final_ids", st, k_final_ids<<<grid_of(n), kThreads, 0, st>>>(
                                      nn, out->cluster, out->target, ws.minv, fid, ws.eta2,
                                      out->final_cluster, out->eta_out));
    HEF_CHECK_LAUNCH();
  }
  // Algorithm 2 step 6: the coarse hypergraph
  if (m > 0) {
    HEF_LAUNCH("k_coarse_count", st, k_coarse_count<<<grid_of(m), kThreads, 0, st>>>(
                                         mm, eptr, pins, out->final_cluster, ws.keep, ws.flag));
    HEF_CHECK_LAUNCH();
  }
  HEF_PASS(exclusive_scan(ws.keep, ws.ne, m, ws.bsum, ws.counter, st));
  HEF_PASS(exclusive_scan(ws.flag, ws.po, m, ws.bsum, ws.counter, st));
  HEF_LAUNCH("k_coarse_fill", st, k_coarse_fill<<<grid_of(m + 1), kThreads, 0, st>>>(
                                      mm, eptr, pins, w, out->final_cluster, ws.keep, ws.ne, ws.po,
                                      out->ceptr, out->cpins, out->cw, out->emap));
  HEF_LAUNCH("k_counts", st, k_counts<<<1, 32, 0, st>>>(nc_dev, fid + n, ws.ne + m, ws.po + m,
                                                         ws.status, out->counts));
  HEF_CHECK_LAUNCH();
  return HEF_OK;
}
