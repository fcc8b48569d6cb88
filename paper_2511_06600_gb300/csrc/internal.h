// Internal host-side declarations shared by the hef translation units.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"

// Host handle of a built incidence.  Every pointer is device memory inside
// the caller's incidence workspace.  "Internal" hyperedge order is the
// locality schedule (ascending smallest pin, ties by caller id); perm maps it
// back to the caller's ids.
struct hef_incidence {
  int64_t n = 0, m = 0, P = 0;
  int32_t clique_mode = 0;
  unsigned int* status = nullptr;   // [0] error bits, [1] first bad edge
  unsigned int* counter = nullptr;  // last-CTA counter for build kernels
  int32_t* perm = nullptr;          // m: internal -> caller hyperedge id
  int32_t* ceptr = nullptr;         // m+1: CSC offsets (internal order)
  int32_t* cpins = nullptr;         // P: pins (internal order)
  int32_t* slot_edge = nullptr;     // P: internal hyperedge of each CSC slot
  int32_t* big_idx = nullptr;       // m: internal ids of hyperedges with > 64 pins
  int32_t* big_pos = nullptr;       // m+1: exclusive scan of the big flags; [m] = count
  int32_t* win_edge = nullptr;      // nwin+1: first hyperedge of each window of CSC slots
  double* ew = nullptr;             // m: w_e, 0 when |e| < 2
  double* ewh = nullptr;            // m: clique pair weight, 0 when |e| < 2
  double* ez = nullptr;             // m: star weight w_e/|e|, 0 when |e| < 2
  int32_t* vptr = nullptr;          // n+1: vertex-major offsets
  int32_t* vedge = nullptr;         // P: internal hyperedge of each entry
  int32_t* vslot = nullptr;         // P: CSC slot of each entry
  double* dc = nullptr;             // n: clique degree
  double* db = nullptr;             // n: star degree of vertices
  double* inv_dc = nullptr;         // n: 1/dc (0 for isolated)
  double* inv_db = nullptr;         // n: 1/db (0 for isolated)
  double* wsc = nullptr;            // n: sum of clique pair weights over e ∋ v
  double* totals = nullptr;         // [0] sum dc, [1] sum db, [2] sum w (|e|>=2)
  // FP32 copies of the scalars above, read by the FP32 form's kernels
  float* f_ew = nullptr;
  float* f_ewh = nullptr;
  float* f_ez = nullptr;
  float* f_dc = nullptr;
  float* f_db = nullptr;
  float* f_inv_dc = nullptr;
  float* f_inv_db = nullptr;
  float* f_wsc = nullptr;
};

namespace hef {

constexpr int kBigEdge = 64;  // hyperedges with more pins are scored by a whole CTA

// Windows of CSC slots for the staged scoring pass: window w covers slots
// [w kWinSlots, (w+1) kWinSlots) and owns the hyperedges whose first slot lies
// in it; win_edge[w] = min{e : ceptr[e] >= w kWinSlots} (internal order, m
// past the end), for w = 0..nwin with nwin = ceil(P / kWinSlots).  A
// hyperedge with at most kBigEdge <= kWinSlots pins ends within the window
// after its own.
constexpr int kWinSlots = 64;
__host__ __device__ inline long long num_windows(long long P) { return (P + kWinSlots - 1) / kWinSlots; }

// Kernel-side view of the incidence (passed by value to kernels).
struct IncView {
  int n, m, P;
  const unsigned int* status;
  const int32_t* perm;
  const int32_t* big_idx;
  const int32_t* big_pos;
  const int32_t* win_edge;
  const int32_t* ceptr;
  const int32_t* cpins;
  const double* ew;
  const double* ewh;
  const double* ez;
  const int32_t* vptr;
  const int32_t* vedge;
  const int32_t* vslot;
  const double* dc;
  const double* db;
  const double* inv_dc;
  const double* inv_db;
  const double* wsc;
  const double* totals;
};

inline IncView view(const hef_incidence* h) {
  IncView v;
  v.n = (int)h->n;
  v.m = (int)h->m;
  v.P = (int)h->P;
  v.status = h->status;
  v.perm = h->perm;
  v.big_idx = h->big_idx;
  v.big_pos = h->big_pos;
  v.win_edge = h->win_edge;
  v.ceptr = h->ceptr;
  v.cpins = h->cpins;
  v.ew = h->ew;
  v.ewh = h->ewh;
  v.ez = h->ez;
  v.vptr = h->vptr;
  v.vedge = h->vedge;
  v.vslot = h->vslot;
  v.dc = h->dc;
  v.db = h->db;
  v.inv_dc = h->inv_dc;
  v.inv_db = h->inv_db;
  v.wsc = h->wsc;
  v.totals = h->totals;
  return v;
}

hef_status check_stream_ptrs(const void* p, const char* what);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null when unavailable.
inline PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// The expansion scalars in the arithmetic type of a form (FP64 arrays for
// double, their FP32 copies for float).
template <typename T>
struct ScalView {
  const T* ew;
  const T* ewh;
  const T* ez;
  const T* dc;
  const T* db;
  const T* inv_dc;
  const T* inv_db;
  const T* wsc;
};

inline ScalView<double> scal_view_d(const hef_incidence* h) {
  return {h->ew, h->ewh, h->ez, h->dc, h->db, h->inv_dc, h->inv_db, h->wsc};
}
inline ScalView<float> scal_view_f(const hef_incidence* h) {
  return {h->f_ew, h->f_ewh, h->f_ez, h->f_dc, h->f_db, h->f_inv_dc, h->f_inv_db, h->f_wsc};
}
template <typename T>
inline ScalView<T> scal_view(const hef_incidence* h);
template <>
inline ScalView<double> scal_view<double>(const hef_incidence* h) {
  return scal_view_d(h);
}
template <>
inline ScalView<float> scal_view<float>(const hef_incidence* h) {
  return scal_view_f(h);
}

// Forward tape of the Krylov chains (hef_krylov_basis_tape), read by the
// backward: coefficients as used by the forward, then the unnormalised chain
// vectors u_j (x_j = u_j * inv_nu[j]) for j = 0..k.
struct TapeLayout {
  double* coef;    // (k+1) x 2S x 4: [deflation, deflation (star edges), alpha, beta]
  double* inv_nu;  // (k+1) x 2S
  void* uc;        // (k+1) x n x S
  void* ub;        // (k+1) x (n+m) x S
};

inline size_t carve_tape(void* base, long long n, long long m, int k, int S, size_t esz,
                         TapeLayout* t) {
  Carver c(base);
  t->coef = c.take<double>((size_t)(k + 1) * 2 * S * 4);
  t->inv_nu = c.take<double>((size_t)(k + 1) * 2 * S);
  t->uc = c.take<char>((size_t)(k + 1) * n * S * esz);
  t->ub = c.take<char>((size_t)(k + 1) * (n + m) * S * esz);
  if (!base) t->uc = t->ub = nullptr, t->coef = t->inv_nu = nullptr;
  return c.bytes();
}

// Device-wide scan and sort (incidence.cu), shared by the build and the
// downstream calls.
int scan_tiles(long long N);
// out[0..N] = exclusive scan of in[0..N); out[N] = total.  bsum needs
// scan_tiles(N) + 1 ints (8-byte aligned); counter is zero on entry (and on
// exit); in and out may alias; a bounded wait that expires sets
// HEF_WAIT_TIMEOUT in *err when err is given.
hef_status exclusive_scan(const int* in, int* out, long long N, int* bsum, unsigned int* counter,
                          cudaStream_t st, unsigned int* err = nullptr);
struct SortBufs {
  uint32_t* k_alt;
  int32_t* v_alt;
  unsigned int* counter;  // of the scans (zero between calls)
  int* counts;            // buckets x tiles + 1
  int* bsum;
};
// Buffers of radix_sort for up to N items (the counter is the caller's).
void carve_sort_bufs(Carver& c, long long N, SortBufs* b);
inline int bits_for(long long maxkey) {
  int b = 1;
  while (b < 32 && (1ll << b) <= maxkey) ++b;
  return b;
}
// Sorts (keys, vals) by key, stable (LSD radix); keys < 2^bits.
hef_status radix_sort(uint32_t* keys, int32_t* vals, long long N, int bits, SortBufs b,
                      cudaStream_t st);

// Whether hef_krylov_basis(_tape) calls from this thread may run all Krylov
// steps as one persistent launch (default on).  The persistent grid needs
// every CTA resident at once, so callers that overlap other work on the GPU
// turn it off.
void krylov_allow_persistent(bool on);

// The batched form's Krylov stage: per hypergraph, the starts on its own
// stream (krylov_batch_start, workspace as for hef_krylov_basis); then all
// k steps of every hypergraph in cooperative launches of up to 64
// hypergraphs, each on a share of the CTAs in proportion to `cost`
// (krylov_batch_steps; V, ldv as for hef_krylov_basis).
struct KrylovBatchArg {
  const hef_incidence* inc;
  void* V;
  long long ldv;
  void* ws;
  double cost;
};
hef_status krylov_batch_start(const hef_incidence* inc, int k, int S, int dtype, const double* x0c,
                              const double* x0b, void* ws, cudaStream_t st);
hef_status krylov_batch_steps(const KrylovBatchArg* items, int G, int k, int S, int dtype,
                              cudaStream_t st);
void krylov_force_oversized(bool on);

// Tensor-core (tcgen05, 3xTF32) Gram matrix of an FP32 basis with K + 1 <= 256
// (ortho_tc.cu): G = V^T V (K x K), c = V^T 1; part is per-CTA scratch.
int gram_tc_supported(int K);
size_t gram_tc_part_doubles(long long n, int K);
hef_status gram_tc(const void* V, bool bf16, long long ldv, long long n, int K, double* part,
                   double* G, double* c, int* err, cudaStream_t st);
// Tensor-core in-place apply Q = (V - 1 mu^T) Rinv of an FP32 basis, K <= 256.
int apply_tc_supported(int K);
size_t apply_tc_scratch_floats(int K);
hef_status apply_tc(void* V, bool bf16, long long ldv, long long n, int K, const float* Rinv,
                    int Kp, const float* mu, float* scratch, int* err, cudaStream_t st);

}  // namespace hef
