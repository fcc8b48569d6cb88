// Batched form: Algorithm 1 on many independent hypergraphs of uneven sizes
// (e.g. every level of a multilevel hierarchy) in one call.
//
// Each hypergraph runs the whole path (incidence, Krylov basis, CholQR2,
// scoring) as its own chain of launches on one stream of a per-device pool;
// the chains of different hypergraphs overlap on the GPU.  The call forks
// from the caller's stream with an event and joins back with one event per
// pool stream, so the whole batch can be captured as one CUDA graph.  Which
// hypergraph runs on which pool stream (the schedule) and how many streams
// take part come from a greedy longest-first assignment of estimated costs,
// and hef_batch_autotune picks the stream count (and with it the schedule)
// by timing the candidates.
#include <algorithm>
#include <mutex>
#include <numeric>
#include <vector>

#include "internal.h"

namespace hef {

namespace {

constexpr int kMaxStreams = 16;
constexpr int kMaxDevices = 64;

struct StreamPool {
  bool ready = false;
  cudaStream_t s[kMaxStreams];
  cudaEvent_t fork;
  cudaEvent_t join[kMaxStreams];
};

std::mutex g_pool_mu;
StreamPool g_pool[kMaxDevices];

// The current device's pool, created on first use (outside stream capture).
hef_status device_pool(StreamPool** out) {
  int dev = 0;
  HEF_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(HEF_ERR_UNSUPPORTED, "batched call: device %d >= %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_pool_mu);
  StreamPool& p = g_pool[dev];
  if (!p.ready) {
    for (int i = 0; i < kMaxStreams; ++i) {
      HEF_CHECK_CUDA(cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking));
      HEF_CHECK_CUDA(cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming));
    }
    HEF_CHECK_CUDA(cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming));
    p.ready = true;
  }
  *out = &p;
  return HEF_OK;
}

struct ItemSizes {
  size_t inc, kry, V, ortho, score;
  long long ldv;
};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

void item_sizes(const hef_batch_item& it, int k, int S, int dtype, ItemSizes* z) {
  hef_incidence shape;  // only n, m, P are read by the size queries
  shape.n = it.n, shape.m = it.m, shape.P = it.P;
  const int K = 2 * k * S;
  const size_t esz = dtype == HEF_F64 ? 8 : (dtype == HEF_BF16 ? 2 : 4);
  z->ldv = (long long)(((size_t)K * esz + 15) / 16 * 16 / esz);
  z->inc = align256(hef_incidence_workspace_bytes(it.n, it.m, it.P));
  z->kry = align256(hef_krylov_workspace_bytes(&shape, k, S, dtype));
  z->V = align256((size_t)it.n * z->ldv * esz);
  z->ortho = align256(hef_orthonormalize_workspace_bytes(it.n, K, dtype));
  z->score = align256(hef_edge_resistance_workspace_bytes(&shape, K));
}

size_t item_bytes(const ItemSizes& z) { return z.inc + z.kry + z.V + z.ortho + z.score; }

// Work estimate of one hypergraph (bytes moved, roughly): Krylov passes over
// the incidence and chain blocks, plus the Gram/apply sweeps over V.
double item_cost(const hef_batch_item& it, int k, int S) {
  const double K = 2.0 * k * S;
  return (double)k * (8.0 * it.P + 16.0 * S * (2.0 * it.n + it.m)) + 16.0 * it.n * K + 8.0 * it.P;
}

// Greedy longest-first assignment onto `ns` streams (least loaded first).
void lpt_schedule(const hef_batch_item* items, int G, int k, int S, int ns, int32_t* sched) {
  std::vector<int> order(G);
  std::iota(order.begin(), order.end(), 0);
  std::vector<double> cost(G);
  for (int g = 0; g < G; ++g) cost[g] = item_cost(items[g], k, S);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<double> load(ns, 0.0);
  for (int g : order) {
    int best = 0;
    for (int s = 1; s < ns; ++s)
      if (load[s] < load[best]) best = s;
    sched[g] = best;
    load[best] += cost[g];
  }
}

hef_status check_items(const hef_batch_item* items, int G, int k, int S, int dtype, const char* fn) {
  if (!items || G < 1) return set_error(HEF_ERR_INVALID_ARG, "%s: need G >= 1 items", fn);
  if (dtype != HEF_F64 && dtype != HEF_F32 && dtype != HEF_BF16)
    return set_error(HEF_ERR_INVALID_ARG, "%s: dtype must be HEF_F64, HEF_F32 or HEF_BF16", fn);
  if (k < 1 || S < 1 || S > 16 || (S & (S - 1)) || 2ll * k * S > 512)
    return set_error(HEF_ERR_UNSUPPORTED, "%s: need k >= 1, S in {1,2,4,8,16}, 2kS <= 512", fn);
  for (int g = 0; g < G; ++g) {
    const hef_batch_item& it = items[g];
    if (it.n < 1 || it.m < 0 || it.P < 0 || !it.eptr || (it.P > 0 && !it.pins) ||
        (it.m > 0 && !it.w) || !it.x0_clique || !it.x0_star || !it.R_out)
      return set_error(HEF_ERR_INVALID_ARG, "%s: item %d has a bad size or a NULL array", fn, g);
  }
  return HEF_OK;
}

// One hypergraph's whole path on stream st, scratch from base.
hef_status run_item(const hef_batch_item& it, int k, int S, int dtype, int clique_mode,
                    const ItemSizes& z, char* base, cudaStream_t st) {
  const int K = 2 * k * S;
  char* p = base;
  void* ws_inc = p;
  p += z.inc;
  void* ws_kry = p;
  p += z.kry;
  void* V = p;
  p += z.V;
  void* ws_ortho = p;
  p += z.ortho;
  void* ws_score = p;
  hef_incidence* inc = nullptr;
  hef_status s = hef_build_incidence(it.n, it.m, it.P, it.eptr, it.pins, it.w, clique_mode, ws_inc,
                                     z.inc, st, &inc);
  if (s) return s;
  s = hef_krylov_basis(inc, k, S, dtype, it.x0_clique, it.x0_star, V, z.ldv, ws_kry, z.kry, st);
  if (!s) s = hef_orthonormalize(it.n, K, dtype, V, z.ldv, nullptr, nullptr, ws_ortho, z.ortho, st);
  if (!s)
    s = hef_edge_resistance(inc, V, z.ldv, K, dtype, HEF_REDUCE_MAX, it.R_out, it.QH_out,
                            it.argvec, it.pmax, it.pmin, ws_score, z.score, st);
  if (!s && it.status_out &&
      cudaMemcpyAsync(it.status_out, inc->status, 2 * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                      st) != cudaSuccess)
    s = set_error(HEF_ERR_CUDA, "batched call: status copy failed");
  // kernels took the incidence by value: the host handle can go now
  hef_free_incidence(inc);
  return s;
}

// Krylov stage of the batched form (a per-thread setting, see
// hef_set_batch_krylov_form): 1 = all hypergraphs' steps in one cooperative
// launch, 0 = per-step launches of each hypergraph on its stream.
thread_local int t_batch_form = 1;

// The batched path with the one-launch Krylov stage: per item on its stream,
// the incidence and the Krylov starts; join; all Krylov steps in one
// cooperative launch on `stream`; fork; per item, CholQR2 and scoring.
hef_status run_batch_one_launch(const hef_batch_item* items, int G, int k, int S, int dtype,
                                int clique_mode, const int32_t* sched, int ns, char* base,
                                const std::vector<size_t>& off, const std::vector<ItemSizes>& zs,
                                const std::vector<int>& order, const std::vector<double>& cost,
                                StreamPool* pool, cudaStream_t stream) {
  const int K = 2 * k * S;
  std::vector<hef_incidence*> incs(G, nullptr);
  hef_status first = HEF_OK;
  auto join = [&]() -> hef_status {
    for (int i = 0; i < ns; ++i) {
      HEF_CHECK_CUDA(cudaEventRecord(pool->join[i], pool->s[i]));
      HEF_CHECK_CUDA(cudaStreamWaitEvent(stream, pool->join[i], 0));
    }
    return HEF_OK;
  };
  for (int g : order) {
    const ItemSizes& z = zs[g];
    char* p = base + off[g];
    const hef_batch_item& it = items[g];
    cudaStream_t st = pool->s[sched[g]];
    hef_status r = hef_build_incidence(it.n, it.m, it.P, it.eptr, it.pins, it.w, clique_mode, p,
                                       z.inc, st, &incs[g]);
    if (!r) r = krylov_batch_start(incs[g], k, S, dtype, it.x0_clique, it.x0_star, p + z.inc, st);
    if (r && !first) first = r;
  }
  if (hef_status r = join()) first = first ? first : r;
  if (!first) {
    std::vector<KrylovBatchArg> args(G);
    for (int g = 0; g < G; ++g)
      args[g] = KrylovBatchArg{incs[g], base + off[g] + zs[g].inc + zs[g].kry, zs[g].ldv,
                               base + off[g] + zs[g].inc, cost[g]};
    first = krylov_batch_steps(args.data(), G, k, S, dtype, stream);
  }
  cudaError_t fe = cudaEventRecord(pool->fork, stream);
  for (int i = 0; i < ns && fe == cudaSuccess; ++i) fe = cudaStreamWaitEvent(pool->s[i], pool->fork, 0);
  if (fe != cudaSuccess && !first) first = set_error(HEF_ERR_CUDA, "batched call: fork failed");
  for (int g : order) {
    const ItemSizes& z = zs[g];
    char* p = base + off[g];
    const hef_batch_item& it = items[g];
    cudaStream_t st = pool->s[sched[g]];
    if (!first && incs[g]) {
      void* V = p + z.inc + z.kry;
      hef_status r = hef_orthonormalize(it.n, K, dtype, V, z.ldv, nullptr, nullptr,
                                        p + z.inc + z.kry + z.V, z.ortho, st);
      if (!r)
        r = hef_edge_resistance(incs[g], V, z.ldv, K, dtype, HEF_REDUCE_MAX, it.R_out, it.QH_out,
                                it.argvec, it.pmax, it.pmin, p + z.inc + z.kry + z.V + z.ortho,
                                z.score, st);
      if (!r && it.status_out &&
          cudaMemcpyAsync(it.status_out, incs[g]->status, 2 * sizeof(uint32_t),
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        r = set_error(HEF_ERR_CUDA, "batched call: status copy failed");
      if (r && !first) first = r;
    }
    if (incs[g]) hef_free_incidence(incs[g]);
  }
  if (hef_status r = join()) first = first ? first : r;
  return first;
}

hef_status run_batch(const hef_batch_item* items, int G, int k, int S, int dtype, int clique_mode,
                     const int32_t* sched, int ns, void* workspace, cudaStream_t stream) {
  StreamPool* pool = nullptr;
  hef_status s = device_pool(&pool);
  if (s) return s;
  HEF_CHECK_CUDA(cudaEventRecord(pool->fork, stream));
  for (int i = 0; i < ns; ++i) HEF_CHECK_CUDA(cudaStreamWaitEvent(pool->s[i], pool->fork, 0));
  char* base = static_cast<char*>(workspace);
  hef_status first = HEF_OK;
  // launch in longest-first order so each stream starts with its largest item
  std::vector<int> order(G);
  std::iota(order.begin(), order.end(), 0);
  std::vector<double> cost(G);
  std::vector<size_t> off(G + 1, 0);
  std::vector<ItemSizes> zs(G);
  for (int g = 0; g < G; ++g) {
    cost[g] = item_cost(items[g], k, S);
    item_sizes(items[g], k, S, dtype, &zs[g]);
    off[g + 1] = off[g] + item_bytes(zs[g]);
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  if (t_batch_form == 1)
    return run_batch_one_launch(items, G, k, S, dtype, clique_mode, sched, ns, base, off, zs, order,
                                cost, pool, stream);
  // items overlap on the GPU: one-launch Krylov grids could not all be resident
  krylov_allow_persistent(false);
  for (int g : order) {
    const int si = sched[g];
    hef_status r = run_item(items[g], k, S, dtype, clique_mode, zs[g], base + off[g], pool->s[si]);
    if (r && !first) first = r;
  }
  krylov_allow_persistent(true);
  // join every stream that took part, also after an error (a capture must
  // end with all forked streams joined)
  for (int i = 0; i < ns; ++i) {
    HEF_CHECK_CUDA(cudaEventRecord(pool->join[i], pool->s[i]));
    HEF_CHECK_CUDA(cudaStreamWaitEvent(stream, pool->join[i], 0));
  }
  return first;
}

}  // namespace

}  // namespace hef

using namespace hef;

extern "C" size_t hef_batch_workspace_bytes(const hef_batch_item* items, int32_t G, int32_t k,
                                            int32_t S, int32_t dtype) {
  if (check_items(items, G, k, S, dtype, "hef_batch_workspace_bytes")) return 0;
  size_t total = 0;
  for (int g = 0; g < G; ++g) {
    ItemSizes z;
    item_sizes(items[g], k, S, dtype, &z);
    total += item_bytes(z);
  }
  return total;
}

extern "C" hef_status hef_batch_schedule(const hef_batch_item* items, int32_t G, int32_t k,
                                         int32_t S, int32_t nstreams, int32_t* schedule) {
  if (hef_status s = check_items(items, G, k, S, HEF_F32, "hef_batch_schedule")) return s;
  if (nstreams < 1 || nstreams > kMaxStreams || !schedule)
    return set_error(HEF_ERR_INVALID_ARG, "hef_batch_schedule: need 1 <= nstreams <= %d and a schedule array",
                     kMaxStreams);
  lpt_schedule(items, G, k, S, nstreams, schedule);
  return HEF_OK;
}

extern "C" hef_status hef_resistance_batched(const hef_batch_item* items, int32_t G, int32_t k,
                                             int32_t S, int32_t dtype, int32_t clique_mode,
                                             const int32_t* schedule, int32_t nstreams,
                                             void* workspace, size_t workspace_bytes, void* stream) {
  HEF_NVTX("hef_resistance_batched");
  static const char* fn = "hef_resistance_batched";
  if (hef_status s = check_items(items, G, k, S, dtype, fn)) return s;
  if (nstreams < 1 || nstreams > kMaxStreams)
    return set_error(HEF_ERR_INVALID_ARG, "%s: need 1 <= nstreams <= %d", fn, kMaxStreams);
  const size_t need = hef_batch_workspace_bytes(items, G, k, S, dtype);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return set_error(HEF_ERR_WORKSPACE, "%s: workspace needs %zu bytes (256-aligned)", fn, need);
  std::vector<int32_t> sched(G);
  if (schedule) {
    for (int g = 0; g < G; ++g) {
      if (schedule[g] < 0 || schedule[g] >= nstreams)
        return set_error(HEF_ERR_INVALID_ARG, "%s: schedule[%d] = %d outside [0, %d)", fn, g,
                         schedule[g], nstreams);
      sched[g] = schedule[g];
    }
  } else {
    lpt_schedule(items, G, k, S, nstreams, sched.data());
  }
  return run_batch(items, G, k, S, dtype, clique_mode, sched.data(), nstreams, workspace,
                   static_cast<cudaStream_t>(stream));
}

extern "C" hef_status hef_batch_autotune(const hef_batch_item* items, int32_t G, int32_t k,
                                         int32_t S, int32_t dtype, int32_t clique_mode,
                                         void* workspace, size_t workspace_bytes, void* stream,
                                         int32_t* nstreams_out, int32_t* schedule_out,
                                         float* ms_out) {
  static const char* fn = "hef_batch_autotune";
  if (hef_status s = check_items(items, G, k, S, dtype, fn)) return s;
  if (!nstreams_out || !schedule_out)
    return set_error(HEF_ERR_INVALID_ARG, "%s: NULL output", fn);
  const size_t need = hef_batch_workspace_bytes(items, G, k, S, dtype);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return set_error(HEF_ERR_WORKSPACE, "%s: workspace needs %zu bytes (256-aligned)", fn, need);
  // candidates run on a private stream after the caller's work, each captured
  // as a graph and timed over three replays (host launch cost excluded)
  HEF_CHECK_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  cudaStream_t ts = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  HEF_CHECK_CUDA(cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking));
  hef_status status = HEF_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    status = set_error(HEF_ERR_CUDA, "%s: event creation failed", fn);
  std::vector<int32_t> sched(G), best_sched(G);
  float best = -1.0f;
  int best_ns = 1, best_form = t_batch_form;
  const int form0 = t_batch_form;
  for (int cand = 0; cand < 2 * 5 && status == HEF_OK; ++cand) {
    const int form = cand < 5 ? 1 : 0, ns = 1 << (cand % 5);
    if (ns > 1 && ns > G) continue;
    t_batch_form = form;
    lpt_schedule(items, G, k, S, ns, sched.data());
    status = run_batch(items, G, k, S, dtype, clique_mode, sched.data(), ns, workspace, ts);
    if (status) break;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      status = set_error(HEF_ERR_CUDA, "%s: capture failed", fn);
      break;
    }
    hef_status r = run_batch(items, G, k, S, dtype, clique_mode, sched.data(), ns, workspace, ts);
    const cudaError_t ce = cudaStreamEndCapture(ts, &graph);
    if (r || ce != cudaSuccess ||
        cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      status = r ? r : set_error(HEF_ERR_CUDA, "%s: graph capture of %d streams failed", fn, ns);
      if (graph) cudaGraphDestroy(graph);
      break;
    }
    float ms = -1.0f;
    if (cudaGraphLaunch(exec, ts) != cudaSuccess || cudaEventRecord(e0, ts) != cudaSuccess ||
        cudaGraphLaunch(exec, ts) != cudaSuccess || cudaGraphLaunch(exec, ts) != cudaSuccess ||
        cudaGraphLaunch(exec, ts) != cudaSuccess || cudaEventRecord(e1, ts) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      status = set_error(HEF_ERR_CUDA, "%s: timing the graph of %d streams failed", fn, ns);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (status) break;
    ms /= 3.0f;
    if (best < 0.0f || ms < best) best = ms, best_ns = ns, best_sched = sched, best_form = form;
  }
  t_batch_form = status ? form0 : best_form;  // the caller's thread keeps the faster form
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(ts);
  cudaStreamDestroy(ts);
  if (status) return status;
  *nstreams_out = best_ns;
  std::copy(best_sched.begin(), best_sched.end(), schedule_out);
  if (ms_out) *ms_out = best;
  return HEF_OK;
}

extern "C" hef_status hef_set_batch_krylov_form(int32_t form) {
  if (form != 0 && form != 1)
    return set_error(HEF_ERR_INVALID_ARG, "hef_set_batch_krylov_form: form must be 0 or 1");
  t_batch_form = form;
  return HEF_OK;
}

extern "C" int32_t hef_batch_krylov_form(void) { return t_batch_form; }
