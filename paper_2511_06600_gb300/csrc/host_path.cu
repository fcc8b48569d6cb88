// Algorithm 1 end to end from host arrays (hef_resistance_host): the copies
// in (the start vectors on a side stream, overlapping the incidence build),
// the four calls of the path, the scores back, one synchronisation.  A C
// caller that holds its hypergraph in host memory needs nothing else but a
// device workspace.
#include <cstring>

#include "internal.h"

namespace hef {
namespace {

// A side stream and two events per calling thread (created on first use):
// the start vectors, which only the Krylov stage reads, are copied on the
// side stream while the incidence is built on the caller's stream.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  int device = -1;
};
thread_local SideStream t_side;

cudaError_t side_stream(SideStream** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  SideStream& s = t_side;
  if (s.device != dev) {
    if (s.s) {  // created for another device: made again for this one
      cudaStreamDestroy(s.s);
      cudaEventDestroy(s.fork);
      cudaEventDestroy(s.join);
      s = SideStream{};
    }
    if ((e = cudaStreamCreateWithFlags(&s.s, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&s.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&s.join, cudaEventDisableTiming)) != cudaSuccess) return e;
    s.device = dev;
  }
  *out = &s;
  return cudaSuccess;
}

struct HostWs {
  int64_t* eptr;
  int32_t* pins;
  double* w;
  double* x0c;
  double* x0b;
  double* R;
  int32_t* rank;
  void* inc;
  size_t inc_b;
  void* V;
  long long ldv;
  void* kry;
  size_t kry_b;
  void* ortho;
  size_t ortho_b;
  void* score;
  size_t score_b;
};

size_t carve_host(void* base, long long n, long long m, long long P, int k, int S, int dtype,
                  HostWs* h) {
  hef_incidence shape;  // the size queries read only n, m, P
  shape.n = n, shape.m = m, shape.P = P;
  const int K = 2 * k * S;
  const size_t esz = dtype == HEF_F64 ? 8 : 4;
  Carver c(base);
  h->eptr = c.take<int64_t>(m + 1);
  h->pins = c.take<int32_t>(P > 0 ? P : 1);
  h->w = c.take<double>(m > 0 ? m : 1);
  h->x0c = c.take<double>((size_t)(n > 0 ? n : 1) * S);
  h->x0b = c.take<double>((size_t)(n + m > 0 ? n + m : 1) * S);
  h->R = c.take<double>(m > 0 ? m : 1);
  h->rank = c.take<int32_t>(1);
  h->inc_b = hef_incidence_workspace_bytes(n, m, P);
  h->inc = c.take<char>(h->inc_b);
  h->ldv = (long long)(((size_t)K * esz + 15) / 16 * 16 / esz);
  h->V = c.take<char>((size_t)(n > 0 ? n : 1) * h->ldv * esz);
  h->kry_b = hef_krylov_workspace_bytes(&shape, k, S, dtype);
  h->kry = c.take<char>(h->kry_b);
  h->ortho_b = hef_orthonormalize_workspace_bytes(n > 0 ? n : 1, K, dtype);
  h->ortho = c.take<char>(h->ortho_b);
  h->score_b = hef_edge_resistance_workspace_bytes(&shape, K);
  h->score = c.take<char>(h->score_b);
  return c.bytes();
}

}  // namespace
}  // namespace hef

using namespace hef;

extern "C" size_t hef_resistance_host_workspace_bytes(int64_t n, int64_t m, int64_t P, int32_t k,
                                                      int32_t S, int32_t dtype) {
  if (n < 1 || m < 0 || P < 0 || k < 1 || S < 1 || (dtype != HEF_F64 && dtype != HEF_F32))
    return 0;
  HostWs h;
  return carve_host(nullptr, n, m, P, k, S, dtype, &h);
}

namespace hef {
namespace {

// The call's device work on stream st, in order: the copies in (the starts on
// the side stream, joined before the Krylov stage), the four calls of the
// path and the copy of R out.  *inc receives the incidence handle (also on
// failure, when one was built).
hef_status enqueue_path(const HostWs& h, int64_t n, int64_t m, int64_t P, const int64_t* eptr,
                        const int32_t* pins, const double* w, const double* x0_clique,
                        const double* x0_star, int32_t k, int32_t S, int32_t dtype,
                        int32_t clique_mode, double* R_out, cudaStream_t st, hef_incidence** inc) {
  static const char* fn = "hef_resistance_host";
  const int K = 2 * k * S;
  *inc = nullptr;
  HEF_CHECK_CUDA(cudaMemcpyAsync(h.eptr, eptr, (m + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  if (P > 0)
    HEF_CHECK_CUDA(cudaMemcpyAsync(h.pins, pins, P * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  if (m > 0) HEF_CHECK_CUDA(cudaMemcpyAsync(h.w, w, m * sizeof(double), cudaMemcpyHostToDevice, st));
  // the starts on the side stream, after everything already queued on st
  // (the workspace may still be in use by earlier work), joined before the
  // Krylov stage
  SideStream* side = nullptr;
  HEF_CHECK_CUDA(side_stream(&side));
  HEF_CHECK_CUDA(cudaEventRecord(side->fork, st));
  HEF_CHECK_CUDA(cudaStreamWaitEvent(side->s, side->fork, 0));
  HEF_CHECK_CUDA(cudaMemcpyAsync(h.x0c, x0_clique, (size_t)n * S * sizeof(double),
                                 cudaMemcpyHostToDevice, side->s));
  HEF_CHECK_CUDA(cudaMemcpyAsync(h.x0b, x0_star, (size_t)(n + m) * S * sizeof(double),
                                 cudaMemcpyHostToDevice, side->s));
  HEF_CHECK_CUDA(cudaEventRecord(side->join, side->s));
  hef_status s = hef_build_incidence(n, m, P, h.eptr, h.pins, h.w, clique_mode, h.inc, h.inc_b,
                                     st, inc);
  if (s) {
    cudaStreamWaitEvent(st, side->join, 0);  // the copies finish before the caller reuses buffers
    return s;
  }
  HEF_CHECK_CUDA(cudaStreamWaitEvent(st, side->join, 0));
  s = hef_krylov_basis(*inc, k, S, dtype, h.x0c, h.x0b, h.V, h.ldv, h.kry, h.kry_b, st);
  if (!s)
    s = hef_orthonormalize(n, K, dtype, h.V, h.ldv, nullptr, h.rank, h.ortho, h.ortho_b, st);
  if (!s)
    s = hef_edge_resistance(*inc, h.V, h.ldv, K, dtype, HEF_REDUCE_MAX, h.R, nullptr, nullptr,
                            nullptr, nullptr, h.score, h.score_b, st);
  if (!s && m > 0) {
    const cudaError_t e = cudaMemcpyAsync(R_out, h.R, m * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) s = set_error(HEF_ERR_CUDA, "%s: copy of R failed: %s", fn, cudaGetErrorString(e));
  }
  return s;
}

// The rank of the basis and the incidence's status, after the work on st:
// synchronises st.
hef_status finish_call(const HostWs& h, const hef_incidence* inc, cudaStream_t st) {
  static const char* fn = "hef_resistance_host";
  int32_t rank = 0;
  const cudaError_t e = cudaMemcpyAsync(&rank, h.rank, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess)
    return set_error(HEF_ERR_CUDA, "%s: copy of the rank failed: %s", fn, cudaGetErrorString(e));
  // synchronises the stream; device-side validation and waits are reported here
  hef_status s = hef_incidence_check(inc, st, nullptr, nullptr);
  if (!s && rank < 0) s = set_error(HEF_ERR_TIMEOUT, "%s: a tensor-core wait timed out", fn);
  return s;
}

// Replay of a repeated call as one CUDA graph.  A caller that scores through
// the same buffers again (the same host arrays, workspace, sizes, form and
// stream) would otherwise pay the launch gaps of about forty dependent
// launches every time: the second such call in a row captures its device
// work into a graph on a private stream, and later calls launch that graph
// on the caller's stream.  The graph reads the host arrays when it runs, so
// new contents in the same buffers are scored.  Only page-locked host arrays
// can be copied inside a graph: calls with pageable arrays always run
// eagerly.  One graph per calling thread; any other call replaces it.
struct GraphKey {
  int device;
  int64_t n, m, P;
  int32_t k, S, dtype, clique_mode;
  const void* host[6];
  void* workspace;
  size_t workspace_bytes;
  void* stream;
  bool operator==(const GraphKey& o) const { return memcmp(this, &o, sizeof(GraphKey)) == 0; }
};
struct HostGraph {
  GraphKey key;
  int calls = 0;                  // calls with this key in a row
  bool no_graph = false;          // this key's work could not be captured
  cudaStream_t cap = nullptr;     // private capture stream (of device cap_device)
  int cap_device = -1;
  cudaGraphExec_t exec = nullptr;
  hef_incidence* inc = nullptr;   // the handle the captured kernels were built with
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    if (inc) hef_free_incidence(inc);
    exec = nullptr;
    inc = nullptr;
    calls = 0;
    no_graph = false;
  }
};
thread_local HostGraph t_graph;

bool page_locked(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

}  // namespace
}  // namespace hef

extern "C" hef_status hef_resistance_host(int64_t n, int64_t m, int64_t P, const int64_t* eptr,
                                          const int32_t* pins, const double* w,
                                          const double* x0_clique, const double* x0_star,
                                          int32_t k, int32_t S, int32_t dtype,
                                          int32_t clique_mode, double* R_out, void* workspace,
                                          size_t workspace_bytes, void* stream) {
  HEF_NVTX("hef_resistance_host (Algorithm 1 from host arrays)");
  static const char* fn = "hef_resistance_host";
  const size_t need = hef_resistance_host_workspace_bytes(n, m, P, k, S, dtype);
  if (!need) return set_error(HEF_ERR_INVALID_ARG, "%s: bad sizes, k, S or dtype", fn);
  if (!eptr || (P > 0 && !pins) || (m > 0 && (!w || !R_out)) || !x0_clique || !x0_star)
    return set_error(HEF_ERR_INVALID_ARG, "%s: NULL host array", fn);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need)
    return set_error(HEF_ERR_WORKSPACE, "%s: workspace needs %zu bytes (256-aligned)", fn, need);
  HostWs h;
  carve_host(workspace, n, m, P, k, S, dtype, &h);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  GraphKey key;
  memset(&key, 0, sizeof(key));
  HEF_CHECK_CUDA(cudaGetDevice(&key.device));
  key.n = n, key.m = m, key.P = P, key.k = k, key.S = S, key.dtype = dtype;
  key.clique_mode = clique_mode;
  const void* host[6] = {eptr, pins, w, x0_clique, x0_star, R_out};
  for (int i = 0; i < 6; ++i) key.host[i] = host[i];
  key.workspace = workspace, key.workspace_bytes = workspace_bytes, key.stream = stream;
  HostGraph& G = t_graph;
  if (!(G.key == key)) {
    G.reset();
    G.key = key;
  }
  if (G.exec) {  // a replay
    HEF_CHECK_CUDA(cudaGraphLaunch(G.exec, st));
    return finish_call(h, G.inc, st);
  }
  ++G.calls;
  bool pinned = G.calls >= 2 && !G.no_graph;
  for (int i = 0; i < 6 && pinned; ++i)
    if (host[i] && !page_locked(host[i])) pinned = false;
  if (pinned) {  // the second call in a row: capture, then launch
    if (G.cap && G.cap_device != key.device) {  // made for another device
      cudaStreamDestroy(G.cap);
      G.cap = nullptr;
    }
    if (!G.cap) {
      if (cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking) == cudaSuccess) {
        G.cap_device = key.device;
      } else {
        (void)cudaGetLastError();
        G.cap = nullptr;
      }
    }
    G.no_graph = true;  // unless the capture below succeeds
    cudaGraph_t graph = nullptr;
    hef_incidence* inc = nullptr;
    if (G.cap && cudaStreamBeginCapture(G.cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const hef_status s = enqueue_path(h, n, m, P, eptr, pins, w, x0_clique, x0_star, k, S,
                                        dtype, clique_mode, R_out, G.cap, &inc);
      const cudaError_t e = cudaStreamEndCapture(G.cap, &graph);
      if (s == HEF_OK && e == cudaSuccess && graph &&
          cudaGraphInstantiate(&G.exec, graph, 0) == cudaSuccess) {
        cudaGraphDestroy(graph);
        G.inc = inc;
        G.no_graph = false;
        HEF_CHECK_CUDA(cudaGraphLaunch(G.exec, st));
        return finish_call(h, G.inc, st);
      }
      // not capturable here: the eager path below
      if (graph) cudaGraphDestroy(graph);
      if (inc) hef_free_incidence(inc);
      G.exec = nullptr;
      (void)cudaGetLastError();
    }
  }
  hef_incidence* inc = nullptr;
  hef_status s = enqueue_path(h, n, m, P, eptr, pins, w, x0_clique, x0_star, k, S, dtype,
                              clique_mode, R_out, st, &inc);
  if (!s) s = finish_call(h, inc, st);
  if (inc) hef_free_incidence(inc);
  return s;
}
