// Library-wide C ABI helpers: error strings and the thread-local message.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace hef {

static thread_local char g_msg[512] = "";

hef_status set_error(hef_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return s;
}

// ------------------------------------------------------------------ tracing

namespace {

std::atomic<unsigned long long> g_launches{0};
std::mutex g_mu;
std::string g_filter;           // kernels whose name contains this are timed
bool g_trace_on = false;
struct Rec {
  const char* name;
  cudaEvent_t a, b;
};
std::vector<Rec> g_recs;        // recorded, not yet read
std::vector<cudaEvent_t> g_pool;
constexpr size_t kMaxRecs = 1 << 16;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

}  // namespace

LaunchTrace::LaunchTrace(const char* name, cudaStream_t s) : slot(-1), st(s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_trace_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_trace_on || g_recs.size() >= kMaxRecs || !strstr(name, g_filter.c_str())) return;
  Rec r{name, take_event(), take_event()};
  if (!r.a || !r.b) return;
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  slot = (int)g_recs.size() - 1;
}

LaunchTrace::~LaunchTrace() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEventRecord(g_recs[slot].b, st);
}

}  // namespace hef

// cudaFuncAttributeMaxDynamicSharedMemorySize is set at most once per kernel,
// device and size (so launches can also be recorded into CUDA graphs).
namespace hef {
namespace {
std::mutex g_attr_mu;
struct AttrRec {
  const void* f;
  int dev;
  int bytes;
};
std::vector<AttrRec> g_attr;
}  // namespace

hef_status ensure_smem(const void* func, int bytes) {
  int dev = 0;
  HEF_CHECK_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_attr_mu);
  for (auto& r : g_attr)
    if (r.f == func && r.dev == dev && r.bytes >= bytes) return HEF_OK;
  HEF_CHECK_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  g_attr.push_back({func, dev, bytes});
  return HEF_OK;
}
}  // namespace hef

extern "C" uint64_t hef_launch_count(void) { return hef::g_launches.load(); }

extern "C" hef_status hef_trace_kernels(const char* name_substring) {
  std::lock_guard<std::mutex> lk(hef::g_mu);
  if (!name_substring || !*name_substring) {
    hef::g_trace_on = false;
    hef::g_filter.clear();
  } else {
    hef::g_trace_on = true;
    hef::g_filter = name_substring;
  }
  return HEF_OK;
}

extern "C" int32_t hef_trace_read(int32_t cap, char* names, int64_t* launches, double* total_ms) {
  std::lock_guard<std::mutex> lk(hef::g_mu);
  std::vector<std::string> nm;
  std::vector<int64_t> cnt;
  std::vector<double> ms;
  for (auto& r : hef::g_recs) {
    float t = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      size_t i = 0;
      while (i < nm.size() && nm[i] != r.name) ++i;
      if (i == nm.size()) {
        nm.push_back(r.name);
        cnt.push_back(0);
        ms.push_back(0.0);
      }
      cnt[i] += 1;
      ms[i] += t;
    }
    hef::g_pool.push_back(r.a);
    hef::g_pool.push_back(r.b);
  }
  hef::g_recs.clear();
  const int32_t k = (int32_t)nm.size();
  for (int32_t i = 0; i < k && i < cap; ++i) {
    if (names) {
      strncpy(names + (size_t)i * 64, nm[i].c_str(), 63);
      names[(size_t)i * 64 + 63] = 0;
    }
    if (launches) launches[i] = cnt[i];
    if (total_ms) total_ms[i] = ms[i];
  }
  return k;
}

extern "C" const char* hef_last_error(void) { return hef::g_msg; }

extern "C" const char* hef_status_string(hef_status s) {
  switch (s) {
    case HEF_OK: return "HEF_OK";
    case HEF_ERR_INVALID_ARG: return "HEF_ERR_INVALID_ARG";
    case HEF_ERR_CUDA: return "HEF_ERR_CUDA";
    case HEF_ERR_WORKSPACE: return "HEF_ERR_WORKSPACE";
    case HEF_ERR_BREAKDOWN: return "HEF_ERR_BREAKDOWN";
    case HEF_ERR_TIMEOUT: return "HEF_ERR_TIMEOUT";
    case HEF_ERR_UNSUPPORTED: return "HEF_ERR_UNSUPPORTED";
    case HEF_ERR_INVALID_INPUT: return "HEF_ERR_INVALID_INPUT";
    case HEF_ERR_BOUNDS: return "HEF_ERR_BOUNDS";
    default: return "HEF_ERR_UNKNOWN";
  }
}

extern "C" int32_t hef_abi_version(void) { return 1; }

extern "C" int32_t hef_debug_checks(void) { return HEF_DEBUG ? 1 : 0; }
