// Status strings, the thread-local error message and the launch counter.
#include <string>

#include "wq_internal.h"

namespace {
thread_local std::string g_last_error;
std::atomic<int64_t> g_launches{0};
}  // namespace

namespace wq {

wq_status set_error(wq_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

wq_status cuda_error(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // clear a non-sticky error so later calls can proceed
  return WQ_ERR_CUDA;
}

void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

}  // namespace wq

extern "C" const char* wq_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* wq_status_string(wq_status status) {
  switch (status) {
    case WQ_OK: return "WQ_OK";
    case WQ_ERR_INVALID_ARG: return "WQ_ERR_INVALID_ARG";
    case WQ_ERR_UNSUPPORTED: return "WQ_ERR_UNSUPPORTED";
    case WQ_ERR_SINGULAR_RULE: return "WQ_ERR_SINGULAR_RULE";
    case WQ_ERR_BAD_GEOMETRY: return "WQ_ERR_BAD_GEOMETRY";
    case WQ_ERR_OOM: return "WQ_ERR_OOM";
    case WQ_ERR_CUDA: return "WQ_ERR_CUDA";
    case WQ_ERR_TIMEOUT: return "WQ_ERR_TIMEOUT";
    case WQ_ERR_INJECTED: return "WQ_ERR_INJECTED";
    case WQ_ERR_NONFINITE: return "WQ_ERR_NONFINITE";
  }
  return "WQ_ERR_UNKNOWN";
}

extern "C" int64_t wq_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }
