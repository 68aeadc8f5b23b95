// qpm_host.cu -- error reporting and device queries for the C ABI.
#include <mutex>
#include <string>
#include <vector>

#include "qpm_internal.h"

namespace qpm {

static thread_local std::string t_last_error;

void set_error(const std::string &msg) { t_last_error = msg; }

qpm_status fail(qpm_status s, const std::string &msg) {
  t_last_error = msg;
  return s;
}

qpm_status cuda_fail(cudaError_t e, const char *what) {
  t_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return QPM_ERR_CUDA;
}

int sm_count() {
  static std::mutex mu;
  static std::vector<int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  std::lock_guard<std::mutex> lock(mu);
  if ((int)cache.size() <= dev) cache.resize(dev + 1, 0);
  if (cache[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    cache[dev] = n;
  }
  return cache[dev];
}

}  // namespace qpm

extern "C" const char *qpm_last_error(void) { return qpm::t_last_error.c_str(); }

extern "C" const char *qpm_status_string(qpm_status s) {
  switch (s) {
    case QPM_OK: return "QPM_OK";
    case QPM_ERR_ARG: return "QPM_ERR_ARG";
    case QPM_ERR_CUDA: return "QPM_ERR_CUDA";
    case QPM_ERR_TIMEOUT: return "QPM_ERR_TIMEOUT";
    case QPM_ERR_UNSUPPORTED: return "QPM_ERR_UNSUPPORTED";
    case QPM_ERR_STATE: return "QPM_ERR_STATE";
  }
  return "QPM_ERR_UNKNOWN";
}

extern "C" int32_t qpm_abi_version(void) { return 2; }
