// Error reporting and small runtime helpers of the qmlr library.
#include "common.cuh"

#include <atomic>
#include <map>
#include <mutex>
#include <utility>

namespace qmlr {

static __device__ int g_device_error = 0;

int* device_error_ptr() {
  static std::mutex mu;
  static int* ptrs[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!ptrs[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_error) != cudaSuccess) return nullptr;
    ptrs[dev] = static_cast<int*>(p);
  }
  return ptrs[dev];
}

static thread_local char t_last_error[512] = "";
static std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_last_error, sizeof(t_last_error), fmt, ap);
  va_end(ap);
}

cudaError_t smem_attr_once(const void* func, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> raised;   // (kernel, device) -> bytes
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(func, dev);
  const auto it = raised.find(key);
  if (it != raised.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) raised[key] = bytes;
  return e;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
  return n;
}

}  // namespace qmlr

extern "C" const char* qmlr_version(void) { return "qmlr 0.1 (sm_103a)"; }

extern "C" const char* qmlr_last_error(void) { return qmlr::t_last_error; }

extern "C" int qmlr_device_status(void* stream, int32_t* host_code) {
  QMLR_REQUIRE(host_code, "host_code is NULL");
  QMLR_CUDA_TRY(cudaStreamSynchronize(qmlr::as_stream(stream)));
  int code = 0, zero = 0;
  QMLR_CUDA_TRY(cudaMemcpyFromSymbol(&code, qmlr::g_device_error, sizeof(int)));
  QMLR_CUDA_TRY(cudaMemcpyToSymbol(qmlr::g_device_error, &zero, sizeof(int)));
  *host_code = code;
  if (code) {
    qmlr::set_error("device-side input error code %d", code);
    return QMLR_EDEVICE;
  }
  return QMLR_OK;
}

extern "C" int64_t qmlr_launch_count(void) { return qmlr::g_launches.load(); }
