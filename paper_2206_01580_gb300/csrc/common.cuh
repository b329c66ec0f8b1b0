// Internal helpers shared by the qmlr CUDA sources (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstdarg>
#include <string>
#include <algorithm>
#include <cmath>

#include "qmlr.h"

namespace qmlr {

// Per-thread message behind qmlr_last_error().
void set_error(const char* fmt, ...);

// Device-side error word: kernels that meet an input they cannot handle
// (a molecule larger than the launch was sized for, an element index out of
// range) skip that work item and record the first such code in the word whose
// device address device_error_ptr() returns (one word per device, passed to
// the kernels as an argument).
int* device_error_ptr();

enum DeviceError : int {
  DEV_OK = 0,
  DEV_MOL_TOO_LARGE = 1,
  DEV_BAD_ELEMENT = 2,
  DEV_BAD_INDEX = 3,
  DEV_TIMEOUT = 4,
  DEV_NOT_SPD = 5,
  DEV_RANGE = 6,
};

__device__ __forceinline__ void record_device_error(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

#define QMLR_CUDA_TRY(expr)                                                     \
  do {                                                                          \
    cudaError_t _e = (expr);                                                    \
    if (_e != cudaSuccess) {                                                    \
      ::qmlr::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), \
                        __FILE__, __LINE__);                                    \
      return QMLR_ECUDA;                                                        \
    }                                                                           \
  } while (0)

#define QMLR_REQUIRE(cond, ...)                                                 \
  do {                                                                          \
    if (!(cond)) {                                                              \
      ::qmlr::set_error(__VA_ARGS__);                                           \
      return QMLR_EINVAL;                                                       \
    }                                                                           \
  } while (0)

// Number of kernels the library has launched (qmlr_launch_count()).
void count_launch();

// Launch check: counts the launch, reports the launch error (if any) and
// returns QMLR_ECUDA.
#define QMLR_LAUNCH_CHECK()                                                     \
  do {                                                                          \
    ::qmlr::count_launch();                                                     \
    cudaError_t _e = cudaGetLastError();                                        \
    if (_e != cudaSuccess) {                                                    \
      ::qmlr::set_error("kernel launch failed: %s (%s:%d)",                     \
                        cudaGetErrorString(_e), __FILE__, __LINE__);            \
      return QMLR_ECUDA;                                                        \
    }                                                                           \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool is_pow2(long v) { return v > 0 && (v & (v - 1)) == 0; }

inline int rep_dim_of(const qmlr_fchl19_params& p) {
  return p.n_el * p.n2 + p.n_el * (p.n_el + 1) / 2 * p.n3 * 2 * p.nfourier;
}

int validate_params(const qmlr_fchl19_params* p);

int sm_count();

// Raises the dynamic shared-memory limit of a kernel to `bytes` on the current
// device, once per (kernel, device) pair; safe to call from several host threads.
cudaError_t smem_attr_once(const void* func, int bytes);

}  // namespace qmlr
