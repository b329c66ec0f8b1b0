// Throughput of single functional units on this GPU (roofline denominators of
// the ALU-bound kernels): every thread runs a fixed count of independent
// operations of one kind, the grid covers 8 CTAs of 256 threads per SM, and
// the rate is operations per second from CUDA events over 5 launches after a
// warm-up. All loops are bounded and all stores in bounds.
#include "common.cuh"

namespace qmlr {
namespace ur {

constexpr int kIters = 2048;

__global__ void dfma_kernel(double* out, double a, double b) {
  double x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = threadIdx.x + j;
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  }
  double s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int OP>   // 0: fma, 1: add, 2: __expf, 3: __sinf, 4: shuffle
__global__ void f32_kernel(float* out, float a, float b) {
  constexpr int N = OP <= 1 ? 16 : 8;
  float x[N];
#pragma unroll
  for (int j = 0; j < N; ++j) x[j] = (threadIdx.x + j) * (OP >= 2 ? 1e-3f : 1.0f);
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      if (OP == 0) x[j] = fmaf(x[j], a, b);
      if (OP == 1) x[j] = x[j] + a;
      if (OP == 2) x[j] = __expf(x[j]) * a;
      if (OP == 3) x[j] = __sinf(x[j]) + a;
      if (OP == 4) x[j] = __shfl_xor_sync(0xffffffffu, x[j], 1 + (j & 15));
    }
  }
  float s = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// packed add.rn.f32x2 (two element adds per instruction)
__global__ void f32x2_kernel(float* out, float a) {
  unsigned long long x[8], av;
  asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float f0 = threadIdx.x + j, f1 = f0 + 0.5f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x[j]) : "f"(f0), "f"(f1));
  }
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) asm volatile("add.rn.f32x2 %0, %0, %1;" : "+l"(x[j]) : "l"(av));
  }
  float s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float f0, f1;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(f0), "=f"(f1) : "l"(x[j]));
    s += f0 + f1;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace ur
}  // namespace qmlr

using namespace qmlr;

extern "C" int qmlr_unit_rates(double* host_rates, int32_t n_rates, void* stream) {
  QMLR_REQUIRE(host_rates && n_rates >= QMLR_RATE_COUNT, "need room for %d rates", QMLR_RATE_COUNT);
  cudaStream_t s = as_stream(stream);
  const int blocks = 8 * sm_count(), threads = 256;
  const size_t n = (size_t)blocks * threads;
  void* buf = nullptr;
  QMLR_CUDA_TRY(cudaMallocAsync(&buf, n * sizeof(double), s));
  double* dd = static_cast<double*>(buf);
  float* df = static_cast<float*>(buf);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = QMLR_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = QMLR_ECUDA;
  auto measure = [&](int idx, double ops_per_thread, auto launch) {
    if (rc) return;
    launch();
    cudaEventRecord(e0, s);
    for (int r = 0; r < 5; ++r) launch();
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      set_error("unit-rate kernel failed");
      rc = QMLR_ECUDA;
      return;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    host_rates[idx] = ops_per_thread * (double)n / (ms / 5.0 * 1e-3);
  };
  const double it = ur::kIters;
  measure(QMLR_RATE_DFMA, 8 * it, [&] { ur::dfma_kernel<<<blocks, threads, 0, s>>>(dd, 0.999, 1e-3); count_launch(); });
  measure(QMLR_RATE_FFMA, 16 * it, [&] { ur::f32_kernel<0><<<blocks, threads, 0, s>>>(df, 0.999f, 1e-3f); count_launch(); });
  measure(QMLR_RATE_FADD, 16 * it, [&] { ur::f32_kernel<1><<<blocks, threads, 0, s>>>(df, 1e-3f, 0.f); count_launch(); });
  measure(QMLR_RATE_FADD_X2, 16 * it, [&] { ur::f32x2_kernel<<<blocks, threads, 0, s>>>(df, 1e-3f); count_launch(); });
  measure(QMLR_RATE_EXP, 8 * it, [&] { ur::f32_kernel<2><<<blocks, threads, 0, s>>>(df, 0.3f, 0.f); count_launch(); });
  measure(QMLR_RATE_SIN, 8 * it, [&] { ur::f32_kernel<3><<<blocks, threads, 0, s>>>(df, 0.5f, 0.f); count_launch(); });
  measure(QMLR_RATE_SHFL, 8 * it, [&] { ur::f32_kernel<4><<<blocks, threads, 0, s>>>(df, 0.5f, 0.f); count_launch(); });
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(buf, s);
  return rc;
}
