// Normal-equation Gram matrix G = Z^T Z and right-hand side c = Z^T y (sm_103a).
//
// RFF section of the paper: (Z^T Z + lambda I) alpha = Z^T E; with forces the
// rows of Z and of the derivative features are stacked; the Z^T Z product is
// the dominant training cost. The paper builds it in FP64, or in FP32 with
// Kahan summation.
//
// Forms built here:
// * QMLR_GRAM_FP32  - plain FP32 SIMT product (the comparison form; no
//                     compensation), upper-triangle tiles mirrored.
// * QMLR_GRAM_BF16X3 / QMLR_GRAM_BF16X6 - split-precision tensor-core
//                     products (gram_tc.cu) over a 2-way / 3-way BF16 split of
//                     Z, FP32 accumulation in TMEM.
// The operand kernel below writes the splits transposed (feature-major, rows
// contiguous: the K-major layout the tensor-core kernel reads with TMA).
#include "common.cuh"
#include <cuda_bf16.h>

namespace qmlr {

// ---------------------------------------------------------------------------
// split + transpose: Z [n_rows][ldz] fp32 -> St[q] [n_features][k_pad] bf16, q < n_split:
//   S0 = bf16(z), S1 = bf16(z - S0), S2 = bf16(z - S0 - S1)   (round to nearest even)
constexpr int kTT = 32;

__global__ void gram_operand_kernel(const float* __restrict__ Z, long n_rows, int n_features,
                                    long ldz, int n_split, __nv_bfloat16* __restrict__ st,
                                    long k_pad) {
  __shared__ float tile[kTT][kTT + 1];
  const long r0 = (long)blockIdx.x * kTT;
  const int f0 = blockIdx.y * kTT;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int j = ty; j < kTT; j += 8) {
    const long r = r0 + j;
    const int f = f0 + tx;
    tile[j][tx] = (r < n_rows && f < n_features) ? __ldg(Z + r * ldz + f) : 0.f;
  }
  __syncthreads();
  const long part = (long)n_features * k_pad;
  for (int j = ty; j < kTT; j += 8) {
    const int f = f0 + j;
    const long r = r0 + tx;
    if (f < n_features && r < k_pad) {
      float v = tile[tx][j];
      for (int q = 0; q < n_split; ++q) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        st[q * part + (long)f * k_pad + r] = h;
        v -= __bfloat162float(h);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// plain FP32 SIMT Gram: tiles 128 x 128, K chunks of 16 rows, upper tiles only,
// each tile written to (i, j) and mirrored to (j, i).
constexpr int GT = 128, GK = 16;

__global__ void __launch_bounds__(256)
gram_fp32_kernel(const float* __restrict__ Z, long n_rows, int n_features, long ldz,
                 float* __restrict__ G) {
  __shared__ __align__(16) float As[GK][GT];
  __shared__ __align__(16) float Bs[GK][GT];
  // linear block -> (bi <= bj) upper-triangular tile
  const int nt = (n_features + GT - 1) / GT;
  int t = blockIdx.x, bi = 0;
  while (t >= nt - bi) {
    t -= nt - bi;
    ++bi;
  }
  const int bj = bi + t;
  const int i0 = bi * GT, j0 = bj * GT;
  const int tid = threadIdx.x, tr = tid / 16, tc = tid % 16;   // 8 x 8 outputs per thread
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

  for (long k0 = 0; k0 < n_rows; k0 += GK) {
    // load 16 rows x 128 features for each operand: 2048 values, 8 per thread
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int idx = tid + q * 256;
      const int kk = idx / GT, cc = idx % GT;
      const long r = k0 + kk;
      const bool rok = r < n_rows;
      As[kk][cc] = (rok && i0 + cc < n_features) ? __ldg(Z + r * ldz + i0 + cc) : 0.f;
      Bs[kk][cc] = (rok && j0 + cc < n_features) ? __ldg(Z + r * ldz + j0 + cc) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      float a[8], b[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        a[u] = As[kk][tr * 4 + (u & 3) + (u >> 2) * 64];
        b[u] = Bs[kk][tc * 4 + (u & 3) + (u >> 2) * 64];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int i = i0 + tr * 4 + (u & 3) + (u >> 2) * 64;
    if (i >= n_features) continue;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int j = j0 + tc * 4 + (v & 3) + (v >> 2) * 64;
      if (j >= n_features) continue;
      G[(long)i * n_features + j] = acc[u][v];
      G[(long)j * n_features + i] = acc[u][v];
    }
  }
}

// ---------------------------------------------------------------------------
// c = Z^T y in FP64: partial sums over row chunks, then a fixed-order reduction.
constexpr int kZtyRows = 2048;

__global__ void zty_partial_kernel(const float* __restrict__ Z, long n_rows, int n_features,
                                   long ldz, const double* __restrict__ y,
                                   double* __restrict__ part) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const long r0 = (long)blockIdx.y * kZtyRows;
  const long r1 = min(n_rows, r0 + kZtyRows);
  if (f >= n_features) return;
  double acc = 0.0;
  for (long r = r0; r < r1; ++r) acc = fma((double)__ldg(Z + r * ldz + f), __ldg(y + r), acc);
  part[(long)blockIdx.y * n_features + f] = acc;
}

__global__ void sum_parts_kernel(const double* __restrict__ part, int n_parts, int n,
                                 double* __restrict__ out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n) return;
  double acc = 0.0;
  for (int p = 0; p < n_parts; ++p) acc += part[(long)p * n + f];
  out[f] = acc;
}

int gram_split_tc(int n_split, const uint16_t* zt, long k_pad, int n_features, float* G, cudaStream_t s);

}  // namespace qmlr

using namespace qmlr;

extern "C" int qmlr_gram_operand(const float* Z, int64_t n_rows, int32_t n_features, int64_t ldz,
                                 int32_t n_split, uint16_t* zt, int64_t k_pad, void* stream) {
  QMLR_REQUIRE(n_rows >= 0 && n_features >= 1 && ldz >= n_features, "bad Z shape");
  QMLR_REQUIRE(n_split == 2 || n_split == 3, "n_split must be 2 or 3 (got %d)", n_split);
  QMLR_REQUIRE(k_pad >= n_rows && k_pad % 64 == 0, "k_pad must be >= n_rows and a multiple of 64");
  QMLR_REQUIRE(zt && (n_rows == 0 || Z), "NULL pointer argument");
  if (k_pad == 0) return QMLR_OK;
  dim3 grid((unsigned)((k_pad + kTT - 1) / kTT), (n_features + kTT - 1) / kTT);
  gram_operand_kernel<<<grid, dim3(32, 8), 0, as_stream(stream)>>>(
      Z, n_rows, n_features, ldz, n_split, reinterpret_cast<__nv_bfloat16*>(zt), k_pad);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

extern "C" int qmlr_gram(int32_t precision, const float* Z, int64_t n_rows, int32_t n_features,
                         int64_t ldz, const uint16_t* zt, int64_t k_pad, float* G, void* stream) {
  QMLR_REQUIRE(n_features >= 1 && G, "bad arguments");
  cudaStream_t s = as_stream(stream);
  if (precision == QMLR_GRAM_FP32) {
    QMLR_REQUIRE(n_rows >= 0 && ldz >= n_features && (n_rows == 0 || Z), "bad Z");
    const int nt = (n_features + GT - 1) / GT;
    gram_fp32_kernel<<<nt * (nt + 1) / 2, 256, 0, s>>>(Z, n_rows, n_features, ldz, G);
    QMLR_LAUNCH_CHECK();
    return QMLR_OK;
  }
  if (precision == QMLR_GRAM_BF16X3 || precision == QMLR_GRAM_BF16X6) {
    QMLR_REQUIRE(zt, "split operand is NULL");
    QMLR_REQUIRE(k_pad % 64 == 0 && k_pad >= 0, "k_pad must be a multiple of 64");
    QMLR_REQUIRE(n_features % 128 == 0, "tensor-core Gram needs n_features %% 128 == 0 (got %d)", n_features);
    return gram_split_tc(precision == QMLR_GRAM_BF16X3 ? 2 : 3, zt, k_pad, n_features, G, s);
  }
  set_error("unknown Gram precision %d", precision);
  return QMLR_EINVAL;
}

extern "C" int64_t qmlr_zty_workspace_bytes(int64_t n_rows, int32_t n_features) {
  const int64_t parts = (n_rows + kZtyRows - 1) / kZtyRows;
  return std::max<int64_t>(parts, 1) * n_features * 8;
}

extern "C" int qmlr_zty(const float* Z, int64_t n_rows, int32_t n_features, int64_t ldz,
                        const double* y, double* c, void* work, int64_t work_bytes, void* stream) {
  QMLR_REQUIRE(n_rows >= 0 && n_features >= 1 && ldz >= n_features, "bad Z shape");
  QMLR_REQUIRE(c && (n_rows == 0 || (Z && y)), "NULL pointer argument");
  QMLR_REQUIRE(work && work_bytes >= qmlr_zty_workspace_bytes(n_rows, n_features),
               "workspace too small");
  cudaStream_t s = as_stream(stream);
  const int parts = (int)std::max<int64_t>((n_rows + kZtyRows - 1) / kZtyRows, 1);
  double* part = static_cast<double*>(work);
  if (n_rows == 0) {
    QMLR_CUDA_TRY(cudaMemsetAsync(c, 0, sizeof(double) * n_features, s));
    return QMLR_OK;
  }
  dim3 grid((n_features + 255) / 256, parts);
  zty_partial_kernel<<<grid, 256, 0, s>>>(Z, n_rows, n_features, ldz, y, part);
  QMLR_LAUNCH_CHECK();
  sum_parts_kernel<<<(n_features + 255) / 256, 256, 0, s>>>(part, parts, n_features, c);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}
