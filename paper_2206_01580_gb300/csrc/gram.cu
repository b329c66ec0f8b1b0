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
#include <cuda_fp8.h>

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

// The same split on 64 x 64 tiles with 16-byte accesses (Z 16-byte aligned,
// ldz a multiple of 4, st 16-byte aligned; k_pad is a multiple of 64): float4
// loads along the features, and each thread writes 8 consecutive rows of one
// feature per part as one 16-byte store. Same values as gram_operand_kernel.
constexpr int kOT = 64;

__global__ void __launch_bounds__(256)
gram_operand_wide_kernel(const float* __restrict__ Z, long n_rows, int n_features, long ldz, int n_split,
                         __nv_bfloat16* __restrict__ st, long k_pad) {
  __shared__ float tile[kOT][kOT + 1];
  const long r0 = (long)blockIdx.x * kOT;
  const int f0 = blockIdx.y * kOT;
  const int tid = threadIdx.x;
  // load: 64 rows x 16 float4, four per thread
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int idx = tid + 256 * u;
    const int j = idx >> 4, c4 = (idx & 15) * 4;
    const long r = r0 + j;
    const int f = f0 + c4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < n_rows) {
      if (f + 3 < n_features) {
        v = __ldg(reinterpret_cast<const float4*>(Z + r * ldz + f));
      } else {
        if (f < n_features) v.x = __ldg(Z + r * ldz + f);
        if (f + 1 < n_features) v.y = __ldg(Z + r * ldz + f + 1);
        if (f + 2 < n_features) v.z = __ldg(Z + r * ldz + f + 2);
      }
    }
    tile[j][c4] = v.x;
    tile[j][c4 + 1] = v.y;
    tile[j][c4 + 2] = v.z;
    tile[j][c4 + 3] = v.w;
  }
  __syncthreads();
  // store: thread -> feature f0 + tid / 4, rows 16 (tid % 4) .. + 15 as two runs of 8
  const int fl = tid >> 2, rc = (tid & 3) * 16;
  const int f = f0 + fl;
  if (f >= n_features) return;
  const long part = (long)n_features * k_pad;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int rl = rc + 8 * h;
    float v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = tile[rl + i][fl];
    for (int q = 0; q < n_split; ++q) {
      __align__(16) __nv_bfloat16 b[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        b[i] = __float2bfloat16_rn(v[i]);
        v[i] -= __bfloat162float(b[i]);
      }
      *reinterpret_cast<uint4*>(st + q * part + (long)f * k_pad + r0 + rl) = *reinterpret_cast<const uint4*>(b);
    }
  }
}

// ---------------------------------------------------------------------------
// e4m3 operand with per-feature power-of-two scales: s_f = 2^floor(log2(448 /
// max_r |Z[r][f]|)) (1 for an all-zero feature), Q[f][r] = e4m3(s_f Z[r][f])
// rounded to nearest even and saturated at 448, inv_scale[f] = 1 / s_f. Since
// G = Z^T Z and each feature has its own scale, the tensor-core products of Q
// give G_ij = (Q^T Q)_ij / (s_i s_j) exactly up to the rounding of Q.

// |Z| column maxima as float bits (non-negative floats order like their bits).
__global__ void column_absmax_kernel(const float* __restrict__ Z, long n_rows, int n_features, long ldz,
                                     unsigned* __restrict__ amax) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_features) return;
  const long r0 = (long)blockIdx.y * 1024, r1 = min(n_rows, r0 + 1024);
  float m = 0.f;
  for (long r = r0; r < r1; ++r) m = fmaxf(m, fabsf(__ldg(Z + r * ldz + f)));
  if (m > 0.f) atomicMax(amax + f, __float_as_uint(m));
}

__global__ void fp8_scales_kernel(int n_features, float* __restrict__ inv_scale) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_features) return;
  const float m = __uint_as_float(reinterpret_cast<unsigned*>(inv_scale)[f]);
  float inv = 1.0f;
  if (m > 0.f && isfinite(m)) {
    int e;
    frexpf(448.0f / m, &e);            // 448/m = mant * 2^e, mant in [0.5, 1)
    inv = ldexpf(1.0f, 1 - e);         // 1 / s with s = 2^(e-1) <= 448/m
  }
  inv_scale[f] = inv;
}

__global__ void gram_operand_fp8_kernel(const float* __restrict__ Z, long n_rows, int n_features, long ldz,
                                        const float* __restrict__ inv_scale, uint8_t* __restrict__ q8,
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
  for (int j = ty; j < kTT; j += 8) {
    const int f = f0 + j;
    const long r = r0 + tx;
    if (f < n_features && r < k_pad) {
      const float v = tile[tx][j] / __ldg(inv_scale + f);   // times s_f (a power of two: exact)
      q8[(long)f * k_pad + r] = (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
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
int gram_tc_form(int form, int tile_n, int promote, const void* zt, long k_pad, int n_features,
                 const float* inv_scale, float* G, cudaStream_t s);

}  // namespace qmlr

using namespace qmlr;

extern "C" int qmlr_gram_operand(const float* Z, int64_t n_rows, int32_t n_features, int64_t ldz,
                                 int32_t n_split, uint16_t* zt, int64_t k_pad, void* stream) {
  QMLR_REQUIRE(n_rows >= 0 && n_features >= 1 && ldz >= n_features, "bad Z shape");
  QMLR_REQUIRE(n_split >= 1 && n_split <= 3, "n_split must be 1, 2 or 3 (got %d)", n_split);
  QMLR_REQUIRE(k_pad >= n_rows && k_pad % 64 == 0, "k_pad must be >= n_rows and a multiple of 64");
  QMLR_REQUIRE(zt && (n_rows == 0 || Z), "NULL pointer argument");
  if (k_pad == 0) return QMLR_OK;
  const bool wide = (n_rows == 0 || reinterpret_cast<uintptr_t>(Z) % 16 == 0) && ldz % 4 == 0 &&
                    reinterpret_cast<uintptr_t>(zt) % 16 == 0;
  if (wide) {
    dim3 grid((unsigned)(k_pad / kOT), (n_features + kOT - 1) / kOT);
    gram_operand_wide_kernel<<<grid, 256, 0, as_stream(stream)>>>(
        Z, n_rows, n_features, ldz, n_split, reinterpret_cast<__nv_bfloat16*>(zt), k_pad);
  } else {
    dim3 grid((unsigned)((k_pad + kTT - 1) / kTT), (n_features + kTT - 1) / kTT);
    gram_operand_kernel<<<grid, dim3(32, 8), 0, as_stream(stream)>>>(
        Z, n_rows, n_features, ldz, n_split, reinterpret_cast<__nv_bfloat16*>(zt), k_pad);
  }
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

extern "C" int qmlr_gram_operand_fp8(const float* Z, int64_t n_rows, int32_t n_features, int64_t ldz,
                                     uint8_t* zt, int64_t k_pad, float* inv_scale, void* stream) {
  QMLR_REQUIRE(n_rows >= 0 && n_features >= 1 && ldz >= n_features, "bad Z shape");
  QMLR_REQUIRE(k_pad >= n_rows && k_pad % 128 == 0, "k_pad must be >= n_rows and a multiple of 128");
  QMLR_REQUIRE(zt && inv_scale && (n_rows == 0 || Z), "NULL pointer argument");
  cudaStream_t s = as_stream(stream);
  QMLR_CUDA_TRY(cudaMemsetAsync(inv_scale, 0, sizeof(float) * n_features, s));
  if (n_rows > 0) {
    dim3 g1((n_features + 255) / 256, (unsigned)((n_rows + 1023) / 1024));
    column_absmax_kernel<<<g1, 256, 0, s>>>(Z, n_rows, n_features, ldz, reinterpret_cast<unsigned*>(inv_scale));
    QMLR_LAUNCH_CHECK();
  }
  fp8_scales_kernel<<<(n_features + 255) / 256, 256, 0, s>>>(n_features, inv_scale);
  QMLR_LAUNCH_CHECK();
  if (k_pad == 0) return QMLR_OK;
  dim3 grid((unsigned)((k_pad + kTT - 1) / kTT), (n_features + kTT - 1) / kTT);
  gram_operand_fp8_kernel<<<grid, dim3(32, 8), 0, s>>>(Z, n_rows, n_features, ldz, inv_scale, zt, k_pad);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

extern "C" int qmlr_gram_tc(const qmlr_gram_opts* o, const void* zt, int64_t k_pad, int32_t n_features,
                            const float* inv_scale, float* G, void* stream) {
  QMLR_REQUIRE(o && zt && G, "NULL pointer argument");
  QMLR_REQUIRE(n_features >= 128 && n_features % 128 == 0,
               "tensor-core Gram needs n_features a positive multiple of 128 (got %d)", n_features);
  const int tile = o->tile_n == 0 ? (o->precision == QMLR_GRAM_BF16X1 || o->precision == QMLR_GRAM_FP8X1 ? 256 : 128)
                                  : o->tile_n;
  QMLR_REQUIRE(tile == 128 || tile == 256, "tile_n must be 0, 128 or 256 (got %d)", o->tile_n);
  QMLR_REQUIRE(n_features % tile == 0, "n_features (%d) must be a multiple of the tile width %d", n_features, tile);
  QMLR_REQUIRE(o->promote >= 0, "promote must be >= 0");
  int form = 0;
  long kq = 64;
  switch (o->precision) {
    case QMLR_GRAM_BF16X1: form = 1; break;
    case QMLR_GRAM_BF16X3: form = 2; break;
    case QMLR_GRAM_BF16X6: form = 3; break;
    case QMLR_GRAM_FP8X1: form = 4; kq = 128; break;
    default: set_error("precision %d is not a tensor-core Gram form", o->precision); return QMLR_EINVAL;
  }
  QMLR_REQUIRE(k_pad >= 0 && k_pad % kq == 0, "k_pad must be a multiple of %ld for this form", kq);
  QMLR_REQUIRE(form != 4 || inv_scale, "inv_scale is NULL");
  return gram_tc_form(form, tile, o->promote, zt, k_pad, n_features, inv_scale, G, as_stream(stream));
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
  if (precision == QMLR_GRAM_BF16X1) {
    QMLR_REQUIRE(zt, "operand is NULL");
    qmlr_gram_opts o{QMLR_GRAM_BF16X1, 0, 0};
    return qmlr_gram_tc(&o, zt, k_pad, n_features, nullptr, G, stream);
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
