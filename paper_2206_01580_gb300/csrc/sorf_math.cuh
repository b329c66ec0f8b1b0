// Arithmetic shared by the SORF kernels: the in-register Walsh-Hadamard
// butterflies, the Rademacher sign flips and the phase reduction for sin/cos.
#pragma once

#include "common.cuh"

namespace qmlr {

template <int D>
__device__ __forceinline__ void fwht(float (&v)[D]) {
#pragma unroll
  for (int h = 1; h < D; h <<= 1) {
#pragma unroll
    for (int i = 0; i < D; i += 2 * h) {
#pragma unroll
      for (int j = i; j < i + h; ++j) {
        const float a = v[j], b = v[j + h];
        v[j] = a + b;
        v[j + h] = a - b;
      }
    }
  }
}

// v[i] *= (bit i of the sign words set ? -1 : +1)
template <int D>
__device__ __forceinline__ void flip(float (&v)[D], const uint32_t* w) {
#pragma unroll
  for (int q = 0; q < (D + 31) / 32; ++q) {
    const uint32_t bits = w[q];
#pragma unroll
    for (int j = 0; j < 32 && 32 * q + j < D; ++j) {
      const uint32_t m = (bits << (31 - j)) & 0x80000000u;
      v[32 * q + j] = __uint_as_float(__float_as_uint(v[32 * q + j]) ^ m);
    }
  }
}

// sin and cos of an FP32 argument: Cody-Waite reduction by 2*pi with a
// two-part constant (2*pi = 6.28125 + 1.9353071795864769e-3; 6.28125 has an
// 8-bit significand so k * 6.28125 is exact for |k| < 2^16, i.e. |u| < 2^17 pi),
// then the hardware approximations on [-pi, pi] (absolute error ~2^-21). The
// kernels check that bound per atom before they use it (check_range below).
__device__ __forceinline__ void fast_sincos(float u, float* sn, float* cs) {
  const float k = rintf(u * 0.15915494309189535f);
  float r = fmaf(-k, 6.28125f, u);
  r = fmaf(-k, 1.9353071795864769e-3f, r);
  *sn = __sinf(r);
  *cs = __cosf(r);
}
__device__ __forceinline__ float fast_cos(float u) {
  const float k = rintf(u * 0.15915494309189535f);
  float r = fmaf(-k, 6.28125f, u);
  r = fmaf(-k, 1.9353071795864769e-3f, r);
  return __cosf(r);
}
__device__ __forceinline__ float fast_sin(float u) {
  const float k = rintf(u * 0.15915494309189535f);
  float r = fmaf(-k, 6.28125f, u);
  r = fmaf(-k, 1.9353071795864769e-3f, r);
  return __sinf(r);
}

// |u_i| <= (sqrt(d)/sigma) |x|_2 + |b_i| (each stack of W is sqrt(d)/sigma times
// an orthogonal matrix), so the reduction above is exact for the whole atom when
// |x|_2^2 <= x2max = ((2^17 - 4) pi)^2 sigma^2 / d (4 pi of margin for b and rounding).
inline float sorf_x2max(int d, double sigma) {
  const double lim = (131072.0 - 4.0) * 3.14159265358979323846;
  return (float)(lim * lim * sigma * sigma / d);
}

}  // namespace qmlr
