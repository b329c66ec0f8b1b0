// FP64 solve of the regularised normal equations (sm_103a).
//
// RFF section of the paper: (Z^T Z + lambda I) alpha = Z^T y. The paper
// factorises with LU; the matrix is symmetric positive definite, so this
// library uses a blocked right-looking Cholesky factorisation in FP64
// (64 x 64 blocks: diagonal factor, panel triangular solve, trailing
// symmetric update), then refines alpha against the exact operator
// A v = Z^T (Z v) + lambda v evaluated in FP64 from the stored FP32 Z, with
// the Cholesky factor as preconditioner (preconditioned conjugate gradients,
// or classical refinement). This keeps the low-precision Gram an
// approximation used only for the factor, while the residual is that of the
// exact FP64 normal equations.
#include "common.cuh"

#include <cuda_bf16.h>

#include <mutex>

namespace qmlr {

constexpr int NB = 64;

// tensor-core trailing update (gram_tc.cu)
// part 0: all lower tiles; 1: the first two 128-wide tile columns; 2: the others
int syrk_tc(const uint16_t* parts, long part_elems, int m, double* A, long lda, int part, cudaStream_t s);

// A = G + (lambda + shift) I in FP64, lower triangle (G symmetric fp32 [n][n]).
__global__ void assemble_kernel(const float* __restrict__ G, int n, double diag,
                                double* __restrict__ L, long ldl) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  double v = (double)G[idx];
  if (i == j) v += diag;
  L[(long)i * ldl + j] = (j <= i) ? v : 0.0;
}

// 1/sqrt(d) in FP64 from an FP32 seed and one Newton-Raphson step for the
// reciprocal square root, y <- y (3 - d y^2) / 2, which squares the seed's
// relative error (~2^-22 -> ~2^-43). Outside the FP32 range of the seed it
// falls back to the division.
__device__ __forceinline__ double rsqrt_newton(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  const double y = (double)rsqrtf((float)d);
  return y * fma(-0.5 * d, y * y, 1.5);
}

// The mixed-precision factor keeps the not yet factorised trailing matrix as
// float pairs (hi, lo) with value hi + lo (about 48 significant bits) in the
// 8 bytes of each FP64 element, so that the tensor-core updates subtract in
// FP32 arithmetic; a 256-column panel is converted to FP64 just before it is
// factorised.
__device__ __forceinline__ float2 to_pair(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}

// A = G + (lambda + shift) I as float pairs in the lower triangle (FP64 zeros above).
__global__ void assemble_pairs_kernel(const float* __restrict__ G, int n, double diag, double* __restrict__ L,
                                      long ldl) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  double* e = L + (long)i * ldl + j;
  if (j < i) *reinterpret_cast<float2*>(e) = make_float2(G[idx], 0.f);
  else if (j == i) *reinterpret_cast<float2*>(e) = to_pair((double)G[idx] + diag);
  else *e = 0.0;
}

// FP64 -> float pairs in place over the lower triangle.
__global__ void to_pairs_kernel(double* __restrict__ L, long ldl, int n) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  if (j > i) return;
  double* e = L + (long)i * ldl + j;
  *reinterpret_cast<float2*>(e) = to_pair(*e);
}

// Unblocked Cholesky of the nb x nb diagonal block at (k0, k0) in shared memory
// (rows past nb are identity rows). Step j: one thread forms the pivot's
// 1/sqrt, the column below it is scaled, and the active triangle j < l <= i is
// updated by all threads from a table of its (i, l) pairs ordered by column
// from the right, so that step j's work is the table's first (63-j)(64-j)/2
// entries (no idle index arithmetic, no lanes outside the triangle).
__global__ void __launch_bounds__(256)
potrf_diag_kernel(double* __restrict__ L, long ldl, int k0, int nb, int* err, int* info) {
  __shared__ double a[NB][NB + 1];
  __shared__ uint16_t tri[NB * (NB - 1) / 2];
  __shared__ double ys;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int i = idx / NB, j = idx % NB;
    a[i][j] = (i < nb && j <= i) ? L[(long)(k0 + i) * ldl + k0 + j] : (i == j ? 1.0 : 0.0);
  }
  if (tid >= 1 && tid < NB) {   // column l = tid: entries (i, l), i = l..63, after columns > l
    const int l = tid, off = (NB - 1 - l) * (NB - l) / 2;
    for (int i = l; i < NB; ++i) tri[off + i - l] = (uint16_t)((i << 8) | l);
  }
  __syncthreads();
  for (int j = 0; j < NB; ++j) {
    if (tid == 0) {
      double d = a[j][j];
      if (!(d > 0.0)) {
        if (j < nb) {
          record_device_error(err, DEV_NOT_SPD);
          if (info && *info == 0) *info = k0 + j + 1;
        }
        d = 1.0;
      }
      const double y = rsqrt_newton(d);
      a[j][j] = d * y;
      ys = y;
    }
    __syncthreads();
    if (tid > j && tid < NB) a[tid][j] *= ys;
    __syncthreads();
    const int cnt = (NB - 1 - j) * (NB - j) / 2;
    for (int e = tid; e < cnt; e += blockDim.x) {
      const int pr = tri[e], i = pr >> 8, l = pr & 255;
      a[i][l] = fma(-a[i][j], a[l][j], a[i][l]);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nb * nb; idx += blockDim.x) {
    const int i = idx / nb, j = idx % nb;
    if (j <= i) L[(long)(k0 + i) * ldl + k0 + j] = a[i][j];
  }
}

// Panel: rows r in [k0+nb, n): L[r][k0:k0+nb] = A[r][k0:k0+nb] * L_kk^{-T}. Four threads
// share a row (thread q owns columns l = q mod 4) in shared memory: after the owner forms
// x_j = a_j / L_jj it is shuffled to the row's other threads and removed from the later
// equations (x_l -= x_j L_lj), so every warp keeps the FP64 units of its SM quarter busy
// and a row's dependency chain is short. With lp set, the solved rows are also written
// as float pairs (lp[r - k0 - nb][0:64]) for the update of the panel's later columns.
constexpr int kTrsmRows = 64;

__global__ void __launch_bounds__(256)
trsm_panel_kernel(double* __restrict__ L, long ldl, int k0, int nb, int n, float2* __restrict__ lp) {
  extern __shared__ double tsm[];
  double (*lkk)[NB + 1] = reinterpret_cast<double (*)[NB + 1]>(tsm);
  double (*X)[NB + 1] = reinterpret_cast<double (*)[NB + 1]>(tsm + NB * (NB + 1));
  double* rdg = tsm + 2 * NB * (NB + 1);
  const int tid = threadIdx.x, lane = tid & 31;
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int i = idx / NB, j = idx % NB;
    lkk[i][j] = (i < nb && j <= i) ? L[(long)(k0 + i) * ldl + k0 + j] : (i == j ? 1.0 : 0.0);
  }
  const int rbase = k0 + nb + blockIdx.x * kTrsmRows;
  for (int idx = tid; idx < kTrsmRows * NB; idx += blockDim.x) {
    const int rr = idx / NB, j = idx % NB, r = rbase + rr;
    X[rr][j] = (r < n && j < nb) ? L[(long)r * ldl + k0 + j] : 0.0;
  }
  __syncthreads();
  if (tid < NB) rdg[tid] = 1.0 / lkk[tid][tid];
  __syncthreads();
  const int row = tid >> 2, q = tid & 3;
  for (int j = 0; j < NB; ++j) {
    double xj = 0.0;
    if (q == (j & 3)) {
      xj = X[row][j] * rdg[j];
      X[row][j] = xj;
    }
    xj = __shfl_sync(0xffffffffu, xj, (lane & ~3) | (j & 3));
    for (int l = j + 1 + ((q - j - 1) & 3); l < NB; l += 4) X[row][l] = fma(-xj, lkk[l][j], X[row][l]);
  }
  __syncthreads();
  for (int idx = tid; idx < kTrsmRows * NB; idx += blockDim.x) {
    const int rr = idx / NB, j = idx % NB, r = rbase + rr;
    if (r < n && j < nb) L[(long)r * ldl + k0 + j] = X[rr][j];
    if (lp && r < n) lp[(long)(r - k0 - nb) * NB + j] = j < nb ? to_pair(X[rr][j]) : make_float2(0.f, 0.f);
  }
}

constexpr size_t kTrsmSmem = (2 * NB * (NB + 1) + NB) * sizeof(double);

// Trailing update of the lower block tiles: A[I][J] -= L[I][k] L[J][k]^T, I >= J > k,
// for the first `cblocks` trailing block columns J (all of them when cblocks >= T).
__global__ void __launch_bounds__(256)
syrk_update_kernel(double* __restrict__ L, long ldl, int k0, int nb, int n, int cblocks) {
  extern __shared__ double dsm[];
  double (*li)[NB + 1] = reinterpret_cast<double (*)[NB + 1]>(dsm);
  double (*lj)[NB + 1] = reinterpret_cast<double (*)[NB + 1]>(dsm + NB * (NB + 1));
  const int t0 = (k0 + nb) / NB;          // first trailing block
  const int T = (n + NB - 1) / NB - t0;   // trailing blocks
  int t = blockIdx.x, bi = 0, bj = 0;
  if (cblocks >= T) {
    while (t > bi) {                      // lower-triangular (bi >= bj) enumeration, by rows
      t -= bi + 1;
      ++bi;
    }
    bj = t;
  } else {
    while (bj < cblocks && t >= T - bj) { // limited to cblocks columns, by columns
      t -= T - bj;
      ++bj;
    }
    if (bj >= cblocks) return;
    bi = bj + t;
  }
  if (bi >= T) return;
  const int i0 = (t0 + bi) * NB, j0 = (t0 + bj) * NB;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < NB * nb; idx += blockDim.x) {
    const int rr = idx / nb, c = idx % nb;
    li[rr][c] = (i0 + rr < n) ? L[(long)(i0 + rr) * ldl + k0 + c] : 0.0;
    lj[rr][c] = (j0 + rr < n) ? L[(long)(j0 + rr) * ldl + k0 + c] : 0.0;
  }
  __syncthreads();
  const int tr = tid / 16, tc = tid % 16;   // 4 x 4 outputs each
  double acc[4][4] = {};
  for (int c = 0; c < nb; ++c) {
    double a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] = li[tr + 16 * u][c];
      b[u] = lj[tc + 16 * u][c];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + tr + 16 * u;
    if (i >= n) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = j0 + tc + 16 * v;
      if (j >= n || j > i) continue;
      L[(long)i * ldl + j] -= acc[u][v];
    }
  }
}

// Update of a panel's later columns inside the mixed-precision factor, in
// double-float FP32 arithmetic: A[I][J] -= L[I][k] L[J][k]^T (I >= J, first
// `cblocks` block columns), with L given as float pairs lp (rows from k0 + nb,
// 64 columns) and A held as float pairs. Each product of pairs is formed by
// Dekker's FMA product of the high parts plus the two cross terms, and summed
// with Knuth's two-sum into a (sum, compensation) pair: about 44 significant
// bits, at FP32 instruction rates instead of the GB300's FP64 rate.
__device__ __forceinline__ void df_fma(float& s, float& c, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float e = __fmaf_rn(ah, bh, -p);
  const float x = __fmaf_rn(ah, bl, __fmul_rn(al, bh));
  const float s1 = __fadd_rn(s, p);
  const float bb = __fsub_rn(s1, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(s1, bb)), __fsub_rn(p, bb));
  s = s1;
  c = __fadd_rn(c, __fadd_rn(err, __fadd_rn(e, x)));
}

// (a.x + a.y) + (b.x + b.y), renormalised (two-sum of the high parts)
__device__ __forceinline__ float2 pair_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bb = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  const float lo = __fadd_rn(__fadd_rn(a.y, b.y), e);
  const float h = __fadd_rn(s, lo);
  return make_float2(h, __fsub_rn(lo, __fsub_rn(h, s)));
}

// (hi + lo) - (s + c) for float pairs, renormalised.
__device__ __forceinline__ float2 pair_sub2(float2 a, float s, float c) {
  const float t = __fsub_rn(a.x, s);
  const float bb = __fsub_rn(t, a.x);
  const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(t, bb)), __fsub_rn(-s, bb));
  const float lo = __fadd_rn(__fsub_rn(a.y, c), e);
  const float h = __fadd_rn(t, lo);
  const float b2 = __fsub_rn(h, t);
  return make_float2(h, __fadd_rn(__fsub_rn(t, __fsub_rn(h, b2)), __fsub_rn(lo, b2)));
}

__global__ void __launch_bounds__(256)
syrk_pairs_kernel(double* __restrict__ L, long ldl, int k0, int nb, int n, int cblocks,
                  const float2* __restrict__ lp) {
  extern __shared__ float fsm[];
  float (*ih)[NB + 1] = reinterpret_cast<float (*)[NB + 1]>(fsm);
  float (*il)[NB + 1] = reinterpret_cast<float (*)[NB + 1]>(fsm + NB * (NB + 1));
  float (*jh)[NB + 1] = reinterpret_cast<float (*)[NB + 1]>(fsm + 2 * NB * (NB + 1));
  float (*jl)[NB + 1] = reinterpret_cast<float (*)[NB + 1]>(fsm + 3 * NB * (NB + 1));
  const int t0 = (k0 + nb) / NB;
  const int T = (n + NB - 1) / NB - t0;
  int t = blockIdx.x, bi = 0, bj = 0;
  while (bj < cblocks && t >= T - bj) {
    t -= T - bj;
    ++bj;
  }
  if (bj >= cblocks) return;
  bi = bj + t;
  if (bi >= T) return;
  const int m = n - k0 - nb;   // rows of lp
  const int tid = threadIdx.x;
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int rr = idx / NB, c = idx % NB;
    const int ri = bi * NB + rr, rj = bj * NB + rr;
    const float2 a = ri < m ? lp[(long)ri * NB + c] : make_float2(0.f, 0.f);
    const float2 b = rj < m ? lp[(long)rj * NB + c] : make_float2(0.f, 0.f);
    ih[rr][c] = a.x;
    il[rr][c] = a.y;
    jh[rr][c] = b.x;
    jl[rr][c] = b.y;
  }
  __syncthreads();
  const int tr = tid / 16, tc = tid % 16;
  float sa[4][4], ca[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) sa[u][v] = ca[u][v] = 0.f;
  for (int c = 0; c < nb; ++c) {
    float ah[4], al[4], bh[4], bl[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      ah[u] = ih[tr + 16 * u][c];
      al[u] = il[tr + 16 * u][c];
      bh[u] = jh[tc + 16 * u][c];
      bl[u] = jl[tc + 16 * u][c];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) df_fma(sa[u][v], ca[u][v], ah[u], al[u], bh[v], bl[v]);
  }
  float2* P = reinterpret_cast<float2*>(L);
  const int i0 = (t0 + bi) * NB, j0 = (t0 + bj) * NB;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + tr + 16 * u;
    if (i >= n) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = j0 + tc + 16 * v;
      if (j > i) continue;
      float2* e = P + (long)i * ldl + j;
      *e = pair_sub2(*e, sa[u][v], ca[u][v]);
    }
  }
}

constexpr size_t kPairsSmem = 4 * NB * (NB + 1) * sizeof(float);

// ---------------------------------------------------------------------------
// Diagonal block and panel solve of the mixed-precision factor in double-float
// arithmetic. The block column still holds the float pairs of the trailing
// matrix; these kernels read them directly, compute with pair products
// (Dekker's product of the high parts plus the cross terms, two-sum
// accumulation: about 44 significant bits) at FP32 rates, and write the FP64
// factor entries (and, for the panel, the pairs the later updates read).
// Reading the pairs saves a conversion pass per block column; the two kernels
// are latency-bound chains of 64 dependent steps, so what matters per step is
// its instruction latency (an FP64 pivot chain made the diagonal factor take
// 95 us per block, the FP32 one below 59 us).

// x * y for float pairs, renormalised
__device__ __forceinline__ float2 pair_mul(float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float e = __fmaf_rn(x.x, y.x, -p);
  e = __fmaf_rn(x.x, y.y, __fmaf_rn(x.y, y.x, e));
  const float h = __fadd_rn(p, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, p)));
}

__device__ __forceinline__ double pair_value(float2 p) { return (double)p.x + (double)p.y; }

// 1/sqrt(d) of a positive float pair without FP64 instructions: an FP32 seed
// y0 (relative error ~2^-23) and one Newton-Raphson step y0 (1 + (1 - d y0^2)/2),
// with d y0^2 formed as a pair product (1 - d y0^2 is then exact to ~2^-46), so
// the result carries ~2^-44 relative error. (On the GB300 each FP64 instruction
// holds the SM quarter's FP64 pipe for tens of cycles; the pivot is on the
// factor's critical path.)
__device__ __forceinline__ float2 pair_rsqrt(float2 d) {
  const float y0 = rsqrtf(d.x);
  const float p = __fmul_rn(y0, y0);
  const float2 u = pair_mul(d, make_float2(p, __fmaf_rn(y0, y0, -p)));
  const float e = __fsub_rn(__fsub_rn(1.f, u.x), u.y);
  const float corr = __fmul_rn(__fmul_rn(y0, e), 0.5f);
  const float h = __fadd_rn(y0, corr);
  return make_float2(h, __fsub_rn(corr, __fsub_rn(h, y0)));
}

// Factor of the diagonal block (float pairs on entry), right-looking over the
// block held in shared memory as float pairs, one barrier per step. Column j is
// kept unscaled (a_ij) until the end: at step j every entry (i, l) of the
// trailing triangle j < l <= i takes a_il -= a_ij a_lj / d_j (a pair product
// with the pair 1/d_j, then a two-sum subtraction), the entries spread evenly
// over the CTA's threads in a compact triangular enumeration (no idle
// predicated work), and the thread holding entry (j+1, j+1) forms the next
// pivot's 1/sqrt (pair_rsqrt) before the barrier. At the end L_ij = a_ij / sqrt(d_j).
// The loop is small and not unrolled: one CTA runs it, on an SM whose
// instruction cache holds none of it. Writes L_kk in FP64 to L, and its pairs
// and the pivots' reciprocals (pairs) to dpairs ([64][64] then [64]).
__device__ __forceinline__ void diag_pivot(float2 a, int j, int k0, int nb, int* err, int* info, float2* ys,
                                           float2* yy) {
  float2 d = pair_add(a, make_float2(0.f, 0.f));
  if (!(d.x > 0.f)) {
    if (j < nb) {
      record_device_error(err, DEV_NOT_SPD);
      if (info && *info == 0) *info = k0 + j + 1;
    }
    d = make_float2(1.f, 0.f);
  }
  const float2 y = pair_rsqrt(d);   // 1 / sqrt(d_j)
  ys[j] = y;
  yy[j] = pair_mul(y, y);           // 1 / d_j
}

constexpr int kDiagThreads = 1024;   // about one trailing entry per thread and step: latency, not work, bounds a step
static_assert(2 * kDiagThreads >= NB * (NB - 1) / 2, "two trailing entries per thread cover the first step");

__global__ void __launch_bounds__(kDiagThreads, 1)
potrf_diag_blk_kernel(double* __restrict__ L, long ldl, int k0, int nb, int* err, int* info,
                      float2* __restrict__ dpairs) {
  __shared__ float2 A[NB][NB + 1];
  __shared__ float2 ys[NB], yy[NB];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int r = idx / NB, c = idx % NB;
    A[r][c] = (r < nb && c <= r) ? *reinterpret_cast<const float2*>(L + (long)(k0 + r) * ldl + k0 + c)
                                 : make_float2(c == r ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  if (tid == 0) diag_pivot(A[0][0], 0, k0, nb, err, info, ys, yy);
  __syncthreads();
  // the triangle's row-major enumeration does not depend on the step: entry
  // e = (ii, ll) of the trailing triangle at step j is (j + 1 + ii, j + 1 + ll),
  // and thread tid holds e = tid + k kDiagThreads (k < 2: at most 2016 entries)
  int tii[2], tll[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int e = tid + k * kDiagThreads;
    float sq;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sq) : "f"(8.0f * (float)e + 1.0f));
    int ii = (int)((sq - 1.0f) * 0.5f);
    if (ii * (ii + 1) / 2 > e) --ii;
    else if ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
    tii[k] = ii;
    tll[k] = e - ii * (ii + 1) / 2;
  }
#pragma unroll 1
  for (int j = 0; j < NB - 1; ++j) {
    const float2 w = yy[j];
    const int m = NB - 1 - j;                 // trailing rows j+1 .. 63
    const int count = m * (m + 1) / 2;        // entries (i, l), j < l <= i
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int e = tid + k * kDiagThreads;
      if (e < count) {
        const int i = j + 1 + tii[k], l = j + 1 + tll[k];
        const float2 t = pair_mul(A[l][j], w);   // a_lj / d_j
        const float2 aij = A[i][j];
        float2 a = A[i][l];
        df_fma(a.x, a.y, -aij.x, -aij.y, t.x, t.y);
        A[i][l] = a;
        if (e == 0) diag_pivot(a, j + 1, k0, nb, err, info, ys, yy);   // entry (j+1, j+1)
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int r = idx / NB, c = idx % NB;
    float2 v = make_float2(0.f, 0.f);
    if (c < r) v = pair_mul(A[r][c], ys[c]);                                          // a_rc / sqrt(d_c)
    else if (c == r) v = pair_mul(pair_add(A[r][r], make_float2(0.f, 0.f)), ys[r]);   // sqrt(d_r)
    dpairs[idx] = v;
    if (r < nb && c <= r) L[(long)(k0 + r) * ldl + k0 + c] = pair_value(v);
  }
  if (tid < NB) dpairs[NB * NB + tid] = ys[tid];
}

// Panel solve as trsm_panel_kernel, on the float pairs of rows [k0+nb, n) of the
// block column, with L_kk and 1/L_jj as pairs from potrf_diag_blk_kernel. A row's
// 64 values stay in the registers of its eight threads (thread q holds columns
// 8k + q); at step j the owner of column j forms x_j, the row's threads get it
// by a shuffle and update their columns l > j (the 64 steps are unrolled, so
// register indices and the skipped column blocks are static). 32 rows per CTA.
// Writes the FP64 entries to L and, with lp set, the pairs
// (lp[r - k0 - nb][0:64]).
constexpr int kTrsmDfTpr = 8;                       // threads per row
constexpr int kTrsmDfRows = 256 / kTrsmDfTpr;       // rows per CTA
constexpr int kTrsmDfCols = NB / kTrsmDfTpr;        // columns per thread

__global__ void __launch_bounds__(256, 2)
trsm_panel_df_kernel(double* __restrict__ L, long ldl, int k0, int nb, int n,
                     const float2* __restrict__ dpairs, float2* __restrict__ lp) {
  constexpr int TPR = kTrsmDfTpr, NC = kTrsmDfCols;
  extern __shared__ float2 psm[];
  float2 (*lkk)[NB + 1] = reinterpret_cast<float2 (*)[NB + 1]>(psm);
  float2* rdg = psm + NB * (NB + 1);
  const int tid = threadIdx.x, lane = tid & 31;
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) lkk[idx / NB][idx % NB] = dpairs[idx];
  if (tid < NB) rdg[tid] = dpairs[NB * NB + tid];
  const int row = tid / TPR, q = tid % TPR;
  const int r = k0 + nb + blockIdx.x * kTrsmDfRows + row;
  float2 x[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const int c = TPR * k + q;
    x[k] = (r < n && c < nb) ? *reinterpret_cast<const float2*>(L + (long)r * ldl + k0 + c) : make_float2(0.f, 0.f);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const int m = j / TPR, jq = j % TPR;
    float2 xj = x[m];
    if (q == jq) {
      xj = pair_mul(xj, rdg[j]);
      x[m] = xj;
    }
    const int src = (lane & ~(TPR - 1)) | jq;
    xj.x = __shfl_sync(0xffffffffu, xj.x, src);
    xj.y = __shfl_sync(0xffffffffu, xj.y, src);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      if (TPR * k + TPR - 1 <= j) continue;   // columns TPR k .. TPR k + TPR - 1 all solved
      const int l = TPR * k + q;
      if (l > j) {
        const float2 v = lkk[l][j];
        df_fma(x[k].x, x[k].y, -xj.x, -xj.y, v.x, v.y);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const int c = TPR * k + q;
    if (r >= n) break;
    const float2 v = pair_add(x[k], make_float2(0.f, 0.f));
    if (c < nb) L[(long)r * ldl + k0 + c] = pair_value(v);
    if (lp) lp[(long)(r - k0 - nb) * NB + c] = c < nb ? v : make_float2(0.f, 0.f);
  }
}

constexpr size_t kTrsmDfSmem = (NB * (NB + 1) + NB) * sizeof(float2);

// pairs of L_kk and of the pivots' reciprocals, per device (the factor's
// panel work runs on one stream per device)
static __device__ float2 g_diag_pairs[NB * NB + NB];

// Panel operand of the tensor-core trailing update: rows [r0, r0 + m) and columns
// [k0, k0 + 256) of the factor, rounded to FP32 and split into three BF16 parts
// S0 = bf16(x), S1 = bf16(x - S0), S2 = bf16(x - S0 - S1) ([3][m_pad][256],
// K-major); rows m..m_pad-1 are zero.
constexpr int kTcPanel = 256;

__global__ void __launch_bounds__(256)
panel_split_kernel(const double* __restrict__ L, long ldl, int r0, int k0, int m, int m_pad,
                   __nv_bfloat16* __restrict__ parts) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long total = (long)m_pad * kTcPanel;
  if (idx >= total) return;
  const int r = (int)(idx / kTcPanel), c = (int)(idx % kTcPanel);
  // rounded to FP32 first (24 bits), which the three BF16 parts then hold exactly
  float x = r < m ? __double2float_rn(L[(long)(r0 + r) * ldl + k0 + c]) : 0.f;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    parts[q * total + idx] = h;
    x = __fsub_rn(x, __bfloat162float(h));
  }
}

// ---------------------------------------------------------------------------
// triangular solves with the factor (lower L; forward L y = b, backward L^T x = y)
//
// The inverses of the 64 x 64 diagonal blocks are formed once after the
// factorisation; each block step of a solve is then one launch in which every
// CTA forms x_k = L_kk^{-1} r_k (a small matrix-vector product) and applies it
// to its share of the remaining rows (forward) or columns (backward).

// Dinv[k] = L_kk^{-1} (lower triangular, 64 x 64, zero above the diagonal). One CTA per block.
__global__ void __launch_bounds__(NB)
diag_inverse_kernel(const double* __restrict__ L, long ldl, int n, double* __restrict__ Dinv) {
  __shared__ double lkk[NB][NB + 1];
  const int k0 = blockIdx.x * NB;
  const int nb = min(NB, n - k0);
  const int j = threadIdx.x;   // column of the inverse
  for (int idx = j; idx < NB * NB; idx += NB) {
    const int r = idx / NB, c = idx % NB;
    lkk[r][c] = (r < nb && c <= r) ? L[(long)(k0 + r) * ldl + k0 + c] : (r == c ? 1.0 : 0.0);
  }
  __syncthreads();
  double x[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    double v = (i == j) ? 1.0 : 0.0;
#pragma unroll
    for (int l = 0; l < i; ++l) v -= lkk[i][l] * x[l];
    x[i] = v / lkk[i][i];
  }
  double* out = Dinv + (long)blockIdx.x * NB * NB;
#pragma unroll
  for (int i = 0; i < NB; ++i) out[i * NB + j] = x[i];
}

// x = Dinv_k^{(T)} v_k for one 64-block: 4 threads per output, 16 products each,
// combined by shuffles (256 threads); result in xk (shared).
__device__ __forceinline__ void block_matvec(const double* __restrict__ D, const double* vk, double* xk,
                                             bool transposed) {
  const int tid = threadIdx.x;
  const int o = tid >> 2, part = tid & 3;
  double acc = 0.0;
  if (o < NB) {
    double a4[4] = {0.0, 0.0, 0.0, 0.0};   // four independent chains: FP64 latency is long
#pragma unroll
    for (int l = part * 16; l < part * 16 + 16; ++l)
      a4[l & 3] = fma(transposed ? D[l * NB + o] : D[o * NB + l], vk[l], a4[l & 3]);
    acc = (a4[0] + a4[1]) + (a4[2] + a4[3]);
  }
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  if (o < NB && part == 0) xk[o] = acc;
}

constexpr int kTriCtas = 304;   // 2 CTAs per SM on 152 SMs

// forward step k: y_k = Dinv_k r_k; r[i] -= L[i][k0:k0+nb] y_k for rows i >= k0 + nb.
// Eight lanes share a row (lane j reads columns j, j+8, ..., j+56: 64 contiguous
// bytes per load instruction and row) and a warp takes 8 rows per pass, so
// every lane has 16 loads in flight; the 8 partial sums meet by shuffles.
// (r and y are read through L2 (ld.cg): inside a persistent sweep, rows written
// by other CTAs in the previous block step must not come from a stale L1 line.)
__device__ __forceinline__ void fwd_step_body(const double* __restrict__ L, long ldl,
                                              const double* __restrict__ Dinv, int k0, int nb, int n,
                                              double* __restrict__ r, double* __restrict__ y) {
  __shared__ double rk[NB], xk[NB];
  const int tid = threadIdx.x;
  if (tid < NB) rk[tid] = tid < nb ? __ldcg(r + k0 + tid) : 0.0;
  __syncthreads();
  block_matvec(Dinv + (long)(k0 / NB) * NB * NB, rk, xk, false);
  __syncthreads();
  if (blockIdx.x == 0 && tid < nb) y[k0 + tid] = xk[tid];
  const int lane = tid & 31, sub = lane & 7, rg = lane >> 3;
  double x[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) x[m] = (8 * m + sub < nb) ? xk[8 * m + sub] : 0.0;
  const int warps = gridDim.x * (blockDim.x >> 5);
  const int base = k0 + nb;
  for (int row0 = base + (blockIdx.x * (blockDim.x >> 5) + (tid >> 5)) * 8; row0 < n; row0 += warps * 8) {
    double sum[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = row0 + 4 * h + rg;
      sum[h] = 0.0;
      if (row < n) {
        const double* Lr = L + (long)row * ldl + k0 + sub;
        double v[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = (8 * m + sub < nb) ? __ldg(Lr + 8 * m) : 0.0;
#pragma unroll
        for (int m = 0; m < 8; ++m) sum[h] = fma(v[m], x[m], sum[h]);
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) sum[h] += __shfl_xor_sync(0xffffffffu, sum[h], o);
      const int row = row0 + 4 * h + rg;
      if (sub == 0 && row < n) r[row] = __ldcg(r + row) - sum[h];
    }
  }
}

__global__ void __launch_bounds__(256)
fwd_step_kernel(const double* __restrict__ L, long ldl, const double* __restrict__ Dinv, int k0, int nb,
                int n, double* __restrict__ r, double* __restrict__ y) {
  fwd_step_body(L, ldl, Dinv, k0, nb, n, r, y);
}

// backward step k: x_k = Dinv_k^T y_k; y[c] -= sum_r L[k0+r][c] x_k[r] for columns c < k0.
// A CTA takes 64 columns; its four 64-thread groups take 16 of the block's rows
// each (coalesced 512-byte row segments) and their partial sums are added in
// a fixed order through shared memory.
__device__ __forceinline__ void bwd_step_body(const double* __restrict__ L, long ldl,
                                              const double* __restrict__ Dinv, int k0, int nb,
                                              double* __restrict__ y, double* __restrict__ x) {
  __shared__ double yk[NB], xk[NB], part[4][NB];
  const int tid = threadIdx.x;
  if (tid < NB) yk[tid] = tid < nb ? __ldcg(y + k0 + tid) : 0.0;
  __syncthreads();
  block_matvec(Dinv + (long)(k0 / NB) * NB * NB, yk, xk, true);
  __syncthreads();
  if (blockIdx.x == 0 && tid < nb) x[k0 + tid] = xk[tid];
  const int cg = tid & 63, rg = tid >> 6;
  for (int c0 = blockIdx.x * 64; c0 < k0; c0 += gridDim.x * 64) {
    const int c = c0 + cg;
    double v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int rr = rg * 16 + u;
      v[u] = (rr < nb && c < k0) ? __ldg(L + (long)(k0 + rr) * ldl + c) : 0.0;
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < 16; ++u) s = fma(v[u], xk[rg * 16 + u], s);
    part[rg][cg] = s;
    __syncthreads();
    if (rg == 0 && c < k0) y[c] = __ldcg(y + c) - ((part[0][cg] + part[1][cg]) + (part[2][cg] + part[3][cg]));
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256)
bwd_step_kernel(const double* __restrict__ L, long ldl, const double* __restrict__ Dinv, int k0, int nb,
                double* __restrict__ y, double* __restrict__ x) {
  bwd_step_body(L, ldl, Dinv, k0, nb, y, x);
}

// Dataflow sweeps: one cooperative launch per substitution. 64-row block b is
// owned by CTA b mod gridDim.x, and owners take their blocks in order. The
// owner of block b accumulates L_bj x_j over the earlier blocks j as soon as
// x_j has been written, then forms x_b = Dinv_b (r_b - sum) and writes it.
// The vector the readers poll is preset (stream-ordered, before the launch)
// to the all-ones bit pattern, a NaN that the sweep's arithmetic on finite
// data never produces, so every 8-byte entry says itself whether it has been
// written: a reader polls the very values it needs (read through L2) until
// none is unset, and the writer needs no fence and no flag. (An 8-byte store
// is seen whole or not at all.) Only the product with the previous block and
// the diagonal solve lie on the critical path of a step. Every wait is
// bounded: on expiry (as also when the data hold that NaN pattern) the kernel
// records a device error and the CTA leaves the sweep. The backward sweep is
// the same on L^T, blocks in decreasing order. All CTAs are co-resident
// (cooperative launch), so an owner never waits on a CTA that is not running.
//
// Two arithmetic forms. FP64 (DF = false): L, Dinv and the polled entries are
// FP64. Double-float (DF = true, the preconditioner inside the solve): L and
// Dinv hold float pairs (hi, lo) in their 8-byte slots, x_j is published as a
// float pair in a separate vector (the FP64 output is written beside it), and
// every product is a pair product summed with two-sum (about 44 significant
// bits, far below the preconditioner's own error) at FP32 rates: on the
// GB300's FP64 units alone a 64 x 64 block product takes ~1.2 us on one SM,
// and a step's critical path holds two of them.
constexpr long long kFlowSpin = 1LL << 22;   // ~1-4 s of polling (one L2 read per poll)
constexpr unsigned char kUnsetByte = 0xFF;   // every byte of an unwritten entry

__device__ __forceinline__ bool entry_set(double v) { return __double_as_longlong(v) != -1LL; }

// a float pair in the 8 bytes of a double (hi in the low word, as a float2 stores it)
__device__ __forceinline__ float2 unpack_pair(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return make_float2(__uint_as_float((unsigned)b), __uint_as_float((unsigned)(b >> 32)));
}
__device__ __forceinline__ double pack_pair(float2 p) {
  return __longlong_as_double(
      (long long)(((unsigned long long)__float_as_uint(p.y) << 32) | (unsigned long long)__float_as_uint(p.x)));
}
__device__ __forceinline__ float2 shfl_xor_pair(float2 a, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, a.x, m), __shfl_xor_sync(0xffffffffu, a.y, m));
}
// four (sum, compensation) accumulators -> one renormalised pair
__device__ __forceinline__ float2 fold4(const float (&s4)[4], const float (&c4)[4]) {
  return pair_add(pair_add(make_float2(s4[0], c4[0]), make_float2(s4[1], c4[1])),
                  pair_add(make_float2(s4[2], c4[2]), make_float2(s4[3], c4[3])));
}

// x = D v (D one 64 x 64 block, transposed or not) with D's 16 values of this
// thread already in registers (thread: output o = tid >> 2, inputs part*16..+15).
__device__ __forceinline__ void block_matvec_reg(const double (&dv)[16], const double* vk, double* xk) {
  const int tid = threadIdx.x;
  const int o = tid >> 2, part = tid & 3;
  double a4[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int q = 0; q < 16; ++q) a4[q & 3] = fma(dv[q], vk[part * 16 + q], a4[q & 3]);
  double acc = (a4[0] + a4[1]) + (a4[2] + a4[3]);
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  if (part == 0) xk[o] = acc;
}

// The same with D and v as packed float pairs; xk[o] gets the packed pair.
__device__ __forceinline__ void block_matvec_pairs(const double (&dv)[16], const double* vk, double* xk) {
  const int tid = threadIdx.x;
  const int o = tid >> 2, part = tid & 3;
  float s4[4] = {0.f, 0.f, 0.f, 0.f}, c4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const float2 d = unpack_pair(dv[q]), v = unpack_pair(vk[part * 16 + q]);
    df_fma(s4[q & 3], c4[q & 3], d.x, d.y, v.x, v.y);
  }
  float2 a = fold4(s4, c4);
  a = pair_add(a, shfl_xor_pair(a, 1));
  a = pair_add(a, shfl_xor_pair(a, 2));
  if (part == 0) xk[o] = pack_pair(a);
}

__device__ __forceinline__ void load_dinv(const double* D, bool transposed, double (&dv)[16]) {
  const int tid = threadIdx.x;
  const int o = tid >> 2, part = tid & 3;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int l = part * 16 + q;
    dv[q] = __ldg(transposed ? D + l * NB + o : D + o * NB + l);
  }
}

// Accumulator of a sweep's block products: FP64, or a double-float
// (sum, compensation) pair fed with packed float-pair operands.
template <bool DF>
struct FlowAcc;
template <>
struct FlowAcc<false> {
  double v = 0.0;
  __device__ __forceinline__ void mac(double l, double x) { v = fma(l, x, v); }
  __device__ __forceinline__ void add(const FlowAcc& o) { v += o.v; }
  __device__ __forceinline__ FlowAcc xor_lane(int m) const {
    FlowAcc a;
    a.v = __shfl_xor_sync(0xffffffffu, v, m);
    return a;
  }
};
template <>
struct FlowAcc<true> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void mac(double l, double x) {
    const float2 a = unpack_pair(l), b = unpack_pair(x);
    df_fma(s, c, a.x, a.y, b.x, b.y);
  }
  __device__ __forceinline__ void add(const FlowAcc& o) {
    const float2 p = pair_add(make_float2(s, c), make_float2(o.s, o.c));
    s = p.x;
    c = p.y;
  }
  __device__ __forceinline__ FlowAcc xor_lane(int m) const {
    FlowAcc a;
    a.s = __shfl_xor_sync(0xffffffffu, s, m);
    a.c = __shfl_xor_sync(0xffffffffu, c, m);
    return a;
  }
};

// rhs - acc as the value the diagonal solve reads: FP64, or a packed pair
// (rp: the right-hand side's pair, split before the wait)
template <bool DF>
__device__ __forceinline__ double rhs_minus(double rv, float2 rp, const FlowAcc<DF>& a);
template <>
__device__ __forceinline__ double rhs_minus<false>(double rv, float2, const FlowAcc<false>& a) {
  return rv - a.v;
}
template <>
__device__ __forceinline__ double rhs_minus<true>(double, float2 rp, const FlowAcc<true>& a) {
  return pack_pair(pair_sub2(rp, a.s, a.c));
}

// Warp-uniform: true once every lane's polled entries are set (re-reading
// them with reload() between polls); false after recording a timeout.
template <typename Ok, typename Reload>
__device__ __forceinline__ bool poll_until_set(Ok ok, Reload reload, int* err) {
  long long it = 0;
  while (!__all_sync(0xffffffffu, ok())) {
    if (++it > kFlowSpin) {
      if ((threadIdx.x & 31) == 0) record_device_error(err, DEV_TIMEOUT);
      return false;
    }
    __nanosleep(32);
    reload();
  }
  return true;
}

// forward: L y = r (r read-only here); readers poll yp (y itself in the FP64
// form, the pair vector in the double-float form), preset to the unset
// pattern. Warp w takes rows 8w..8w+7 of the block; lane l takes columns l
// and l + 32 of every tile (each load instruction reads 256 contiguous bytes
// of one row), and the warp's 8 row sums meet at the end in a shuffle
// reduce-scatter (lane l then holds row 4 b4 + 2 b3 + b2 of its warp, b_k =
// bit k of l). L tiles and x entries are loaded three tiles deep (registers),
// x speculatively: an entry still unset when its tile is used is polled
// again. Dinv_b and r_b are loaded before the walk, so that a step's critical
// path is x_{b-1} and the arithmetic.
template <bool DF>
__global__ void __launch_bounds__(256)
fwd_flow_kernel(const double* __restrict__ L, long ldl, const double* __restrict__ Dinv, int n,
                const double* __restrict__ r, double* __restrict__ y, double* yp, int* err) {
  __shared__ double rb[NB], xb[NB];
  __shared__ int fail;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rs = 4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1);
  const int nblk = (n + NB - 1) / NB;
  if (tid == 0) fail = 0;
  __syncthreads();
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    const int r0 = b * NB, nb = min(NB, n - r0);
    double dv[16];
    load_dinv(Dinv + (long)b * NB * NB, false, dv);
    const int myrow = 8 * warp + rs;
    const double rv = ((lane & 3) == 0 && myrow < nb) ? __ldcg(r + r0 + myrow) : 0.0;
    float2 rp = make_float2(0.f, 0.f);
    if constexpr (DF) rp = to_pair(rv);
    FlowAcc<DF> acc[8];
    auto load_tile = [&](int j, double (&t)[16]) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const double* p = L + (long)min(r0 + 8 * warp + i, n - 1) * ldl + (long)j * NB + lane;
        t[2 * i] = __ldg(p);
        t[2 * i + 1] = __ldg(p + 32);
      }
    };
    auto load_x = [&](int j, double (&xx)[2]) {
      xx[0] = __ldcg(yp + (long)j * NB + lane);
      xx[1] = __ldcg(yp + (long)j * NB + lane + 32);
    };
    auto consume = [&](int j, const double (&t)[16], double (&xx)[2]) -> bool {
      if (!poll_until_set([&] { return entry_set(xx[0]) && entry_set(xx[1]); }, [&] { load_x(j, xx); }, err))
        return false;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        acc[i].mac(t[2 * i], xx[0]);
        acc[i].mac(t[2 * i + 1], xx[1]);
      }
      return true;
    };
    double T0[16], T1[16], T2[16], X0[2], X1[2], X2[2];
    bool ok = true;
    if (b > 0) {
      load_tile(0, T0);
      load_x(0, X0);
    }
    if (b > 1) {
      load_tile(1, T1);
      load_x(1, X1);
    }
    for (int j = 0; j < b; j += 3) {
      if (j + 2 < b) {
        load_tile(j + 2, T2);
        load_x(j + 2, X2);
      }
      if (!(ok = consume(j, T0, X0)) || j + 1 >= b) break;
      if (j + 3 < b) {
        load_tile(j + 3, T0);
        load_x(j + 3, X0);
      }
      if (!(ok = consume(j + 1, T1, X1)) || j + 2 >= b) break;
      if (j + 4 < b) {
        load_tile(j + 4, T1);
        load_x(j + 4, X1);
      }
      if (!(ok = consume(j + 2, T2, X2))) break;
    }
    if (!ok) fail = 1;
    // reduce-scatter of the 8 row sums over the warp's lanes
    {
      const bool h = lane & 16;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        FlowAcc<DF> keep = h ? acc[k + 4] : acc[k];
        keep.add((h ? acc[k] : acc[k + 4]).xor_lane(16));
        acc[k] = keep;
      }
    }
    {
      const bool h = lane & 8;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        FlowAcc<DF> keep = h ? acc[k + 2] : acc[k];
        keep.add((h ? acc[k] : acc[k + 2]).xor_lane(8));
        acc[k] = keep;
      }
    }
    {
      const bool h = lane & 4;
      FlowAcc<DF> keep = h ? acc[1] : acc[0];
      keep.add((h ? acc[0] : acc[1]).xor_lane(4));
      acc[0] = keep;
    }
    acc[0].add(acc[0].xor_lane(2));
    acc[0].add(acc[0].xor_lane(1));
    __syncthreads();
    if (fail) return;
    if ((lane & 3) == 0) rb[myrow] = myrow < nb ? rhs_minus<DF>(rv, rp, acc[0]) : 0.0;
    __syncthreads();
    if constexpr (DF) block_matvec_pairs(dv, rb, xb);
    else block_matvec_reg(dv, rb, xb);
    __syncthreads();
    if (tid < nb) {
      const double v = xb[tid];
      if constexpr (DF) {
        yp[r0 + tid] = v;
        const float2 xx = unpack_pair(v);
        y[r0 + tid] = (double)xx.x + (double)xx.y;
      } else {
        y[r0 + tid] = v;
      }
    }
  }
}

// backward: L^T x = y; block b needs x_j for j > b: x_b = Dinv_b^T (y_b - sum_j
// L_jb^T x_j); readers poll xp (x itself, or the pair vector). Thread
// (c = tid & 63, g = tid >> 6) sums 16 of block j's rows for column c (each
// load instruction reads 256 contiguous bytes of one row); lane l loads entry
// g*16 + (l & 15) of x_j and the warp shares them by shuffles. L tiles and x
// entries are loaded three tiles deep, x speculatively, as in the forward
// sweep.
template <bool DF>
__global__ void __launch_bounds__(256)
bwd_flow_kernel(const double* __restrict__ L, long ldl, const double* __restrict__ Dinv, int n,
                const double* __restrict__ yv, double* __restrict__ x, double* xp, int* err) {
  __shared__ double yb[NB], xb[NB], part[4][NB];
  __shared__ int fail;
  const int tid = threadIdx.x, lane = tid & 31;
  const int c = tid & 63, g = tid >> 6;
  const int nblk = (n + NB - 1) / NB;
  if (tid == 0) fail = 0;
  __syncthreads();
  for (int b = nblk - 1 - blockIdx.x; b >= 0; b -= gridDim.x) {
    const int r0 = b * NB, nb = min(NB, n - r0);
    double dv[16];
    load_dinv(Dinv + (long)b * NB * NB, true, dv);
    const double yr = tid < nb ? __ldcg(yv + r0 + tid) : 0.0;
    float2 yrp = make_float2(0.f, 0.f);
    if constexpr (DF) yrp = to_pair(yr);
    FlowAcc<DF> a4[4];
    const bool colok = c < nb;
    const int xi = g * 16 + (lane & 15);   // entry of x_j this lane loads
    auto load_tile = [&](int j, double (&t)[16]) {
      const int j0 = j * NB, jn = min(NB, n - j0);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int rr = g * 16 + q;
        t[q] = (rr < jn && colok) ? __ldg(L + (long)(j0 + rr) * ldl + r0 + c) : 0.0;
      }
    };
    auto load_x = [&](int j, double& xr) {
      const int j0 = j * NB, jn = min(NB, n - j0);
      xr = xi < jn ? __ldcg(xp + j0 + xi) : 0.0;
    };
    auto consume = [&](int j, const double (&t)[16], double& xr) -> bool {
      const int jn = min(NB, n - j * NB);
      if (!poll_until_set([&] { return xi >= jn || entry_set(xr); }, [&] { load_x(j, xr); }, err)) return false;
#pragma unroll
      for (int q = 0; q < 16; ++q) a4[q & 3].mac(t[q], __shfl_sync(0xffffffffu, xr, q));
      return true;
    };
    double T0[16], T1[16], T2[16], X0 = 0.0, X1 = 0.0, X2 = 0.0;
    bool ok = true;
    const int j_hi = nblk - 1;   // tiles j = j_hi, j_hi - 1, ..., b + 1
    const int cnt = j_hi - b;
    if (cnt > 0) {
      load_tile(j_hi, T0);
      load_x(j_hi, X0);
    }
    if (cnt > 1) {
      load_tile(j_hi - 1, T1);
      load_x(j_hi - 1, X1);
    }
    for (int k = 0; k < cnt; k += 3) {
      if (k + 2 < cnt) {
        load_tile(j_hi - k - 2, T2);
        load_x(j_hi - k - 2, X2);
      }
      if (!(ok = consume(j_hi - k, T0, X0)) || k + 1 >= cnt) break;
      if (k + 3 < cnt) {
        load_tile(j_hi - k - 3, T0);
        load_x(j_hi - k - 3, X0);
      }
      if (!(ok = consume(j_hi - k - 1, T1, X1)) || k + 2 >= cnt) break;
      if (k + 4 < cnt) {
        load_tile(j_hi - k - 4, T1);
        load_x(j_hi - k - 4, X1);
      }
      if (!(ok = consume(j_hi - k - 2, T2, X2))) break;
    }
    if (!ok) fail = 1;
    FlowAcc<DF> sum = a4[0];
    sum.add(a4[1]);
    FlowAcc<DF> s23 = a4[2];
    s23.add(a4[3]);
    sum.add(s23);
    if constexpr (DF) part[g][c] = pack_pair(make_float2(sum.s, sum.c));
    else part[g][c] = sum.v;
    __syncthreads();
    if (fail) return;
    if (tid < NB) {
      if constexpr (DF) {
        const float2 sm = pair_add(pair_add(unpack_pair(part[0][tid]), unpack_pair(part[1][tid])),
                                   pair_add(unpack_pair(part[2][tid]), unpack_pair(part[3][tid])));
        yb[tid] = tid < nb ? pack_pair(pair_sub2(yrp, sm.x, sm.y)) : 0.0;
      } else {
        yb[tid] = tid < nb ? yr - ((part[0][tid] + part[1][tid]) + (part[2][tid] + part[3][tid])) : 0.0;
      }
    }
    __syncthreads();
    if constexpr (DF) block_matvec_pairs(dv, yb, xb);
    else block_matvec_reg(dv, yb, xb);
    __syncthreads();
    if (tid < nb) {
      const double v = xb[tid];
      if constexpr (DF) {
        xp[r0 + tid] = v;
        const float2 xx = unpack_pair(v);
        x[r0 + tid] = (double)xx.x + (double)xx.y;
      } else {
        x[r0 + tid] = v;
      }
    }
  }
}

// FP64 -> float pairs in place over count entries (the diagonal-block inverses)
__global__ void to_pairs_flat_kernel(double* __restrict__ v, long count) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < count) *reinterpret_cast<float2*>(v + idx) = to_pair(v[idx]);
}

constexpr int kMaxFlowBlocks = 4096;   // n <= 262144

// ---------------------------------------------------------------------------
// exact operator pieces: t = Z p (rows), q = Z^T t + lambda p (features).
//
// Z is FP32; p and t are FP64 vectors, carried as float pairs vh + vl with
// vh = fl32(v), vl = fl32(v - vh). Each product z * vh is split exactly into
// its rounded value and its error by one FMA (Dekker's product); the rounded
// products are summed by Knuth's two-sum into a float pair (sum, compensation)
// that also collects the product errors and z * vl (which is ~2^-24 of the
// product), and every kFold terms the pair is folded into an FP64
// accumulator. The sums are those of about twice FP32's precision (error of
// order kFold^2 2^-48 of the sum of |terms| per fold at worst) at FP32
// instruction throughput: in FP64 arithmetic the GB300's FP64 units, not HBM,
// would bound these passes.
constexpr int kFold = 128;

__device__ __forceinline__ void dot2_step(float z, float vh, float vl, float& s, float& c) {
  const float p = __fmul_rn(z, vh);
  const float e = __fmaf_rn(z, vh, -p);
  const float s1 = __fadd_rn(s, p);
  const float bb = __fsub_rn(s1, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(s1, bb)), __fsub_rn(p, bb));
  s = s1;
  c = __fmaf_rn(z, vl, __fadd_rn(c, __fadd_rn(err, e)));
}

__device__ __forceinline__ double fold2(float s, float c) { return (double)s + (double)c; }

// vh, vl <- the float pair of v
__global__ void split_kernel(long n, const double* __restrict__ v, float* __restrict__ vh,
                             float* __restrict__ vl) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = v[i];
  const float h = __double2float_rn(x);
  vh[i] = h;
  vl[i] = __double2float_rn(x - (double)h);
}

// t = Z p: one warp per kZmvRows rows (lanes stride the features), so that each
// load of the pair of p serves kZmvRows products; also writes t's float pair.
constexpr int kZmvRows = 4;

__global__ void __launch_bounds__(256)
zmv_kernel(const float* __restrict__ Z, long n_rows, int n_features, long ldz, const float* __restrict__ ph,
           const float* __restrict__ pl, double* __restrict__ t, float* __restrict__ th,
           float* __restrict__ tl) {
  const long r0 = (((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kZmvRows;
  const int lane = threadIdx.x & 31;
  if (r0 >= n_rows) return;
  const float* zr[kZmvRows];
  float s[kZmvRows], c[kZmvRows];
  double acc[kZmvRows];
#pragma unroll
  for (int k = 0; k < kZmvRows; ++k) {
    zr[k] = Z + min(r0 + k, n_rows - 1) * ldz;   // rows past the end repeat the last (not stored)
    s[k] = c[k] = 0.f;
    acc[k] = 0.0;
  }
  for (int fb = 0; fb < n_features; fb += 32 * kFold) {
    const int fe = min(n_features, fb + 32 * kFold);
#pragma unroll 4
    for (int f = fb + lane; f < fe; f += 32) {
      const float h = __ldg(ph + f), l = __ldg(pl + f);
#pragma unroll
      for (int k = 0; k < kZmvRows; ++k) dot2_step(__ldg(zr[k] + f), h, l, s[k], c[k]);
    }
#pragma unroll
    for (int k = 0; k < kZmvRows; ++k) {
      acc[k] += fold2(s[k], c[k]);
      s[k] = c[k] = 0.f;
    }
  }
#pragma unroll
  for (int k = 0; k < kZmvRows; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
  }
  if (lane < kZmvRows) {
    double v = acc[0];
#pragma unroll
    for (int k = 1; k < kZmvRows; ++k)
      if (lane == k) v = acc[k];
    const long r = r0 + lane;
    if (r < n_rows) {
      t[r] = v;
      const float h = __double2float_rn(v);
      th[r] = h;
      tl[r] = __double2float_rn(v - (double)h);
    }
  }
}

// The same with 16-byte loads (Z rows, ldz and the pair arrays 16-byte aligned,
// n_features a multiple of 4): a warp reads 512 contiguous bytes per row and
// instruction, and each float4 of the operand's pair serves kZmvRows rows.
__global__ void __launch_bounds__(256)
zmv4_kernel(const float* __restrict__ Z, long n_rows, int n_features, long ldz, const float* __restrict__ ph,
            const float* __restrict__ pl, double* __restrict__ t, float* __restrict__ th,
            float* __restrict__ tl) {
  const long r0 = (((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kZmvRows;
  const int lane = threadIdx.x & 31;
  if (r0 >= n_rows) return;
  const float4* zr[kZmvRows];
  float s[kZmvRows], c[kZmvRows];
  double acc[kZmvRows];
#pragma unroll
  for (int k = 0; k < kZmvRows; ++k) {
    zr[k] = reinterpret_cast<const float4*>(Z + min(r0 + k, n_rows - 1) * ldz);
    s[k] = c[k] = 0.f;
    acc[k] = 0.0;
  }
  const float4* h4 = reinterpret_cast<const float4*>(ph);
  const float4* l4 = reinterpret_cast<const float4*>(pl);
  const int n4 = n_features / 4;
  for (int fb = 0; fb < n4; fb += 32 * (kFold / 4)) {
    const int fe = min(n4, fb + 32 * (kFold / 4));
#pragma unroll 2
    for (int f = fb + lane; f < fe; f += 32) {
      const float4 h = __ldg(h4 + f), l = __ldg(l4 + f);
#pragma unroll
      for (int k = 0; k < kZmvRows; ++k) {
        const float4 z = __ldg(zr[k] + f);
        dot2_step(z.x, h.x, l.x, s[k], c[k]);
        dot2_step(z.y, h.y, l.y, s[k], c[k]);
        dot2_step(z.z, h.z, l.z, s[k], c[k]);
        dot2_step(z.w, h.w, l.w, s[k], c[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < kZmvRows; ++k) {
      acc[k] += fold2(s[k], c[k]);
      s[k] = c[k] = 0.f;
    }
  }
#pragma unroll
  for (int k = 0; k < kZmvRows; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
  }
  if (lane < kZmvRows) {
    double v = acc[0];
#pragma unroll
    for (int k = 1; k < kZmvRows; ++k)
      if (lane == k) v = acc[k];
    const long r = r0 + lane;
    if (r < n_rows) {
      t[r] = v;
      const float h = __double2float_rn(v);
      th[r] = h;
      tl[r] = __double2float_rn(v - (double)h);
    }
  }
}

constexpr int kZtRows = 2048;

// part[blk][f] = sum over the block's kZtRows rows r of Z[r][f] t[r] (one thread per feature)
__global__ void __launch_bounds__(256)
ztmv_partial_kernel(const float* __restrict__ Z, long n_rows, int n_features, long ldz,
                    const float* __restrict__ th, const float* __restrict__ tl,
                    double* __restrict__ part) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const long r0 = (long)blockIdx.y * kZtRows;
  const long r1 = min(n_rows, r0 + kZtRows);
  if (f >= n_features) return;
  double acc = 0.0;
  for (long rb = r0; rb < r1; rb += kFold) {
    const long re = min(r1, rb + (long)kFold);
    float s = 0.f, c = 0.f;
#pragma unroll 8
    for (long r = rb; r < re; ++r) dot2_step(__ldg(Z + r * ldz + f), __ldg(th + r), __ldg(tl + r), s, c);
    acc += fold2(s, c);
  }
  part[(long)blockIdx.y * n_features + f] = acc;
}

// Z^T t partial sums ([parts][n]).
static void ztmv_launch(const float* Z, long n_rows, int n, long ldz, const float* th, const float* tl,
                        double* part, int parts, cudaStream_t s) {
  dim3 grid((n + 255) / 256, parts);
  ztmv_partial_kernel<<<grid, 256, 0, s>>>(Z, n_rows, n, ldz, th, tl, part);
}

// (p and q may be the same vector: each thread reads p[f] before it writes q[f])
__global__ void ztmv_finish_kernel(const double* __restrict__ part, int n_parts, int n, const double* p,
                                   double lambda, double* q) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n) return;
  double acc = 0.0;
  for (int k = 0; k < n_parts; ++k) acc += part[(long)k * n + f];
  q[f] = acc + lambda * p[f];
}

// small vector kernels (single CTA reductions keep the order fixed)
__global__ void dot_kernel(const double* __restrict__ a, const double* __restrict__ b, int n,
                           double* __restrict__ out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(a[i], b[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void axpy_kernel(int n, const double* __restrict__ coef, double sign,
                            const double* __restrict__ x, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += sign * (*coef) * x[i];
}

// p = z + (rz_new / rz_old) p
__global__ void pupdate_kernel(int n, const double* __restrict__ rz_new,
                               const double* __restrict__ rz_old, const double* __restrict__ z,
                               double* __restrict__ p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = z[i] + (*rz_new / *rz_old) * p[i];
}

__global__ void maxdiag_kernel(const float* __restrict__ G, int n, double* out) {
  __shared__ double red[1024];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, (double)G[(long)i * n + i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void add_kernel(int n, const double* __restrict__ x, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += x[i];
}

__global__ void ratio_kernel(const double* a, const double* b, double* out) { *out = *a / *b; }

__global__ void sub_kernel(int n, const double* __restrict__ a, const double* __restrict__ b,
                           double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] - b[i];
}

// ---------------------------------------------------------------------------
struct SolveCtx {
  int n;
  long n_rows, ldz;
  const float* Z;
  double lambda;
  double* L;
  long ldl;
  double* part;  // [parts][n]
  int parts;
  double* t;     // [n_rows]
  float *th, *tl;  // float pair of t (or of y) [n_rows]
  float *ph, *pl;  // float pair of the operand [n]
  cudaStream_t s;
};

constexpr size_t kPanelSmem = 2 * NB * (NB + 1) * sizeof(double);

static int cholesky(double* L, long ldl, int n, cudaStream_t s, int* info) {
  int* err = device_error_ptr();
  QMLR_CUDA_TRY(smem_attr_once((const void*)syrk_update_kernel, (int)kPanelSmem));
  QMLR_CUDA_TRY(smem_attr_once((const void*)trsm_panel_kernel, (int)kTrsmSmem));
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int nb = std::min(NB, n - k0);
    potrf_diag_kernel<<<1, 256, 0, s>>>(L, ldl, k0, nb, err, info);
    QMLR_LAUNCH_CHECK();
    const int rows = n - k0 - nb;
    if (rows <= 0) break;
    trsm_panel_kernel<<<(rows + kTrsmRows - 1) / kTrsmRows, 256, kTrsmSmem, s>>>(L, ldl, k0, nb, n, nullptr);
    QMLR_LAUNCH_CHECK();
    const int T = (rows + NB - 1) / NB;
    syrk_update_kernel<<<T * (T + 1) / 2, 256, kPanelSmem, s>>>(L, ldl, k0, nb, n, T);
    QMLR_LAUNCH_CHECK();
  }
  return QMLR_OK;
}

static size_t tc_parts_elems(int n) {
  const long m_pad = ((long)std::max(n, 1) + 127) / 128 * 128;
  return (size_t)3 * m_pad * kTcPanel;
}

// Side stream (highest priority) and events of the mixed factor's lookahead, per device.
struct Lookahead {
  cudaStream_t panel = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

static int lookahead(Lookahead** out) {
  static Lookahead la[64];
  int dev = 0;
  QMLR_CUDA_TRY(cudaGetDevice(&dev));
  QMLR_REQUIRE(dev >= 0 && dev < 64, "device index out of range");
  Lookahead& l = la[dev];
  if (!l.panel) {
    int lo = 0, hi = 0;
    QMLR_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    QMLR_CUDA_TRY(cudaStreamCreateWithPriority(&l.panel, cudaStreamNonBlocking, hi));
    for (int k = 0; k < 4; ++k) QMLR_CUDA_TRY(cudaEventCreateWithFlags(&l.ev[k], cudaEventDisableTiming));
  }
  *out = &l;
  return QMLR_OK;
}

// Mixed-precision factor (the preconditioner of the ridge solve): right-looking
// with 256-column panels. On entry the lower triangle holds float pairs. A
// panel's 64-column blocks are converted to FP64 in turn, factorised (diagonal
// block, triangular solve of the rows below), and applied to the panel's later
// columns in double-float arithmetic; the update of the remaining matrix by
// the whole panel runs on the tensor cores from the panel's 3-way BF16 split
// (products to ~2^-24 relative, FP32 sums per 64-deep K block, subtracted from
// the float pairs). Lookahead: the tensor-core update is issued in two parts,
// first the next panel's columns, then the rest; the next panel's FP64 work
// runs on a high-priority side stream beside the second part (the two touch
// disjoint columns). Two split buffers alternate between panels.
// The lookahead stream, its events and the diagonal-block pairs are one set per
// device, so calls on one device run one at a time: the lock is held until the
// call's work on the device has finished.
static std::mutex& factor_mutex(int dev) {
  static std::mutex mu[64];
  return mu[dev];
}

static int cholesky_mixed_locked(double* L, long ldl, int n, __nv_bfloat16* parts2, cudaStream_t s, int* info);

static int cholesky_mixed(double* L, long ldl, int n, __nv_bfloat16* parts2, cudaStream_t s, int* info) {
  int dev = 0;
  QMLR_CUDA_TRY(cudaGetDevice(&dev));
  QMLR_REQUIRE(dev >= 0 && dev < 64, "device index out of range");
  std::lock_guard<std::mutex> lock(factor_mutex(dev));
  const int rc = cholesky_mixed_locked(L, ldl, n, parts2, s, info);
  const cudaError_t e = cudaStreamSynchronize(s);
  if (rc) return rc;
  QMLR_CUDA_TRY(e);
  return QMLR_OK;
}

static int cholesky_mixed_locked(double* L, long ldl, int n, __nv_bfloat16* parts2, cudaStream_t s, int* info) {
  int* err = device_error_ptr();
  QMLR_CUDA_TRY(smem_attr_once((const void*)syrk_pairs_kernel, (int)kPairsSmem));
  QMLR_CUDA_TRY(smem_attr_once((const void*)trsm_panel_kernel, (int)kTrsmSmem));
  QMLR_CUDA_TRY(smem_attr_once((const void*)trsm_panel_df_kernel, (int)kTrsmDfSmem));
  Lookahead* la = nullptr;
  int rc = lookahead(&la);
  if (rc) return rc;
  cudaStream_t p = la->panel;
  float2* dpairs = nullptr;
  QMLR_CUDA_TRY(cudaGetSymbolAddress(reinterpret_cast<void**>(&dpairs), g_diag_pairs));
  cudaEvent_t ev_start = la->ev[0], ev_split = la->ev[1], ev_next = la->ev[2], ev_end = la->ev[3];
  const size_t half = tc_parts_elems(n);
  QMLR_CUDA_TRY(cudaEventRecord(ev_start, s));
  QMLR_CUDA_TRY(cudaStreamWaitEvent(p, ev_start, 0));
  for (int k0 = 0; k0 < n; k0 += kTcPanel) {
    const int w = std::min(kTcPanel, n - k0);
    __nv_bfloat16* parts = parts2 + ((k0 / kTcPanel) & 1) * half;
    // the solved 64-column block rows as float pairs, in the (then idle) split buffer
    float2* lp = reinterpret_cast<float2*>(parts);
    for (int c0 = k0; c0 < k0 + w; c0 += NB) {
      const int nb = std::min(NB, n - c0);
      potrf_diag_blk_kernel<<<1, kDiagThreads, 0, p>>>(L, ldl, c0, nb, err, info, dpairs);
      QMLR_LAUNCH_CHECK();
      const int rows = n - c0 - nb;
      if (rows <= 0) break;
      const int cblocks = (k0 + w - (c0 + nb) + NB - 1) / NB;   // panel columns still to update
      trsm_panel_df_kernel<<<(rows + kTrsmDfRows - 1) / kTrsmDfRows, 256, kTrsmDfSmem, p>>>(
          L, ldl, c0, nb, n, dpairs, cblocks > 0 ? lp : nullptr);
      QMLR_LAUNCH_CHECK();
      if (cblocks > 0) {
        const int T = (rows + NB - 1) / NB;
        const int tiles = cblocks * T - cblocks * (cblocks - 1) / 2;
        syrk_pairs_kernel<<<tiles, 256, kPairsSmem, p>>>(L, ldl, c0, nb, n, cblocks, lp);
        QMLR_LAUNCH_CHECK();
      }
    }
    const int r0 = k0 + w, m = n - r0;
    if (m <= 0) break;
    const int m_pad = (m + 127) / 128 * 128;
    const long total = (long)m_pad * kTcPanel;
    panel_split_kernel<<<(unsigned)((total + 255) / 256), 256, 0, p>>>(L, ldl, r0, k0, m, m_pad, parts);
    QMLR_LAUNCH_CHECK();
    QMLR_CUDA_TRY(cudaEventRecord(ev_split, p));
    QMLR_CUDA_TRY(cudaStreamWaitEvent(s, ev_split, 0));
    double* A = L + (long)r0 * ldl + r0;
    const uint16_t* pu = reinterpret_cast<const uint16_t*>(parts);
    if ((rc = syrk_tc(pu, total, m, A, ldl, 1, s))) return rc;   // the next panel's columns
    QMLR_CUDA_TRY(cudaEventRecord(ev_next, s));
    QMLR_CUDA_TRY(cudaStreamWaitEvent(p, ev_next, 0));
    if ((rc = syrk_tc(pu, total, m, A, ldl, 2, s))) return rc;   // the rest, beside the next panel
  }
  QMLR_CUDA_TRY(cudaEventRecord(ev_end, p));
  QMLR_CUDA_TRY(cudaStreamWaitEvent(s, ev_end, 0));
  return QMLR_OK;
}


// Grid of the dataflow sweeps (all CTAs co-resident) on the current device;
// 0 when cooperative launch is not available.
static int flow_grid() {
  static int grid[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (grid[dev] == 0) {
    int coop = 0, pf = 0, pb = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    int pf2 = 0, pb2 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pf, fwd_flow_kernel<false>, 256, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pb, bwd_flow_kernel<false>, 256, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pf2, fwd_flow_kernel<true>, 256, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pb2, bwd_flow_kernel<true>, 256, 0);
    const int per_sm = std::min(std::min(std::min(pf, pb), std::min(pf2, pb2)), 2);
    grid[dev] = (coop && per_sm > 0) ? per_sm * sm_count() : -1;
  }
  return grid[dev] > 0 ? grid[dev] : 0;
}

// Whether the dataflow sweeps run for an n x n factor on the current device.
static bool flow_available(int n) {
  const int nblk = (n + NB - 1) / NB;
  return nblk <= kMaxFlowBlocks && flow_grid() > 0;
}

// v <- (L L^T)^{-1} v; tmp is an n-vector of scratch. One dataflow launch per
// sweep where cooperative launch is available (the polled vector preset to
// the unset pattern first), else one launch per block step. pairs == nullptr:
// L and Dinv are FP64. Otherwise they hold float pairs (double-float sweeps,
// which need flow_available(n)) and pairs is an n-vector for the published
// pairs.
static int chol_apply(const double* L, long ldl, const double* Dinv, int n, double* v, double* tmp,
                      cudaStream_t s, double* pairs = nullptr) {
  const int nblk = (n + NB - 1) / NB;
  const int grid = nblk <= kMaxFlowBlocks ? std::min(flow_grid(), nblk) : 0;
  QMLR_REQUIRE(grid || !pairs, "double-float sweeps need a cooperative launch");
  if (grid) {
    int* err = device_error_ptr();
    const bool df = pairs != nullptr;
    const void* fk = df ? (const void*)fwd_flow_kernel<true> : (const void*)fwd_flow_kernel<false>;
    const void* bk = df ? (const void*)bwd_flow_kernel<true> : (const void*)bwd_flow_kernel<false>;
    double* fpoll = df ? pairs : tmp;
    double* bpoll = df ? pairs : v;
    QMLR_CUDA_TRY(cudaMemsetAsync(fpoll, kUnsetByte, (size_t)n * sizeof(double), s));
    {
      void* args[] = {(void*)&L, (void*)&ldl, (void*)&Dinv, (void*)&n, (void*)&v, (void*)&tmp, (void*)&fpoll,
                      (void*)&err};
      QMLR_CUDA_TRY(cudaLaunchCooperativeKernel(fk, grid, 256, args, 0, s));
      count_launch();
    }
    QMLR_CUDA_TRY(cudaMemsetAsync(bpoll, kUnsetByte, (size_t)n * sizeof(double), s));
    {
      void* args[] = {(void*)&L, (void*)&ldl, (void*)&Dinv, (void*)&n, (void*)&tmp, (void*)&v, (void*)&bpoll,
                      (void*)&err};
      QMLR_CUDA_TRY(cudaLaunchCooperativeKernel(bk, grid, 256, args, 0, s));
      count_launch();
    }
    return QMLR_OK;
  }
  // forward: L tmp = v (v is consumed as the running residual)
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int nb = std::min(NB, n - k0);
    const int rows = std::max(n - k0 - nb, 0);
    const int grid = std::min(std::max((rows + 63) / 64, 1), kTriCtas);   // 8 warps x 8 rows
    fwd_step_kernel<<<grid, 256, 0, s>>>(L, ldl, Dinv, k0, nb, n, v, tmp);
    QMLR_LAUNCH_CHECK();
  }
  // backward: L^T v = tmp (tmp is consumed)
  const int last = ((n - 1) / NB) * NB;
  for (int k0 = last; k0 >= 0; k0 -= NB) {
    const int nb = std::min(NB, n - k0);
    const int grid = std::min(std::max((k0 + 63) / 64, 1), kTriCtas);
    bwd_step_kernel<<<grid, 256, 0, s>>>(L, ldl, Dinv, k0, nb, tmp, v);
    QMLR_LAUNCH_CHECK();
  }
  return QMLR_OK;
}

static int diag_inverses(const double* L, long ldl, int n, double* Dinv, cudaStream_t s) {
  diag_inverse_kernel<<<(n + NB - 1) / NB, NB, 0, s>>>(L, ldl, n, Dinv);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

static int apply_exact(const SolveCtx& c, const double* p, double* q) {
  const long threads = (c.n_rows + kZmvRows - 1) / kZmvRows * 32;
  if (c.n_rows > 0) {
    split_kernel<<<(c.n + 255) / 256, 256, 0, c.s>>>(c.n, p, c.ph, c.pl);
    QMLR_LAUNCH_CHECK();
    const bool vec = (c.n % 4 == 0) && (c.ldz % 4 == 0) && ((reinterpret_cast<uintptr_t>(c.Z) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(c.ph) & 15) == 0) && ((reinterpret_cast<uintptr_t>(c.pl) & 15) == 0);
    if (vec)
      zmv4_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, c.s>>>(c.Z, c.n_rows, c.n, c.ldz, c.ph, c.pl,
                                                                      c.t, c.th, c.tl);
    else
      zmv_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, c.s>>>(c.Z, c.n_rows, c.n, c.ldz, c.ph, c.pl,
                                                                     c.t, c.th, c.tl);
    QMLR_LAUNCH_CHECK();
    ztmv_launch(c.Z, c.n_rows, c.n, c.ldz, c.th, c.tl, c.part, c.parts, c.s);
    QMLR_LAUNCH_CHECK();
  } else {
    QMLR_CUDA_TRY(cudaMemsetAsync(c.part, 0, sizeof(double) * c.n, c.s));
  }
  ztmv_finish_kernel<<<(c.n + 255) / 256, 256, 0, c.s>>>(c.part, c.n_rows > 0 ? c.parts : 1, c.n,
                                                        p, c.lambda, q);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

}  // namespace qmlr

using namespace qmlr;

extern "C" int64_t qmlr_solve_workspace_bytes(int64_t n_rows, int32_t n_features) {
  const int64_t n = n_features;
  const int64_t parts = std::max<int64_t>((n_rows + kZtRows - 1) / kZtRows, 1);
  const int64_t nblk = (n + NB - 1) / NB;
  return n * n * 8                 // factor L
         + nblk * NB * NB * 8      // inverses of the diagonal blocks
         + n * 8                   // triangular-solve scratch
         + parts * n * 8           // partial sums of Z^T t
         + std::max<int64_t>(n_rows, 1) * 16  // t = Z p and its float pair
         + n * 8                   // float pair of the operand
         + 7 * n * 8               // c, r, z, p, q, tmp, published float pairs of the sweeps
         + (int64_t)tc_parts_elems((int)n) * 4   // two split panels of the mixed-precision factor
         + 8 * 8 + 8192;           // scalars + alignment
}

extern "C" int qmlr_cholesky(double* L, int64_t ldl, int32_t n, int32_t* host_info, void* stream) {
  QMLR_REQUIRE(L && n >= 1 && ldl >= n, "bad factor arguments");
  cudaStream_t s = as_stream(stream);
  int* info = nullptr;
  QMLR_CUDA_TRY(cudaMallocAsync(&info, sizeof(int), s));
  QMLR_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int), s));
  int rc = cholesky(L, ldl, n, s, info);
  int h = 0;
  if (rc == QMLR_OK) {
    QMLR_CUDA_TRY(cudaMemcpyAsync(&h, info, sizeof(int), cudaMemcpyDeviceToHost, s));
    QMLR_CUDA_TRY(cudaStreamSynchronize(s));
  }
  cudaFreeAsync(info, s);
  if (host_info) *host_info = h;
  return rc;
}

extern "C" int64_t qmlr_cholesky_mixed_workspace_bytes(int32_t n) {
  if (n < 1) return 0;
  return (int64_t)tc_parts_elems(n) * 4 + 256;
}

extern "C" int qmlr_cholesky_mixed(double* L, int64_t ldl, int32_t n, void* work, int64_t work_bytes,
                                   int32_t* host_info, void* stream) {
  QMLR_REQUIRE(L && n >= 1 && ldl >= n, "bad factor arguments");
  QMLR_REQUIRE(work && work_bytes >= qmlr_cholesky_mixed_workspace_bytes(n), "workspace too small");
  QMLR_REQUIRE((reinterpret_cast<uintptr_t>(work) & 255) == 0, "workspace must be 256-byte aligned");
  cudaStream_t s = as_stream(stream);
  int* info = nullptr;
  QMLR_CUDA_TRY(cudaMallocAsync(&info, sizeof(int), s));
  QMLR_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int), s));
  const long nn = (long)n * n;
  to_pairs_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(L, ldl, n);
  QMLR_LAUNCH_CHECK();
  int rc = cholesky_mixed(L, ldl, n, static_cast<__nv_bfloat16*>(work), s, info);
  int h = 0;
  if (rc == QMLR_OK) {
    QMLR_CUDA_TRY(cudaMemcpyAsync(&h, info, sizeof(int), cudaMemcpyDeviceToHost, s));
    QMLR_CUDA_TRY(cudaStreamSynchronize(s));
  }
  cudaFreeAsync(info, s);
  if (host_info) *host_info = h;
  return rc;
}

extern "C" int qmlr_cholesky_solve(const double* L, int64_t ldl, int32_t n, double* v, void* stream) {
  QMLR_REQUIRE(L && v && n >= 1 && ldl >= n, "bad arguments");
  cudaStream_t s = as_stream(stream);
  const int nblk = (n + NB - 1) / NB;
  double* buf = nullptr;
  QMLR_CUDA_TRY(cudaMallocAsync(&buf, sizeof(double) * ((size_t)nblk * NB * NB + n), s));
  int rc = diag_inverses(L, ldl, n, buf, s);
  if (rc == QMLR_OK) rc = chol_apply(L, ldl, buf, n, v, buf + (size_t)nblk * NB * NB, s);
  cudaFreeAsync(buf, s);
  return rc;
}

static void carve(char*& p, void** out, size_t bytes) {
  *out = p;
  p += (bytes + 255) & ~size_t(255);
}

extern "C" int64_t qmlr_normal_apply_workspace_bytes(int64_t n_rows, int32_t n_features) {
  const int64_t n = n_features;
  const int64_t parts = std::max<int64_t>((n_rows + kZtRows - 1) / kZtRows, 1);
  return parts * n * 8 + std::max<int64_t>(n_rows, 1) * 16 + n * 8 + 4 * 256;
}

extern "C" int qmlr_normal_apply(const float* Z, int64_t n_rows, int32_t n_features, int64_t ldz, double lambda,
                                 const double* p, double* q, void* work, int64_t work_bytes, void* stream) {
  QMLR_REQUIRE(p && q, "NULL pointer argument");
  QMLR_REQUIRE(n_features >= 1 && n_rows >= 0 && ldz >= n_features, "bad shapes");
  QMLR_REQUIRE(n_rows == 0 || Z, "Z is NULL");
  QMLR_REQUIRE(work && work_bytes >= qmlr_normal_apply_workspace_bytes(n_rows, n_features),
               "workspace too small");
  SolveCtx c{};
  c.n = n_features;
  c.n_rows = n_rows;
  c.ldz = ldz;
  c.Z = Z;
  c.lambda = lambda;
  c.s = as_stream(stream);
  c.parts = (int)std::max<int64_t>((n_rows + kZtRows - 1) / kZtRows, 1);
  char* w = static_cast<char*>(work);
  void *vpart, *vt, *vth, *vph;
  carve(w, &vpart, (size_t)c.parts * c.n * 8);
  carve(w, &vt, (size_t)std::max<int64_t>(n_rows, 1) * 8);
  carve(w, &vth, (size_t)std::max<int64_t>(n_rows, 1) * 8);
  carve(w, &vph, (size_t)c.n * 8);
  c.part = static_cast<double*>(vpart);
  c.t = static_cast<double*>(vt);
  c.th = static_cast<float*>(vth);
  c.tl = c.th + std::max<int64_t>(n_rows, 1);
  c.ph = static_cast<float*>(vph);
  c.pl = c.ph + c.n;
  return apply_exact(c, p, q);
}

extern "C" int qmlr_gram_solve(const float* G, const float* Z, int64_t n_rows, int32_t n_features,
                               int64_t ldz, const double* y, double lambda, qmlr_solve_opts* opts,
                               double* alpha, void* work, int64_t work_bytes, void* stream) {
  QMLR_REQUIRE(G && alpha && opts, "NULL pointer argument");
  QMLR_REQUIRE(n_features >= 1 && n_rows >= 0 && ldz >= n_features, "bad shapes");
  QMLR_REQUIRE(n_rows == 0 || (Z && y), "Z/y are NULL");
  QMLR_REQUIRE(lambda >= 0, "lambda must be >= 0");
  QMLR_REQUIRE(opts->max_iter >= 0, "max_iter must be >= 0");
  QMLR_REQUIRE(work && work_bytes >= qmlr_solve_workspace_bytes(n_rows, n_features),
               "workspace too small");
  QMLR_REQUIRE(opts->method == QMLR_SOLVE_PCG || opts->method == QMLR_SOLVE_REFINE,
               "unknown solve method %d", opts->method);
  QMLR_REQUIRE(opts->factor == QMLR_FACTOR_FP64 || opts->factor == QMLR_FACTOR_MIXED,
               "unknown factor kind %d", opts->factor);
  cudaStream_t s = as_stream(stream);
  const int n = n_features;
  SolveCtx c;
  c.n = n;
  c.n_rows = n_rows;
  c.ldz = ldz;
  c.Z = Z;
  c.lambda = lambda;
  c.ldl = n;
  c.s = s;
  c.parts = (int)std::max<int64_t>((n_rows + kZtRows - 1) / kZtRows, 1);
  char* p = static_cast<char*>(work);
  void *vL, *vpart, *vt, *vc, *vr, *vz, *vp, *vq, *vtmp, *vsc, *vdinv, *vtri, *vsplit, *vth, *vph, *vpub;
  const int nblk = (n + NB - 1) / NB;
  carve(p, &vL, (size_t)n * n * 8);
  carve(p, &vdinv, (size_t)nblk * NB * NB * 8);
  carve(p, &vtri, (size_t)n * 8);
  carve(p, &vpart, (size_t)c.parts * n * 8);
  carve(p, &vt, (size_t)std::max<int64_t>(n_rows, 1) * 8);
  carve(p, &vc, (size_t)n * 8);
  carve(p, &vr, (size_t)n * 8);
  carve(p, &vz, (size_t)n * 8);
  carve(p, &vp, (size_t)n * 8);
  carve(p, &vq, (size_t)n * 8);
  carve(p, &vtmp, (size_t)n * 8);
  carve(p, &vsc, 8 * 8);
  carve(p, &vsplit, tc_parts_elems(n) * 4);
  carve(p, &vth, (size_t)std::max<int64_t>(n_rows, 1) * 8);
  carve(p, &vph, (size_t)n * 8);
  carve(p, &vpub, (size_t)n * 8);
  c.L = static_cast<double*>(vL);
  c.part = static_cast<double*>(vpart);
  c.t = static_cast<double*>(vt);
  c.th = static_cast<float*>(vth);
  c.tl = c.th + std::max<int64_t>(n_rows, 1);
  c.ph = static_cast<float*>(vph);
  c.pl = c.ph + n;
  double *cv = static_cast<double*>(vc), *r = static_cast<double*>(vr), *z = static_cast<double*>(vz);
  double *pv = static_cast<double*>(vp), *q = static_cast<double*>(vq);
  double* sc = static_cast<double*>(vsc);
  double* Dinv = static_cast<double*>(vdinv);
  double* tri = static_cast<double*>(vtri);   // [0]=rz, [1]=rz_new, [2]=pq, [3]=a, [4]=rr, [5]=cc
  int* info = reinterpret_cast<int*>(sc + 7);
  const int vb = (n + 255) / 256;

  // right-hand side c = Z^T y
  if (n_rows > 0) {
    split_kernel<<<(unsigned)((n_rows + 255) / 256), 256, 0, s>>>(n_rows, y, c.th, c.tl);
    QMLR_LAUNCH_CHECK();
    ztmv_launch(Z, n_rows, n, ldz, c.th, c.tl, c.part, c.parts, s);
    QMLR_LAUNCH_CHECK();
    ztmv_finish_kernel<<<vb, 256, 0, s>>>(c.part, c.parts, n, cv, 0.0, cv);
    QMLR_LAUNCH_CHECK();
  } else {
    QMLR_CUDA_TRY(cudaMemsetAsync(cv, 0, sizeof(double) * n, s));
  }
  // factor of G + (lambda + shift) I; a negative opts->shift means |shift| * max_i G_ii.
  // A non-positive pivot (the low-precision Gram can be slightly indefinite)
  // raises the shift tenfold, up to 8 times.
  double shift = opts->shift;
  if (shift < 0) {
    maxdiag_kernel<<<1, 1024, 0, s>>>(G, n, sc + 6);
    QMLR_LAUNCH_CHECK();
    double md = 0;
    QMLR_CUDA_TRY(cudaMemcpyAsync(&md, sc + 6, sizeof(double), cudaMemcpyDeviceToHost, s));
    QMLR_CUDA_TRY(cudaStreamSynchronize(s));
    shift = -shift * md;
  }
  const long nn = (long)n * n;
  int hinfo = 0;
  cudaEvent_t ev[3];
  for (int k = 0; k < 3; ++k) QMLR_CUDA_TRY(cudaEventCreate(&ev[k]));
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() {
      for (int k = 0; k < 3; ++k) cudaEventDestroy(e[k]);
    }
  } ev_guard{ev};
  QMLR_CUDA_TRY(cudaEventRecord(ev[0], s));
  for (int attempt = 0;; ++attempt) {
    if (opts->factor == QMLR_FACTOR_MIXED)
      assemble_pairs_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(G, n, lambda + shift, c.L, c.ldl);
    else
      assemble_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(G, n, lambda + shift, c.L, c.ldl);
    QMLR_LAUNCH_CHECK();
    QMLR_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int), s));
    int rc = opts->factor == QMLR_FACTOR_MIXED
                 ? cholesky_mixed(c.L, c.ldl, n, static_cast<__nv_bfloat16*>(vsplit), s, info)
                 : cholesky(c.L, c.ldl, n, s, info);
    if (rc) return rc;
    QMLR_CUDA_TRY(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
    QMLR_CUDA_TRY(cudaStreamSynchronize(s));
    if (hinfo == 0) break;
    int32_t code;
    qmlr_device_status(stream, &code);   // clear the recorded pivot failure
    if (attempt == 8) {
      set_error("Cholesky factorisation failed at column %d with shift %.3e "
                "(matrix not positive definite)", hinfo, shift);
      return QMLR_EINVAL;
    }
    shift = shift > 0 ? 10.0 * shift : 1e-12;
  }
  opts->shift_used = shift;
  {
    int rc0 = diag_inverses(c.L, c.ldl, n, Dinv, s);
    if (rc0) return rc0;
  }
  // The preconditioner's sweeps in double-float: L (lower triangle) and the
  // diagonal-block inverses become float pairs in place.
  double* pub = nullptr;
  if (flow_available(n)) {
    pub = static_cast<double*>(vpub);
    to_pairs_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(c.L, c.ldl, n);
    QMLR_LAUNCH_CHECK();
    const long nd = (long)nblk * NB * NB;
    to_pairs_flat_kernel<<<(unsigned)((nd + 255) / 256), 256, 0, s>>>(Dinv, nd);
    QMLR_LAUNCH_CHECK();
  }
  QMLR_CUDA_TRY(cudaEventRecord(ev[1], s));
  int rc = QMLR_OK;
  // alpha = M^{-1} c
  QMLR_CUDA_TRY(cudaMemcpyAsync(alpha, cv, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  if ((rc = chol_apply(c.L, c.ldl, Dinv, n, alpha, tri, s, pub))) return rc;
  dot_kernel<<<1, 1024, 0, s>>>(cv, cv, n, sc + 5);
  QMLR_LAUNCH_CHECK();
  // r = c - A alpha
  if ((rc = apply_exact(c, alpha, q))) return rc;
  sub_kernel<<<vb, 256, 0, s>>>(n, cv, q, r);
  QMLR_LAUNCH_CHECK();
  double h[2];
  auto residual = [&](double* out) -> int {
    dot_kernel<<<1, 1024, 0, s>>>(r, r, n, sc + 4);
    QMLR_LAUNCH_CHECK();
    QMLR_CUDA_TRY(cudaMemcpyAsync(h, sc + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    QMLR_CUDA_TRY(cudaStreamSynchronize(s));
    *out = sqrt(h[0]) / std::max(sqrt(h[1]), 1e-300);
    return QMLR_OK;
  };
  double rel = 0;
  if ((rc = residual(&rel))) return rc;
  int it = 0;
  if (opts->method == QMLR_SOLVE_REFINE) {
    // alpha += M^{-1} r ; r = c - A alpha
    for (; it < opts->max_iter && rel > opts->tol; ++it) {
      QMLR_CUDA_TRY(cudaMemcpyAsync(z, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      if ((rc = chol_apply(c.L, c.ldl, Dinv, n, z, tri, s, pub))) return rc;
      add_kernel<<<vb, 256, 0, s>>>(n, z, alpha);
      QMLR_LAUNCH_CHECK();
      if ((rc = apply_exact(c, alpha, q))) return rc;
      sub_kernel<<<vb, 256, 0, s>>>(n, cv, q, r);
      QMLR_LAUNCH_CHECK();
      if ((rc = residual(&rel))) return rc;
    }
  } else {
    // preconditioned conjugate gradients on the exact operator
    QMLR_CUDA_TRY(cudaMemcpyAsync(z, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if ((rc = chol_apply(c.L, c.ldl, Dinv, n, z, tri, s, pub))) return rc;
    QMLR_CUDA_TRY(cudaMemcpyAsync(pv, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    dot_kernel<<<1, 1024, 0, s>>>(r, z, n, sc + 0);
    QMLR_LAUNCH_CHECK();
    for (; it < opts->max_iter && rel > opts->tol; ++it) {
      if ((rc = apply_exact(c, pv, q))) return rc;
      dot_kernel<<<1, 1024, 0, s>>>(pv, q, n, sc + 2);
      QMLR_LAUNCH_CHECK();
      ratio_kernel<<<1, 1, 0, s>>>(sc + 0, sc + 2, sc + 3);
      QMLR_LAUNCH_CHECK();
      axpy_kernel<<<vb, 256, 0, s>>>(n, sc + 3, 1.0, pv, alpha);
      QMLR_LAUNCH_CHECK();
      axpy_kernel<<<vb, 256, 0, s>>>(n, sc + 3, -1.0, q, r);
      QMLR_LAUNCH_CHECK();
      if ((rc = residual(&rel))) return rc;
      if (rel <= opts->tol) {
        ++it;
        break;
      }
      QMLR_CUDA_TRY(cudaMemcpyAsync(z, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      if ((rc = chol_apply(c.L, c.ldl, Dinv, n, z, tri, s, pub))) return rc;
      dot_kernel<<<1, 1024, 0, s>>>(r, z, n, sc + 1);
      QMLR_LAUNCH_CHECK();
      pupdate_kernel<<<vb, 256, 0, s>>>(n, sc + 1, sc + 0, z, pv);
      QMLR_LAUNCH_CHECK();
      QMLR_CUDA_TRY(cudaMemcpyAsync(sc + 0, sc + 1, sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
  }
  QMLR_CUDA_TRY(cudaEventRecord(ev[2], s));
  QMLR_CUDA_TRY(cudaEventSynchronize(ev[2]));
  cudaEventElapsedTime(&opts->factor_ms, ev[0], ev[1]);
  cudaEventElapsedTime(&opts->refine_ms, ev[1], ev[2]);
  opts->iters_done = it;
  opts->rel_resid = rel;
  if (rel > opts->tol) {
    set_error("refinement stopped at relative residual %.3e after %d iterations", rel, it);
    return QMLR_ENOTCONV;
  }
  return QMLR_OK;
}
