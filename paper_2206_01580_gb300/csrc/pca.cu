// Per-element PCA basis U_e on the GPU (setup step, once per model).
//
// SORF section of the paper: the representations of element e are the
// columns of Z~_e = U_e S_e V_e^T; the projection keeps the first N_PCA = d
// columns of U_e, i.e. the leading eigenvectors of C_e = Z~_e Z~_e^T =
// sum_i rho_i rho_i^T (uncentred).
//
// Method (all FP64, small sizes): C_e by a tiled SYRK over the element's
// atoms; randomized subspace iteration for the leading l = d + 32 directions
// (Halko, Martinsson, Tropp 2011: Y = C Omega, then q rounds of
// orthonormalise-and-multiply), orthonormalisation by modified Gram-Schmidt
// applied twice, Rayleigh-Ritz B = Q^T C Q, and a cyclic Jacobi
// eigensolver for B in one CTA. U_e = Q W (first d Ritz vectors by
// descending eigenvalue), each column signed so that its largest-magnitude
// entry is positive; columns whose eigenvalue is <= 1e-12 of the largest are
// zero (rank-deficient elements). The random test matrix comes from a
// counter-based splitmix64 hash (Steele, Lea, Flood 2014) with Box-Muller.
#include "common.cuh"

namespace qmlr {

constexpr int kPcaOversample = 32;
constexpr int kPcaPowerIters = 6;
constexpr int kJacobiSweeps = 30;
constexpr int kMaxL = 160;

// C[i][j] = sum_r X[perm[r]][i] X[perm[r]][j], rows r in [0, n), FP64, 32x32 tiles.
__global__ void syrk_f64_kernel(const float* __restrict__ rep, int ld, int R, const int32_t* __restrict__ rows,
                                int n, double* __restrict__ C) {
  __shared__ double a[16][33], b[16][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // 32 x 8 threads, 4 outputs each
  double acc[4] = {0, 0, 0, 0};
  for (int r0 = 0; r0 < n; r0 += 16) {
    for (int k = threadIdx.x; k < 16 * 32; k += blockDim.x) {
      const int rr = k / 32, cc = k % 32;
      const int r = r0 + rr;
      const long row = r < n ? rows[r] : -1;
      a[rr][cc] = (row >= 0 && i0 + cc < R) ? (double)rep[row * ld + i0 + cc] : 0.0;
      b[rr][cc] = (row >= 0 && j0 + cc < R) ? (double)rep[row * ld + j0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) {
      const double bv = b[rr][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fma(a[rr][ty + 8 * u], bv, acc[u]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + ty + 8 * u, j = j0 + tx;
    if (i < R && j < R) C[(long)i * R + j] = acc[u];
  }
}

// C[M][N] = op(A) B, A [M][K] (or [K][M] when transA), B [K][N], row-major FP64.
__global__ void dgemm_kernel(const double* __restrict__ A, const double* __restrict__ B,
                             double* __restrict__ Cm, int M, int N, int K, int transA) {
  __shared__ double a[16][33], b[16][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  double acc[4] = {0, 0, 0, 0};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int k = threadIdx.x; k < 16 * 32; k += blockDim.x) {
      const int kk = k / 32, cc = k % 32;
      const int kr = k0 + kk;
      double av = 0.0;
      if (kr < K && i0 + cc < M) av = transA ? A[(long)kr * M + i0 + cc] : A[(long)(i0 + cc) * K + kr];
      a[kk][cc] = av;
      b[kk][cc] = (kr < K && j0 + cc < N) ? B[(long)kr * N + j0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const double bv = b[kk][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fma(a[kk][ty + 8 * u], bv, acc[u]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + ty + 8 * u, j = j0 + tx;
    if (i < M && j < N) Cm[(long)i * N + j] = acc[u];
  }
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void gaussian_kernel(double* __restrict__ out, long n, uint64_t seed) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t h1 = splitmix64(seed ^ (2 * (uint64_t)i));
  const uint64_t h2 = splitmix64(seed ^ (2 * (uint64_t)i + 1));
  const double u1 = ((h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  const double u2 = ((h2 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  out[i] = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// Modified Gram-Schmidt on the l columns of Y [R][l] (in place), twice. One CTA.
__global__ void mgs_kernel(double* __restrict__ Y, int R, int l) {
  __shared__ double red[1024];
  __shared__ double coef[kMaxL];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int pass = 0; pass < 2; ++pass) {
    for (int j = 0; j < l; ++j) {
      // norm of column j
      double s = 0.0;
      for (int r = tid; r < R; r += nt) s = fma(Y[(long)r * l + j], Y[(long)r * l + j], s);
      red[tid] = s;
      __syncthreads();
      for (int w = nt / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
      }
      const double nrm = sqrt(red[0]);
      __syncthreads();
      const double inv = nrm > 1e-280 ? 1.0 / nrm : 0.0;
      for (int r = tid; r < R; r += nt) Y[(long)r * l + j] *= inv;
      __syncthreads();
      // coefficients against later columns: coef[k] = y_j . y_k
      for (int k = j + 1 + tid / 32; k < l; k += nt / 32) {
        double c = 0.0;
        for (int r = tid % 32; r < R; r += 32) c = fma(Y[(long)r * l + j], Y[(long)r * l + k], c);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (tid % 32 == 0) coef[k] = c;
      }
      __syncthreads();
      for (long idx = tid; idx < (long)R * (l - j - 1); idx += nt) {
        const int r = (int)(idx / (l - j - 1)), k = j + 1 + (int)(idx % (l - j - 1));
        Y[(long)r * l + k] -= coef[k] * Y[(long)r * l + j];
      }
      __syncthreads();
    }
  }
}

// Cyclic Jacobi for symmetric B [l][l] (round-robin pairs, rows then columns).
// Outputs eigenvalues lam[l] and eigenvectors as columns of V [l][l]. One CTA.
__global__ void jacobi_kernel(const double* __restrict__ Bg, int l, double* __restrict__ V,
                              double* __restrict__ lam) {
  extern __shared__ double A[];        // [lp][lp]
  __shared__ double cs[kMaxL / 2], sn[kMaxL / 2];
  __shared__ int pp[kMaxL / 2], qq[kMaxL / 2];
  const int lp = l + (l & 1);          // even count: index l is a dummy
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < lp * lp; idx += nt) {
    const int i = idx / lp, j = idx % lp;
    A[idx] = (i < l && j < l) ? Bg[(long)i * l + j] : 0.0;
  }
  for (int idx = tid; idx < l * l; idx += nt) V[idx] = (idx / l == idx % l) ? 1.0 : 0.0;
  __syncthreads();
  const int half = lp / 2;
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    for (int step = 0; step < lp - 1; ++step) {
      // circle-method round robin: (step, lp-1) and (step+k, step-k) mod (lp-1)
      for (int k = tid; k < half; k += nt) {
        int a, b;
        if (k == 0) {
          a = step;
          b = lp - 1;
        } else {
          a = (step + k) % (lp - 1);
          b = (step - k + (lp - 1)) % (lp - 1);
        }
        const int p = min(a, b), q = max(a, b);
        double c = 1.0, sv = 0.0;
        if (q < l) {
          const double apq = A[p * lp + q];
          const double app = A[p * lp + p], aqq = A[q * lp + q];
          if (fabs(apq) > 1e-300 && fabs(apq) > 1e-18 * sqrt(fabs(app * aqq))) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            sv = t * c;
          }
        }
        pp[k] = p;
        qq[k] = q;
        cs[k] = c;
        sn[k] = sv;
      }
      __syncthreads();
      // rows p, q
      for (int idx = tid; idx < half * lp; idx += nt) {
        const int k = idx / lp, j = idx % lp;
        if (sn[k] == 0.0) continue;
        const int p = pp[k], q = qq[k];
        const double ap = A[p * lp + j], aq = A[q * lp + j];
        A[p * lp + j] = cs[k] * ap - sn[k] * aq;
        A[q * lp + j] = sn[k] * ap + cs[k] * aq;
      }
      __syncthreads();
      // columns p, q of A and of V
      for (int idx = tid; idx < half * lp; idx += nt) {
        const int k = idx / lp, i = idx % lp;
        if (sn[k] == 0.0) continue;
        const int p = pp[k], q = qq[k];
        const double ap = A[i * lp + p], aq = A[i * lp + q];
        A[i * lp + p] = cs[k] * ap - sn[k] * aq;
        A[i * lp + q] = sn[k] * ap + cs[k] * aq;
        if (i < l && q < l) {
          const double vp = V[(long)i * l + p], vq = V[(long)i * l + q];
          V[(long)i * l + p] = cs[k] * vp - sn[k] * vq;
          V[(long)i * l + q] = sn[k] * vp + cs[k] * vq;
        }
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < l; i += nt) lam[i] = A[i * lp + i];
}

// U_e[:, c] = sign * Q W[:, order[c]] for the d leading Ritz pairs; zero below rank.
__global__ void pca_finish_kernel(const double* __restrict__ Q, const double* __restrict__ W,
                                  const double* __restrict__ lam, int R, int l, int d, int rep_dim,
                                  float* __restrict__ U) {
  __shared__ int order[kMaxL];
  __shared__ double sgn[kMaxL];
  __shared__ double lmax;
  const int tid = threadIdx.x, nt = blockDim.x;
  // rank of each eigenvalue (descending, ties by index)
  for (int i = tid; i < l; i += nt) {
    int rank = 0;
    for (int j = 0; j < l; ++j) rank += (lam[j] > lam[i]) || (lam[j] == lam[i] && j < i);
    order[rank] = i;
  }
  __syncthreads();
  if (tid == 0) lmax = fmax(lam[order[0]], 0.0);
  __syncthreads();
  // sign: the largest-magnitude entry of each kept column is positive (lowest row on ties)
  for (int c = tid / 32; c < d; c += nt / 32) {
    double best = -1.0, val = 0.0;
    int brow = 1 << 30;
    if (c < l) {
      const int e = order[c];
      for (int r = tid % 32; r < rep_dim; r += 32) {
        double u = 0.0;
        for (int k = 0; k < l; ++k) u = fma(Q[(long)r * l + k], W[(long)k * l + e], u);
        if (fabs(u) > best) {
          best = fabs(u);
          val = u;
          brow = r;
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const double ov = __shfl_xor_sync(0xffffffffu, val, o);
      const int orow = __shfl_xor_sync(0xffffffffu, brow, o);
      if (ob > best || (ob == best && orow < brow)) {
        best = ob;
        val = ov;
        brow = orow;
      }
    }
    if (tid % 32 == 0) sgn[c] = val < 0 ? -1.0 : 1.0;
  }
  __syncthreads();
  for (long idx = tid; idx < (long)rep_dim * d; idx += nt) {
    const int r = (int)(idx / d), c = (int)(idx % d);
    double u = 0.0;
    if (c < l) {
      const int e = order[c];
      const bool keep = lmax > 0 && lam[e] > 1e-12 * lmax;
      if (keep) {
        for (int k = 0; k < l; ++k) u = fma(Q[(long)r * l + k], W[(long)k * l + e], u);
        u *= sgn[c];
      }
    }
    U[idx] = (float)u;
  }
}

}  // namespace qmlr

using namespace qmlr;

extern "C" int64_t qmlr_pca_workspace_bytes(int32_t rep_ld, int32_t d) {
  const int64_t R = rep_ld, l = std::min<int64_t>(d + kPcaOversample, R);
  return (R * R + 3 * R * l + 2 * l * l + 2 * l) * 8 + 8 * 256;
}

extern "C" int qmlr_pca_fit(const float* rep, int32_t rep_ld, int32_t rep_dim, const int32_t* perm,
                            const int32_t* elem_offsets, int32_t n_el, int32_t max_per_element,
                            int32_t d, float* U, void* work, int64_t work_bytes, void* stream) {
  QMLR_REQUIRE(rep && perm && elem_offsets && U && work, "NULL pointer argument");
  QMLR_REQUIRE(n_el >= 1 && n_el <= 8, "n_el must be in 1..8");
  QMLR_REQUIRE(rep_dim >= 1 && rep_ld >= rep_dim, "need 1 <= rep_dim <= rep_ld");
  QMLR_REQUIRE(d >= 1 && d <= rep_dim && d + kPcaOversample <= kMaxL + kPcaOversample,
               "d must be in 1..min(rep_dim, 128)");
  QMLR_REQUIRE(d <= 128, "d must be <= 128");
  QMLR_REQUIRE(max_per_element >= 1, "max_per_element must be >= 1");
  QMLR_REQUIRE(work_bytes >= qmlr_pca_workspace_bytes(rep_ld, d), "workspace too small");
  cudaStream_t s = as_stream(stream);
  const int R = rep_ld;
  const int l = std::min(d + kPcaOversample, R);
  int32_t offs[9];
  QMLR_CUDA_TRY(cudaMemcpyAsync(offs, elem_offsets, sizeof(int32_t) * (n_el + 1), cudaMemcpyDeviceToHost, s));
  QMLR_CUDA_TRY(cudaStreamSynchronize(s));
  double* C = static_cast<double*>(work);
  double* Y = C + (long)R * R;
  double* Q = Y + (long)R * l;
  double* T = Q + (long)R * l;
  double* B = T + (long)R * l;
  double* W = B + (long)l * l;
  double* lam = W + (long)l * l;
  const size_t jsm = (size_t)(l + 1) * (l + 1) * 8;
  QMLR_CUDA_TRY(smem_attr_once((const void*)jacobi_kernel, (int)((kMaxL + 1) * (kMaxL + 1) * 8)));
  for (int e = 0; e < n_el; ++e) {
    float* Ue = U + (long)e * rep_dim * d;
    const int n = std::min(offs[e + 1] - offs[e], max_per_element);
    if (n <= 0) {
      QMLR_CUDA_TRY(cudaMemsetAsync(Ue, 0, sizeof(float) * rep_dim * d, s));
      continue;
    }
    dim3 gC((R + 31) / 32, (R + 31) / 32);
    syrk_f64_kernel<<<gC, 256, 0, s>>>(rep, rep_ld, R, perm + offs[e], n, C);
    QMLR_LAUNCH_CHECK();
    gaussian_kernel<<<(R * l + 255) / 256, 256, 0, s>>>(T, (long)R * l, 0x5eed0000ull + e);
    QMLR_LAUNCH_CHECK();
    dim3 gY((l + 31) / 32, (R + 31) / 32);
    dgemm_kernel<<<gY, 256, 0, s>>>(C, T, Y, R, l, R, 0);   // Y = C Omega
    QMLR_LAUNCH_CHECK();
    for (int it = 0; it < kPcaPowerIters; ++it) {
      mgs_kernel<<<1, 1024, 0, s>>>(Y, R, l);
      QMLR_LAUNCH_CHECK();
      dgemm_kernel<<<gY, 256, 0, s>>>(C, Y, T, R, l, R, 0);  // T = C Q
      QMLR_LAUNCH_CHECK();
      QMLR_CUDA_TRY(cudaMemcpyAsync(Y, T, sizeof(double) * R * l, cudaMemcpyDeviceToDevice, s));
    }
    mgs_kernel<<<1, 1024, 0, s>>>(Y, R, l);
    QMLR_LAUNCH_CHECK();
    QMLR_CUDA_TRY(cudaMemcpyAsync(Q, Y, sizeof(double) * R * l, cudaMemcpyDeviceToDevice, s));
    dgemm_kernel<<<gY, 256, 0, s>>>(C, Q, T, R, l, R, 0);     // T = C Q
    QMLR_LAUNCH_CHECK();
    dim3 gB((l + 31) / 32, (l + 31) / 32);
    dgemm_kernel<<<gB, 256, 0, s>>>(Q, T, B, l, l, R, 1);     // B = Q^T C Q
    QMLR_LAUNCH_CHECK();
    jacobi_kernel<<<1, 1024, jsm, s>>>(B, l, W, lam);
    QMLR_LAUNCH_CHECK();
    pca_finish_kernel<<<1, 1024, 0, s>>>(Q, W, lam, R, l, d, rep_dim, Ue);
    QMLR_LAUNCH_CHECK();
  }
  return QMLR_OK;
}
