// Dense random Fourier features (RFF section of the paper: z(x) = sqrt(2/N_F)
// cos(W x + b) with W = G / sigma, G standard normal, b uniform on [0, 2 pi)),
// the feature map that the structured SORF transform replaces. This is the
// reference form of the paper's SORF-versus-RFF comparison, not the training
// path: a dense [N_F x d] W costs N_F d multiply-adds per atom where SORF
// costs T N_F log2 d additions.
//
// One CTA of 128 threads owns 128 consecutive features for a strided set of
// molecules. Its slice of G sits transposed in shared memory (row stride 129
// words: the transposing stores and the per-thread column reads are both free
// of bank conflicts); the CTA stages one atom's x at a time, and each thread
// forms its feature's dot product in FP32 (four partial sums, fixed order),
// scales by 1/sigma, adds b and takes cosf. Per-molecule sums run over the
// molecule's atoms in order (deterministic).
#include "common.cuh"

namespace qmlr {

namespace {

constexpr int kRffTile = 128;     // features per CTA
constexpr int kRffMaxD = 256;     // 256 x 129 x 4 B = 129 KB of G per CTA

__global__ void __launch_bounds__(kRffTile)
rff_kernel(const float* __restrict__ x, int d, const int32_t* __restrict__ mol_ptr, int n_mol,
           const float* __restrict__ G, const float* __restrict__ b, int n_features, float inv_sigma,
           float pref, int per_mol, float* __restrict__ out) {
  extern __shared__ float rsm[];
  float* gt = rsm;                               // [d][kRffTile + 1]
  float* xs = rsm + (size_t)d * (kRffTile + 1);  // [d]
  const int tid = threadIdx.x;
  const int f0 = blockIdx.x * kRffTile, f = f0 + tid;
  for (int idx = tid; idx < d * kRffTile; idx += kRffTile) {
    const int t = idx / d, k = idx % d;   // consecutive idx: consecutive k of one feature row
    gt[k * (kRffTile + 1) + t] = f0 + t < n_features ? G[(long)(f0 + t) * d + k] : 0.f;
  }
  const float bf = f < n_features ? b[f] : 0.f;
  for (int m = blockIdx.y; m < n_mol; m += gridDim.y) {
    const int a0 = mol_ptr[m], a1 = mol_ptr[m + 1];
    float zsum = 0.f;
    for (int a = a0; a < a1; ++a) {
      __syncthreads();   // the previous atom's x is no longer read (and G is staged)
      for (int k = tid; k < d; k += kRffTile) xs[k] = x[(long)a * d + k];
      __syncthreads();
      float p[4] = {0.f, 0.f, 0.f, 0.f};
      int k = 0;
      for (; k + 4 <= d; k += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) p[u] = fmaf(gt[(k + u) * (kRffTile + 1) + tid], xs[k + u], p[u]);
      }
      for (; k < d; ++k) p[0] = fmaf(gt[k * (kRffTile + 1) + tid], xs[k], p[0]);
      const float dot = (p[0] + p[1]) + (p[2] + p[3]);
      const float c = cosf(fmaf(dot, inv_sigma, bf));
      if (per_mol) {
        zsum += c;
      } else if (f < n_features) {
        out[(long)a * n_features + f] = pref * c;
      }
    }
    if (per_mol && f < n_features) out[(long)m * n_features + f] = pref * zsum;
  }
}

// ---------------------------------------------------------------------------
// Tensor-core form: u = x (G / sigma)^T is a dense contraction (K = d), run by
// the projection's tcgen05 grouped GEMM (3-way BF16 splits of both operands,
// FP32 accumulation in TMEM, one "element" and the identity row order) into a
// chunk of u rows; an epilogue then applies cos(u + b) and, per molecule, sums
// the chunk's atoms in order.

constexpr int kRffChunk = 65536;   // atoms per GEMM chunk (per-molecule mode)

__global__ void iota_kernel(int32_t* __restrict__ v, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = i;
}

__global__ void offsets_kernel(int32_t* __restrict__ offs, int n) {
  offs[0] = 0;
  offs[1] = n;
}

// out[a][f] = pref * cos(u[a][f] + b[f]) in place
__global__ void rff_cos_kernel(float* __restrict__ u, long n_atoms, int n_features, const float* __restrict__ b,
                               float pref) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_atoms * n_features) return;
  const int f = (int)(idx % n_features);
  u[idx] = pref * cosf(u[idx] + __ldg(b + f));
}

// Z[m][f] (+)= pref * sum over the atoms a of molecule m in [c0, c1), in order,
// of cos(u[a - c0][f] + b[f]); molecules from the first one that ends after c0.
__global__ void rff_mol_epilogue_kernel(const float* __restrict__ u, int n_features, const float* __restrict__ b,
                                        const int32_t* __restrict__ mol_ptr, int n_mol, int c0, int c1, float pref,
                                        float* __restrict__ Z) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  __shared__ int s_m0;
  if (threadIdx.x == 0) {
    int lo = 0, hi = n_mol;   // first m with mol_ptr[m + 1] > c0
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(mol_ptr + mid + 1) > c0) hi = mid; else lo = mid + 1;
    }
    s_m0 = lo;
  }
  __syncthreads();
  if (f >= n_features) return;
  const float bf = __ldg(b + f);
  for (int m = s_m0 + blockIdx.y; m < n_mol; m += gridDim.y) {
    const int m_lo = __ldg(mol_ptr + m), m_hi = __ldg(mol_ptr + m + 1);
    if (m_lo >= c1) break;
    const int a0 = max(m_lo, c0), a1 = min(m_hi, c1);
    if (a0 >= a1) continue;
    float sum = 0.f;
    for (int a = a0; a < a1; ++a) sum += cosf(u[(long)(a - c0) * n_features + f] + bf);
    Z[(long)m * n_features + f] += pref * sum;
  }
}

}  // namespace

size_t proj_tc_basis_bytes(int n_el, int K, int N);
int proj_tc_split_basis(const float* U, int n_el, int K, int N, long es, int ldu, bool trans, uint16_t* out,
                        cudaStream_t s, float scale);
int proj_tc_launch(const float* A, int lda, int K, int n_part, long a_part_stride, const uint16_t* basis, int N,
                   const int32_t* perm, const int32_t* elem_offsets, int n_atoms, int n_el, float* C, int ldc,
                   int zero_pad_to, cudaStream_t s);

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

extern "C" int64_t qmlr_rff_tc_workspace_bytes(int32_t n_atoms, int32_t d, int32_t n_features, int32_t mode) {
  if (n_atoms < 0 || d < 1 || n_features < 1) return 0;
  const int chunk = std::min(std::max(n_atoms, 1), kRffChunk);
  size_t b = align256(proj_tc_basis_bytes(1, d, n_features)) + align256((size_t)chunk * 4) + 256;
  if (mode == QMLR_SORF_PER_MOL) b += align256((size_t)chunk * n_features * 4);
  return (int64_t)b + 256;
}

extern "C" int qmlr_rff_tc(const float* x, int32_t d, const int32_t* mol_ptr, int32_t n_mol, int32_t n_atoms,
                           const float* G, const float* b, int32_t n_features, double sigma, int32_t mode,
                           float* out, void* work, int64_t work_bytes, void* stream) {
  QMLR_REQUIRE(mode == QMLR_SORF_PER_ATOM || mode == QMLR_SORF_PER_MOL,
               "qmlr_rff_tc supports the per-atom and per-molecule modes (got %d)", mode);
  QMLR_REQUIRE(d >= 1 && d <= 512, "d must be in 1..512 (got %d)", d);
  QMLR_REQUIRE(n_features >= 1 && n_mol >= 0 && n_atoms >= 0, "bad sizes");
  QMLR_REQUIRE(sigma > 0, "sigma must be positive");
  QMLR_REQUIRE(mol_ptr && G && b && out && (n_atoms == 0 || x), "NULL pointer argument");
  QMLR_REQUIRE(work && work_bytes >= qmlr_rff_tc_workspace_bytes(n_atoms, d, n_features, mode),
               "workspace too small (%lld < %lld bytes)", (long long)work_bytes,
               (long long)qmlr_rff_tc_workspace_bytes(n_atoms, d, n_features, mode));
  cudaStream_t s = as_stream(stream);
  const float pref = (float)std::sqrt(2.0 / n_features);
  if (mode == QMLR_SORF_PER_MOL) QMLR_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)n_mol * n_features, s));
  if (n_atoms == 0 || n_mol == 0) return QMLR_OK;
  const int chunk = std::min(n_atoms, kRffChunk);
  char* w = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(work) + 255) & ~uintptr_t(255));
  uint16_t* basis = reinterpret_cast<uint16_t*>(w);
  w += align256(proj_tc_basis_bytes(1, d, n_features));
  int32_t* perm = reinterpret_cast<int32_t*>(w);
  w += align256((size_t)chunk * 4);
  int32_t* offs = reinterpret_cast<int32_t*>(w);
  w += 256;
  float* u = reinterpret_cast<float*>(w);
  int rc = proj_tc_split_basis(G, 1, d, n_features, 0, d, true, basis, s, (float)(1.0 / sigma));
  if (rc) return rc;
  iota_kernel<<<(chunk + 255) / 256, 256, 0, s>>>(perm, chunk);
  QMLR_LAUNCH_CHECK();
  for (int c0 = 0; c0 < n_atoms; c0 += chunk) {
    const int nc = std::min(chunk, n_atoms - c0);
    offsets_kernel<<<1, 1, 0, s>>>(offs, nc);   // stream order keeps the previous chunk's value until it is used
    QMLR_LAUNCH_CHECK();
    if (mode == QMLR_SORF_PER_ATOM) {
      float* uo = out + (size_t)c0 * n_features;
      rc = proj_tc_launch(x + (size_t)c0 * d, d, d, 1, 0, basis, n_features, perm, offs, nc, 1, uo, n_features,
                          n_features, s);
      if (rc) return rc;
      const long tot = (long)nc * n_features;
      rff_cos_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(uo, nc, n_features, b, pref);
      QMLR_LAUNCH_CHECK();
    } else {
      rc = proj_tc_launch(x + (size_t)c0 * d, d, d, 1, 0, basis, n_features, perm, offs, nc, 1, u, n_features,
                          n_features, s);
      if (rc) return rc;
      dim3 grid((n_features + 255) / 256, std::min(nc + 1, 4096));
      rff_mol_epilogue_kernel<<<grid, 256, 0, s>>>(u, n_features, b, mol_ptr, n_mol, c0, c0 + nc, pref, out);
      QMLR_LAUNCH_CHECK();
    }
  }
  return QMLR_OK;
}

extern "C" int qmlr_rff(const float* x, int32_t d, const int32_t* mol_ptr, int32_t n_mol, int32_t n_atoms,
                        const float* G, const float* b, int32_t n_features, double sigma, int32_t mode,
                        float* out, void* stream) {
  QMLR_REQUIRE(mode == QMLR_SORF_PER_ATOM || mode == QMLR_SORF_PER_MOL,
               "qmlr_rff supports the per-atom and per-molecule modes (got %d)", mode);
  QMLR_REQUIRE(d >= 1 && d <= kRffMaxD, "d must be in 1..%d (got %d)", kRffMaxD, d);
  QMLR_REQUIRE(n_features >= 1 && n_mol >= 0 && n_atoms >= 0, "bad sizes");
  QMLR_REQUIRE(sigma > 0, "sigma must be positive");
  QMLR_REQUIRE(mol_ptr && G && b && out && (n_atoms == 0 || x), "NULL pointer argument");
  cudaStream_t s = as_stream(stream);
  if (n_mol == 0) return QMLR_OK;
  const size_t smem = ((size_t)d * (kRffTile + 1) + d) * sizeof(float);
  QMLR_CUDA_TRY(smem_attr_once((const void*)rff_kernel, (int)(((size_t)kRffMaxD * (kRffTile + 1) + kRffMaxD) * sizeof(float))));
  const int tiles = (n_features + kRffTile - 1) / kRffTile;
  // about four CTAs per SM over all feature tiles; each walks every chunks-th molecule
  const int chunks = std::max(1, std::min(n_mol, (4 * sm_count() + tiles - 1) / tiles));
  dim3 grid(tiles, chunks);
  rff_kernel<<<grid, kRffTile, smem, s>>>(x, d, mol_ptr, n_mol, G, b, n_features, (float)(1.0 / sigma),
                                          (float)std::sqrt(2.0 / n_features),
                                          mode == QMLR_SORF_PER_MOL ? 1 : 0, out);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

}  // namespace qmlr
