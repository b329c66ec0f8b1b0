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

}  // namespace

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
