// Per-element projection rho_proj = rho^T U_e and its transpose (sm_103a).
//
// SORF section of the paper: each element has its own basis U_e (leading
// left singular vectors of that element's representations); the projection
// is one matrix product per element. Atoms are first grouped by element with
// a stable device counting sort (count / scan / scatter), then a grouped GEMM
// runs on the tensor cores over 128-atom tiles that each hold one element
// (project_tc.cu).
#include "common.cuh"

#include <mutex>

namespace qmlr {

constexpr int kGroupChunk = 1024;  // atoms per CTA of the counting sort
constexpr int kMaxEl = 8;

__global__ void group_count_kernel(const int32_t* __restrict__ elem, int n_atoms, int n_el,
                                   int* __restrict__ counts, int* err) {
  __shared__ int c[kMaxEl];
  if (threadIdx.x < kMaxEl) c[threadIdx.x] = 0;
  __syncthreads();
  const int i = blockIdx.x * kGroupChunk + threadIdx.x;
  if (i < n_atoms) {
    int e = __ldg(elem + i);
    if (e < 0 || e >= n_el) {
      record_device_error(err, DEV_BAD_ELEMENT);
      e = 0;
    }
    atomicAdd(&c[e], 1);  // integer counts: order-independent
  }
  __syncthreads();
  if (threadIdx.x < kMaxEl) counts[blockIdx.x * kMaxEl + threadIdx.x] = c[threadIdx.x];
}

// Exclusive scan over (element, chunk) in element-major order. One CTA.
__global__ void group_scan_kernel(const int* __restrict__ counts, int n_chunks, int n_el,
                                  int* __restrict__ offsets, int32_t* __restrict__ elem_offsets) {
  __shared__ int tot[kMaxEl];
  const int e = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (e < n_el) {
    // per element: warp-wide chunked scan over the chunks
    int run = 0;
    for (int base = 0; base < n_chunks; base += 32) {
      const int k = base + lane;
      int v = k < n_chunks ? counts[k * kMaxEl + e] : 0;
      int incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      if (k < n_chunks) offsets[k * kMaxEl + e] = run + incl - v;
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) tot[e] = run;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int k = 0; k < n_el; ++k) {
      elem_offsets[k] = acc;
      acc += tot[k];
    }
    elem_offsets[n_el] = acc;
  }
  __syncthreads();
  // shift per-chunk offsets by the element start
  for (int idx = threadIdx.x; idx < n_chunks * n_el; idx += blockDim.x) {
    const int k = idx / n_el, ee = idx % n_el;
    offsets[k * kMaxEl + ee] += elem_offsets[ee];
  }
}

__global__ void group_scatter_kernel(const int32_t* __restrict__ elem, int n_atoms, int n_el,
                                     const int* __restrict__ offsets, int32_t* __restrict__ perm) {
  __shared__ int wtot[kGroupChunk / 32][kMaxEl];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kGroupChunk + threadIdx.x;
  int e = -1;
  if (i < n_atoms) {
    e = __ldg(elem + i);
    if (e < 0 || e >= n_el) e = 0;
  }
  int rank = 0;
  for (int k = 0; k < n_el; ++k) {
    const unsigned mask = __ballot_sync(0xffffffffu, e == k);
    if (e == k) rank = __popc(mask & ((1u << lane) - 1u));
    if (lane == 0) wtot[warp][k] = __popc(mask);
  }
  __syncthreads();
  if (e >= 0) {
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wtot[w][e];
    perm[offsets[blockIdx.x * kMaxEl + e] + before + rank] = i;
  }
}

// ---------------------------------------------------------------------------
// The grouped projection itself runs on the tensor cores (project_tc.cu).
size_t proj_tc_basis_bytes(int n_el, int K, int N);
int proj_tc_split_basis(const float* U, int n_el, int K, int N, long es, int ldu, bool trans, uint16_t* out,
                        cudaStream_t s, float scale = 1.0f);
int proj_tc_launch(const float* A, int lda, int K, int n_part, long a_part_stride, const uint16_t* basis, int N,
                   const int32_t* perm, const int32_t* elem_offsets, int n_atoms, int n_el, float* C, int ldc,
                   int zero_pad_to, cudaStream_t s);

}  // namespace qmlr

using namespace qmlr;

extern "C" int64_t qmlr_group_workspace_bytes(int32_t n_atoms) {
  const int64_t chunks = (n_atoms + kGroupChunk - 1) / kGroupChunk;
  return 2 * chunks * kMaxEl * (int64_t)sizeof(int) + 256;
}

extern "C" int qmlr_group_by_element(const int32_t* elem, int32_t n_atoms, int32_t n_el,
                                     int32_t* perm, int32_t* elem_offsets, void* work,
                                     int64_t work_bytes, void* stream) {
  QMLR_REQUIRE(n_el >= 1 && n_el <= kMaxEl, "n_el must be in 1..8 (got %d)", n_el);
  QMLR_REQUIRE(n_atoms >= 0, "n_atoms must be >= 0");
  QMLR_REQUIRE(elem_offsets, "elem_offsets is NULL");
  QMLR_REQUIRE(n_atoms == 0 || (elem && perm), "elem/perm are NULL");
  QMLR_REQUIRE(work && work_bytes >= qmlr_group_workspace_bytes(n_atoms),
               "workspace too small (%lld < %lld bytes)", (long long)work_bytes,
               (long long)qmlr_group_workspace_bytes(n_atoms));
  cudaStream_t s = as_stream(stream);
  const int chunks = (n_atoms + kGroupChunk - 1) / kGroupChunk;
  int* counts = static_cast<int*>(work);
  int* offsets = counts + (size_t)chunks * kMaxEl;
  if (chunks > 0) {
    group_count_kernel<<<chunks, kGroupChunk, 0, s>>>(elem, n_atoms, n_el, counts, device_error_ptr());
    QMLR_LAUNCH_CHECK();
  }
  group_scan_kernel<<<1, 256, 0, s>>>(counts, chunks, n_el, offsets, elem_offsets);
  QMLR_LAUNCH_CHECK();
  if (chunks > 0) {
    group_scatter_kernel<<<chunks, kGroupChunk, 0, s>>>(elem, n_atoms, n_el, offsets, perm);
    QMLR_LAUNCH_CHECK();
  }
  return QMLR_OK;
}

extern "C" int64_t qmlr_project_workspace_bytes(int32_t n_el, int32_t rep_dim, int32_t d) {
  if (n_el < 1 || n_el > kMaxEl || rep_dim < 1 || d < 1) return 0;
  // the split basis of either direction (the same element count) plus alignment slack
  return (int64_t)std::max(proj_tc_basis_bytes(n_el, rep_dim, d), proj_tc_basis_bytes(n_el, d, rep_dim)) + 256;
}

static uint16_t* aligned_basis(void* work) {
  return reinterpret_cast<uint16_t*>((reinterpret_cast<uintptr_t>(work) + 255) & ~uintptr_t(255));
}

extern "C" int qmlr_project(const float* rep, int32_t rep_ld, int32_t rep_dim, const int32_t* perm,
                            const int32_t* elem_offsets, int32_t n_atoms, int32_t n_el,
                            const float* U, int32_t d, float* x, void* work, int64_t work_bytes,
                            void* stream) {
  QMLR_REQUIRE(n_el >= 1 && n_el <= kMaxEl, "n_el must be in 1..8");
  QMLR_REQUIRE(is_pow2(d) && d >= 16 && d <= 512, "d must be a power of two in 16..512 (got %d)", d);
  QMLR_REQUIRE(rep_dim >= 1 && rep_ld >= rep_dim, "need 1 <= rep_dim <= rep_ld");
  QMLR_REQUIRE(n_atoms >= 0, "n_atoms must be >= 0");
  if (n_atoms == 0) return QMLR_OK;
  QMLR_REQUIRE(rep && perm && elem_offsets && U && x, "NULL pointer argument");
  QMLR_REQUIRE(work && work_bytes >= qmlr_project_workspace_bytes(n_el, rep_dim, d),
               "workspace too small (%lld < %lld bytes)", (long long)work_bytes,
               (long long)qmlr_project_workspace_bytes(n_el, rep_dim, d));
  // the basis is split into the caller's workspace on every call (a model keeps its split basis)
  cudaStream_t s = as_stream(stream);
  uint16_t* basis = aligned_basis(work);
  int rc = proj_tc_split_basis(U, n_el, rep_dim, d, (long)rep_dim * d, d, false, basis, s);
  if (rc == QMLR_OK)
    rc = proj_tc_launch(rep, rep_ld, rep_dim, 1, 0, basis, d, perm, elem_offsets, n_atoms, n_el, x, d, d, s);
  return rc;
}

extern "C" int qmlr_project_t(const float* gx, int32_t n_part, const int32_t* perm,
                              const int32_t* elem_offsets, int32_t n_atoms, int32_t n_el,
                              const float* U, int32_t d, int32_t rep_dim, float* grad_rep,
                              int32_t rep_ld, void* work, int64_t work_bytes, void* stream) {
  QMLR_REQUIRE(n_el >= 1 && n_el <= kMaxEl, "n_el must be in 1..8");
  QMLR_REQUIRE(is_pow2(d) && d >= 16 && d <= 512, "d must be a power of two in 16..512 (got %d)", d);
  QMLR_REQUIRE(rep_dim >= 1 && rep_ld >= rep_dim, "need 1 <= rep_dim <= rep_ld");
  QMLR_REQUIRE(n_part >= 1, "n_part must be >= 1");
  if (n_atoms == 0) return QMLR_OK;
  QMLR_REQUIRE(gx && perm && elem_offsets && U && grad_rep, "NULL pointer argument");
  QMLR_REQUIRE(work && work_bytes >= qmlr_project_workspace_bytes(n_el, rep_dim, d),
               "workspace too small (%lld < %lld bytes)", (long long)work_bytes,
               (long long)qmlr_project_workspace_bytes(n_el, rep_dim, d));
  cudaStream_t s = as_stream(stream);
  uint16_t* basis = aligned_basis(work);
  int rc = proj_tc_split_basis(U, n_el, d, rep_dim, (long)rep_dim * d, d, true, basis, s);
  if (rc == QMLR_OK)
    rc = proj_tc_launch(gx, d, d, n_part, (long)n_atoms * d, basis, rep_dim, perm, elem_offsets, n_atoms, n_el,
                        grad_rep, rep_ld, rep_ld, s);
  return rc;
}

// ---------------------------------------------------------------------------
// Element grouping without any allocation (same kernels, fixed scratch).
//
// Some callers cannot allocate device memory at the moment they need the
// grouping: a host framework that hands out all device memory from its own
// pool, or a latency-critical service that must not block on the allocator. For them the
// counting sort's per-chunk counts and offsets live in a file-scope device
// array sized for QMLR_GROUP_NOALLOC_MAX_ATOMS atoms; every device that loads
// the library holds it (256 KiB) until the process exits.
namespace qmlr {

constexpr int kNoAllocChunks = QMLR_GROUP_NOALLOC_MAX_ATOMS / kGroupChunk;
static __device__ __align__(256) int g_group_scratch[2 * kNoAllocChunks * kMaxEl];

// Device address of g_group_scratch on the current device. In host code the
// symbol is only a host-side stand-in, so the address is looked up once per
// device (with that device current) and cached.
static int* group_scratch_address() {
  static std::mutex mu;
  static int* addr[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_group_scratch) != cudaSuccess) return nullptr;
    addr[dev] = static_cast<int*>(p);
  }
  return addr[dev];
}

}  // namespace qmlr

extern "C" int qmlr_group_by_element_noalloc(const int32_t* elem, int32_t n_atoms, int32_t n_el,
                                             int32_t* perm, int32_t* elem_offsets, void* stream) {
  QMLR_REQUIRE(n_el >= 1 && n_el <= kMaxEl, "n_el must be in 1..8 (got %d)", n_el);
  QMLR_REQUIRE(n_atoms >= 0, "n_atoms must be >= 0");
  QMLR_REQUIRE(n_atoms <= QMLR_GROUP_NOALLOC_MAX_ATOMS,
               "n_atoms = %d exceeds the fixed scratch of the no-allocation grouping "
               "(QMLR_GROUP_NOALLOC_MAX_ATOMS = %d); use qmlr_group_by_element with a workspace",
               n_atoms, QMLR_GROUP_NOALLOC_MAX_ATOMS);
  QMLR_REQUIRE(elem_offsets, "elem_offsets is NULL");
  QMLR_REQUIRE(n_atoms == 0 || (elem && perm), "elem/perm are NULL");
  int* scratch = group_scratch_address();
  if (!scratch) {
    set_error("cudaGetSymbolAddress of the grouping scratch failed on the current device");
    return QMLR_ECUDA;
  }
  cudaStream_t s = as_stream(stream);
  const int chunks = (n_atoms + kGroupChunk - 1) / kGroupChunk;
  int* counts = scratch;
  int* offsets = scratch + (size_t)kNoAllocChunks * kMaxEl;
  // counts and offsets of every chunk used are written by the kernels below
  // before they are read, so nothing left over from an earlier call is used.
  if (chunks > 0) {
    group_count_kernel<<<chunks, kGroupChunk, 0, s>>>(elem, n_atoms, n_el, counts, device_error_ptr());
    QMLR_LAUNCH_CHECK();
  }
  group_scan_kernel<<<1, 256, 0, s>>>(counts, chunks, n_el, offsets, elem_offsets);
  QMLR_LAUNCH_CHECK();
  if (chunks > 0) {
    group_scatter_kernel<<<chunks, kGroupChunk, 0, s>>>(elem, n_atoms, n_el, offsets, perm);
    QMLR_LAUNCH_CHECK();
  }
  return QMLR_OK;
}
