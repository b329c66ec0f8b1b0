// Split-BF16 tensor-core Gram G = Z^T Z on sm_103a (tcgen05 + TMA + TMEM).
//
// The normal equations' Z^T Z (RFF section of the paper; "the dominant
// term", built in FP32 with Kahan summation in the paper) is the one dense
// contraction of the method, so it runs on the 5th-generation tensor cores:
//   Z = H + L,  H = bf16(Z), L = bf16(Z - H)
//   G ~= H^T H + H^T L + L^T H      (FP32 accumulation in tensor memory)
// Operands are the transposed split matrices Zt_hi, Zt_lo [N_F][K] (rows of
// Z contiguous: K-major), loaded by TMA into 128-byte-swizzled shared memory.
//
// One CTA computes a 128 x 256 tile of G (rows i0.., columns j0..) for the
// upper triangle only: warp 0 lane 0 issues TMA copies into a 2-stage ring
// (full/empty mbarriers), warp 1 lane 0 issues 3 x 4 tcgen05.mma per 64-deep
// K block into one TMEM accumulator (256 columns), and all four warps drain
// TMEM with tcgen05.ld and write G[i][j] and its mirror G[j][i] for j >= i.
// Every mbarrier wait is bounded by a clock budget: on expiry the CTA records
// a device error, waits (bounded) for its own copies, frees TMEM and returns.
#include "common.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

namespace qmlr {

namespace tc {

constexpr int BM = 128;          // tile rows (features i)
constexpr int BN = 256;          // tile columns (features j)
constexpr int BK = 64;           // K block: 64 bf16 = 128 bytes (one swizzle row)
constexpr int STAGES = 2;
constexpr int A_BYTES = BM * BK * 2;        // 16 KB per split part
constexpr int B_BYTES = BN * BK * 2;        // 32 KB per split part
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;   // 96 KB
constexpr int TMEM_COLS = 256;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr long long WAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: true when the phase completed, false when the budget ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const volatile int* abort) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;            // start address
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                  // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                  // layout: 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D f32, A/B bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
      " [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__global__ void __launch_bounds__(128, 1)
gram_bf16x3_kernel(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
                   int n_features, int k_blocks, int tiles_j, float* __restrict__ G, int* err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accum = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* never_abort = abort + 1;   // a flag nobody sets: waits bounded by the clock only

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // tile (bi, bj): upper-triangle tiles of 128 x 256, enumerated row-major over bi
  int t = blockIdx.x, bi = 0;
  for (;;) {
    const int first = (bi * BM) / BN;          // first column tile reaching the diagonal
    const int cnt = tiles_j - first;
    if (t < cnt) {
      t += first;
      break;
    }
    t -= cnt;
    ++bi;
  }
  const int bj = t;
  const int i0 = bi * BM, j0 = bj * BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    *abort = 0;
    *never_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  int last_round[STAGES];  // producer: round of the last TMA batch issued per stage (-1 = none)
#pragma unroll
  for (int s = 0; s < STAGES; ++s) last_round[s] = -1;
  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    for (int kb = 0; kb < k_blocks; ++kb) {
      const int s = kb % STAGES;
      const uint32_t round = kb / STAGES;
      if (kb >= STAGES && !mbar_wait(&empty[s], (round - 1) & 1, abort)) {
        record_device_error(err, DEV_TIMEOUT);
        *abort = 1;
        break;
      }
      uint8_t* st = smem + s * STAGE_BYTES;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      const int k = kb * BK;
      tma_load_2d(st, &map_hi, &full[s], k, i0);
      tma_load_2d(st + A_BYTES, &map_lo, &full[s], k, i0);
      tma_load_2d(st + 2 * A_BYTES, &map_hi, &full[s], k, j0);
      tma_load_2d(st + 2 * A_BYTES + A_BYTES, &map_hi, &full[s], k, j0 + BM);
      tma_load_2d(st + 2 * A_BYTES + B_BYTES, &map_lo, &full[s], k, j0);
      tma_load_2d(st + 2 * A_BYTES + B_BYTES + A_BYTES, &map_lo, &full[s], k, j0 + BM);
      last_round[s] = (int)round;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    for (int kb = 0; kb < k_blocks; ++kb) {
      const int s = kb % STAGES;
      const uint32_t round = kb / STAGES;
      if (!mbar_wait(&full[s], round & 1, abort)) {
        record_device_error(err, DEV_TIMEOUT);
        *abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint8_t* st = smem + s * STAGE_BYTES;
      const uint8_t* a_hi = st;
      const uint8_t* a_lo = st + A_BYTES;
      const uint8_t* b_hi = st + 2 * A_BYTES;
      const uint8_t* b_lo = st + 2 * A_BYTES + B_BYTES;
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const int off = kk * 32;   // 16 bf16 along K inside the 128-byte swizzled row
        const uint32_t acc0 = (kb > 0 || kk > 0) ? 1u : 0u;
        mma_bf16(tmem, smem_desc(a_hi + off), smem_desc(b_hi + off), idesc, acc0);
        mma_bf16(tmem, smem_desc(a_hi + off), smem_desc(b_lo + off), idesc, 1u);
        mma_bf16(tmem, smem_desc(a_lo + off), smem_desc(b_hi + off), idesc, 1u);
      }
      mma_commit(&empty[s]);   // frees the stage once these MMAs have read it
    }
    mma_commit(accum);
  }
  __syncwarp();

  // ---------------- epilogue: TMEM -> registers -> G (upper triangle + mirror)
  // The MMA thread always commits `accum` last, so this wait also covers an
  // aborted main loop (it then only drains MMAs already issued).
  bool ok = mbar_wait(accum, 0, never_abort);
  if (!ok) {
    record_device_error(err, DEV_TIMEOUT);
    *abort = 1;
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();
  if (ok && !*abort) {
    const int row = i0 + warp * 32 + lane;                 // TMEM lane = tile row
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + c0, v);
      if (row < n_features) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int col = j0 + c0 + k;
          if (col >= row && col < n_features) {
            G[(long)row * n_features + col] = v[k];
            G[(long)col * n_features + row] = v[k];
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (*abort && warp == 0 && lane == 0) {
    // bounded wait for the TMA copies this CTA issued, before the CTA exits
    for (int s = 0; s < STAGES; ++s)
      if (last_round[s] >= 0) mbar_wait(&full[s], (uint32_t)last_round[s] & 1, never_abort);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

static int make_map(CUtensorMap* map, const void* base, long k_pad, int n_features) {
  auto fn = encode_fn();
  QMLR_REQUIRE(fn, "cuTensorMapEncodeTiled is not available");
  QMLR_REQUIRE((reinterpret_cast<uintptr_t>(base) & 15) == 0, "operand not 16-byte aligned");
  cuuint64_t dims[2] = {(cuuint64_t)k_pad, (cuuint64_t)n_features};
  cuuint64_t strides[1] = {(cuuint64_t)k_pad * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  QMLR_REQUIRE(r == CUDA_SUCCESS, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return QMLR_OK;
}

}  // namespace tc

int gram_bf16x3_tc(const uint16_t* zt_hi, const uint16_t* zt_lo, long k_pad, int n_features,
                   float* G, cudaStream_t s) {
  using namespace tc;
  if (k_pad == 0) {
    QMLR_CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(float) * (size_t)n_features * n_features, s));
    return QMLR_OK;
  }
  CUtensorMap mh, ml;
  int rc = make_map(&mh, zt_hi, k_pad, n_features);
  if (rc) return rc;
  rc = make_map(&ml, zt_lo, k_pad, n_features);
  if (rc) return rc;
  const int tiles_i = n_features / BM;
  const int tiles_j = (n_features + BN - 1) / BN;
  int n_tiles = 0;
  for (int bi = 0; bi < tiles_i; ++bi) n_tiles += tiles_j - (bi * BM) / BN;
  static bool attr = false;
  if (!attr) {
    QMLR_CUDA_TRY(cudaFuncSetAttribute(gram_bf16x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       SMEM_BYTES));
    attr = true;
  }
  gram_bf16x3_kernel<<<n_tiles, 128, SMEM_BYTES, s>>>(mh, ml, n_features, (int)(k_pad / BK), tiles_j, G,
                                                      device_error_ptr());
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

}  // namespace qmlr
