// Per-element PCA projection on the tensor cores (sm_103a).
//
// SORF section of the paper: each atomic representation is projected onto the
// leading principal directions of its element, x_I = U_{e(I)}^T rho_I (and, for
// the forces, the transposed map g_rho = U_e g_x). With the atoms grouped by
// element this is a grouped GEMM C[row][n] = sum_k A[row][k] B_e[k][n] over the
// rows of each element; it runs here as tcgen05.mma (BF16 in, FP32 in TMEM)
// on 3-way BF16 splits of both operands (products to ~2^-24 relative, the
// accuracy of an FP32 GEMM):
//   * A (representations or gradients, FP32, rows gathered through the
//     element permutation, n_part slices summed) is split by the CTA's own
//     producer warps and written into 128-byte-swizzled shared memory;
//   * B_e (the element's basis) is split once (per model, or per call of the
//     public entry points) into a K-major bf16 buffer [e][3][N_pad][K_pad]
//     that TMA loads.
// One CTA computes a 128-row x 128-column tile of one element; two TMEM
// accumulators take the even and odd 64-deep K blocks (so that each sees half
// of the truncating accumulator adds), and the producer warps drain them.
#include "tcgen05.cuh"

#include <cuda_bf16.h>

namespace qmlr {
namespace tcp {

using namespace tc;

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;   // 16 KB each per split part
constexpr int STAGE_BYTES = 3 * A_BYTES + 3 * B_BYTES;         // 96 KB
constexpr int NST = 2;
constexpr int SMEM_BYTES = NST * STAGE_BYTES + 1024 + 1024;   // stages, alignment, barriers + rows
constexpr int kProd = 8;                                        // producer / drain warps
constexpr int kThreads = 32 * (kProd + 2);
__device__ __constant__ int kPA[6] = {0, 0, 1, 0, 2, 1};
__device__ __constant__ int kPB[6] = {0, 1, 0, 2, 0, 1};

struct Args {
  const float* A;
  int lda, K, n_part;
  long a_part_stride;
  int N, N_pad, K_pad;
  const int32_t* perm;
  const int32_t* elem_offsets;
  int n_el;
  float* C;
  int ldc, zero_pad_to;
  int* err;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
         ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

// Split 8 consecutive values into three BF16 parts (v = p0 + p1 + p2 to ~2^-24)
// and store chunk c of line r of each part (128-byte swizzle).
__device__ __forceinline__ void store_split_chunk(uint8_t* sp, int r, int c, const float (&v)[8]) {
  float r1[8], r2[8];
  uint32_t w0[4], w1[4], w2[4];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float h0 = __bfloat162float(__float2bfloat16_rn(v[j]));
    r1[j] = __fsub_rn(v[j], h0);
    const float h1 = __bfloat162float(__float2bfloat16_rn(r1[j]));
    r2[j] = __fsub_rn(r1[j], h1);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    w0[j] = pack_bf16(v[2 * j], v[2 * j + 1]);
    w1[j] = pack_bf16(r1[2 * j], r1[2 * j + 1]);
    w2[j] = pack_bf16(r2[2 * j], r2[2 * j + 1]);
  }
  const uint32_t off = (uint32_t)r * 128u + (uint32_t)((c ^ (r & 7)) * 16);
  const uint32_t base = smem_u32(sp) + off;
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(base), "r"(w0[0]), "r"(w0[1]), "r"(w0[2]),
               "r"(w0[3]) : "memory");
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(base + A_BYTES), "r"(w1[0]), "r"(w1[1]),
               "r"(w1[2]), "r"(w1[3]) : "memory");
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(base + 2 * A_BYTES), "r"(w2[0]), "r"(w2[1]),
               "r"(w2[2]), "r"(w2[3]) : "memory");
}

// 32 values of row `row` starting at column k (zero past K, for row < 0, and summed over slices)
__device__ __forceinline__ void load_row32(const Args& a, int row, int k, bool vec, float (&v)[32]) {
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = 0.f;
  if (row < 0) return;
  for (int p = 0; p < a.n_part; ++p) {
    const float* src = a.A + (long)p * a.a_part_stride + (long)row * a.lda + k;
    if (vec && k + 32 <= a.K) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 f = __ldg(reinterpret_cast<const float4*>(src) + q);
        v[4 * q] += f.x;
        v[4 * q + 1] += f.y;
        v[4 * q + 2] += f.z;
        v[4 * q + 3] += f.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (k + j < a.K) v[j] += __ldg(src + j);
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1)
proj_tc_kernel(const __grid_constant__ CUtensorMap bmap, Args a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NST * STAGE_BYTES);
  uint64_t* empty = full + NST;
  uint64_t* accf = empty + NST;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accf + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* never_abort = abort + 1;
  int* rows = const_cast<int*>(reinterpret_cast<volatile int*>(never_abort + 1));   // [BM]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  // (element, row tile) of this CTA
  int e = -1, tile = blockIdx.x, start = 0, count = 0;
  for (int k = 0; k < a.n_el; ++k) {
    const int s = a.elem_offsets[k], cnt = a.elem_offsets[k + 1] - s;
    const int nt = (cnt + BM - 1) / BM;
    if (tile < nt) {
      e = k;
      start = s + tile * BM;
      count = min(BM, cnt - tile * BM);
      break;
    }
    tile -= nt;
  }
  if (e < 0) return;   // whole CTA, before any barrier or allocation
  const int n0 = blockIdx.y * BN;
  const int k_blocks = a.K_pad / BK;

  if (tid < BM) rows[tid] = tid < count ? a.perm[start + tid] : -1;
  if (tid == 0) {
    for (int q = 0; q < NST; ++q) {
      mbar_init(&full[q], 32 * kProd + 1);   // producers + the TMA thread's expect_tx arrive
      mbar_init(&empty[q], 1);
    }
    mbar_init(accf, 1);
    *abort = 0;
    *never_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  int last_round[NST];
#pragma unroll
  for (int q = 0; q < NST; ++q) last_round[q] = -1;

  if (warp < kProd) {
    // ---------------- producers: thread (r, h) splits columns [32h, 32h+32) of row r
    const int r = tid & (BM - 1), h = tid >> 7;
    const int row = rows[r];
    const bool vec = ((a.lda & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.A) & 15) == 0) &&
                     ((a.a_part_stride & 3) == 0);
    float cur[32];
    load_row32(a, row, h * 32, vec, cur);
    bool ok = true;
    for (int kb = 0; kb < k_blocks && ok; ++kb) {
      const int st = kb % NST;
      const uint32_t round = kb / NST;
      float nxt[32];
      if (kb + 1 < k_blocks) load_row32(a, row, (kb + 1) * BK + h * 32, vec, nxt);
      if (kb >= NST && !mbar_wait(&empty[st], (round - 1) & 1, abort)) {
        record_device_error(a.err, DEV_TIMEOUT);
        *abort = 1;
        ok = false;
        break;
      }
      uint8_t* sp = smem + st * STAGE_BYTES;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float v8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v8[j] = cur[8 * c + j];
        store_split_chunk(sp, r, h * 4 + c, v8);
      }
      fence_proxy_async_smem();
      mbar_arrive(&full[st]);
      if (kb + 1 < k_blocks) {
#pragma unroll
        for (int j = 0; j < 32; ++j) cur[j] = nxt[j];
      }
    }
    // ---------------- drain: rows quarter*32.., columns half*64..
    const int quarter = warp & 3, half = warp >> 2;
    const bool vec_out = ((a.ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.C) & 15) == 0);
    const bool done = ok && mbar_wait(accf, 0, abort);
    if (__any_sync(0xffffffffu, !done)) {
      if (lane == 0) {
        record_device_error(a.err, DEV_TIMEOUT);
        *abort = 1;
      }
    } else {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int rr = quarter * 32 + lane;
      const int orow = rows[rr];
      const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        float v0[16], v1[16];
        const int col = half * 64 + c4 * 16;
        tmem_ld16(tmem + lane_base + col, v0);
        tmem_ld16(tmem + lane_base + BN + col, v1);
        if (orow >= 0) {
          float* dst = a.C + (long)orow * a.ldc + n0 + col;
          if (vec_out && n0 + col + 16 <= a.N) {
            float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
            for (int j = 0; j < 4; ++j)
              d4[j] = make_float4(v0[4 * j] + v1[4 * j], v0[4 * j + 1] + v1[4 * j + 1], v0[4 * j + 2] + v1[4 * j + 2],
                                  v0[4 * j + 3] + v1[4 * j + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int n = n0 + col + j;
              if (n < a.N) dst[j] = v0[j] + v1[j];
              else if (n < a.zero_pad_to) dst[j] = 0.f;
            }
          }
        }
      }
    }
  } else if (warp == kProd && lane == 0) {
    // ---------------- TMA: B_e parts (rows (e*3+q)*N_pad + n0)
    for (int kb = 0; kb < k_blocks; ++kb) {
      const int st = kb % NST;
      const uint32_t round = kb / NST;
      if (kb >= NST && !mbar_wait(&empty[st], (round - 1) & 1, abort)) {
        record_device_error(a.err, DEV_TIMEOUT);
        *abort = 1;
        break;
      }
      uint8_t* sp = smem + st * STAGE_BYTES + 3 * A_BYTES;
      mbar_expect_tx(&full[st], 3 * B_BYTES);
#pragma unroll
      for (int q = 0; q < 3; ++q) tma_load_2d(sp + q * B_BYTES, &bmap, &full[st], kb * BK, (e * 3 + q) * a.N_pad + n0);
      last_round[st] = (int)round;
    }
  } else if (warp == kProd + 1 && lane == 0) {
    // ---------------- MMA: even K blocks into accumulator 0, odd into accumulator 1
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    for (int kb = 0; kb < k_blocks; ++kb) {
      const int st = kb % NST;
      const uint32_t round = kb / NST;
      if (!mbar_wait(&full[st], round & 1, abort)) {
        record_device_error(a.err, DEV_TIMEOUT);
        *abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint8_t* sp = smem + st * STAGE_BYTES;
      const uint32_t d = tmem + (kb & 1) * BN;
#pragma unroll
      for (int q = 5; q >= 0; --q) {   // smallest split products first
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint8_t* pa = sp + kPA[q] * A_BYTES + kk * 32;
          const uint8_t* pb = sp + 3 * A_BYTES + kPB[q] * B_BYTES + kk * 32;
          mma_bf16(d, smem_desc(pa), smem_desc(pb), idesc, (kb >= 2 || q < 5 || kk > 0) ? 1u : 0u);
        }
      }
      mma_commit(&empty[st]);
    }
    mma_commit(accf);   // (K is padded to at least two blocks, so both accumulators are written)
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (*abort) {
    if (warp == kProd && lane == 0)
      for (int q = 0; q < NST; ++q)
        if (last_round[q] >= 0) mbar_wait(&full[q], (uint32_t)last_round[q] & 1, never_abort);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN));
  }
}

// Short-K form (K_pad <= 128, the transposed projection g_rho = U_e g_x): the
// CTA splits its 128 gathered rows once into shared memory (two K blocks stay
// resident) and walks all output column tiles, streaming the basis tiles through
// a 2-stage TMA ring; two TMEM accumulators alternate between column tiles so
// that the drain of one overlaps the products of the next.
constexpr int RK = 2;                                         // resident K blocks
constexpr int R_A_BYTES = RK * 3 * A_BYTES;                   // 96 KB
constexpr int R_STAGE = 3 * B_BYTES;                          // 48 KB per K block of a column tile
constexpr int R_NST = 2;
constexpr int R_SMEM_BYTES = R_A_BYTES + R_NST * R_STAGE + 1024 + 1024;

__global__ void __launch_bounds__(kThreads, 1)
proj_tc_resident_kernel(const __grid_constant__ CUtensorMap bmap, Args a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* As = smem;                                          // [RK][3][A_BYTES]
  uint8_t* Bs = smem + R_A_BYTES;                              // [R_NST][3][B_BYTES]
  uint64_t* full = reinterpret_cast<uint64_t*>(Bs + R_NST * R_STAGE);
  uint64_t* empty = full + R_NST;
  uint64_t* accf = empty + R_NST;      // [2]
  uint64_t* acce = accf + 2;           // [2]
  uint64_t* aready = acce + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(aready + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* never_abort = abort + 1;
  int* rows = const_cast<int*>(reinterpret_cast<volatile int*>(never_abort + 1));   // [BM]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  int e = -1, tile = blockIdx.x, start = 0, count = 0;
  for (int k = 0; k < a.n_el; ++k) {
    const int s0 = a.elem_offsets[k], cnt = a.elem_offsets[k + 1] - s0;
    const int nt = (cnt + BM - 1) / BM;
    if (tile < nt) {
      e = k;
      start = s0 + tile * BM;
      count = min(BM, cnt - tile * BM);
      break;
    }
    tile -= nt;
  }
  if (e < 0) return;   // whole CTA, before any barrier or allocation
  const int k_blocks = a.K_pad / BK;                           // 1 or 2 (host guarantees <= RK)
  const int n_tiles = (max(a.N, a.zero_pad_to) + BN - 1) / BN;
  const int steps = n_tiles * k_blocks;

  if (tid < BM) rows[tid] = tid < count ? a.perm[start + tid] : -1;
  if (tid == 0) {
    for (int q = 0; q < R_NST; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&accf[q], 1);
      mbar_init(&acce[q], kProd);
    }
    mbar_init(aready, 32 * kProd);
    *abort = 0;
    *never_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  int last_round[R_NST];
#pragma unroll
  for (int q = 0; q < R_NST; ++q) last_round[q] = -1;

  if (warp < kProd) {
    // ---------------- producers: the rows' K blocks, split once
    const int r = tid & (BM - 1), h = tid >> 7;
    const int row = rows[r];
    const bool vec = ((a.lda & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.A) & 15) == 0) &&
                     ((a.a_part_stride & 3) == 0);
    for (int kb = 0; kb < k_blocks; ++kb) {
      float cur[32];
      load_row32(a, row, kb * BK + h * 32, vec, cur);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float v8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v8[j] = cur[8 * c + j];
        store_split_chunk(As + kb * 3 * A_BYTES, r, h * 4 + c, v8);
      }
    }
    fence_proxy_async_smem();
    mbar_arrive(aready);
    // ---------------- drain: one column tile per accumulator use
    const int quarter = warp & 3, half = warp >> 2;
    const bool vec_out = ((a.ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.C) & 15) == 0);
    const int rr = quarter * 32 + lane;
    const int orow = rows[rr];
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    for (int nt = 0; nt < n_tiles; ++nt) {
      const int buf = nt & 1;
      const uint32_t use = nt >> 1;
      const bool ok = mbar_wait(&accf[buf], use & 1, abort);
      if (__any_sync(0xffffffffu, !ok)) {
        if (lane == 0) {
          record_device_error(a.err, DEV_TIMEOUT);
          *abort = 1;
        }
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int n0 = nt * BN;
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        float v[16];
        const int col = half * 64 + c4 * 16;
        tmem_ld16(tmem + lane_base + buf * BN + col, v);
        if (orow >= 0) {
          float* dst = a.C + (long)orow * a.ldc + n0 + col;
          if (vec_out && n0 + col + 16 <= a.N) {
            // whole chunk inside the output: four 16-byte stores (a scalar store
            // per element made one L2 write request per element)
            float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
            for (int j = 0; j < 4; ++j) d4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int n = n0 + col + j;
              if (n < a.N) dst[j] = v[j];
              else if (n < a.zero_pad_to) dst[j] = 0.f;
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[buf]);
    }
  } else if (warp == kProd && lane == 0) {
    // ---------------- TMA: basis tiles (column tile nt, K block kb) through the ring
    for (int i = 0; i < steps; ++i) {
      const int nt = i / k_blocks, kb = i % k_blocks;
      const int st = i % R_NST;
      const uint32_t round = i / R_NST;
      if (i >= R_NST && !mbar_wait(&empty[st], (round - 1) & 1, abort)) {
        record_device_error(a.err, DEV_TIMEOUT);
        *abort = 1;
        break;
      }
      uint8_t* sp = Bs + st * R_STAGE;
      mbar_expect_tx(&full[st], R_STAGE);
#pragma unroll
      for (int q = 0; q < 3; ++q)
        tma_load_2d(sp + q * B_BYTES, &bmap, &full[st], kb * BK, (e * 3 + q) * a.N_pad + nt * BN);
      last_round[st] = (int)round;
    }
  } else if (warp == kProd + 1 && lane == 0) {
    // ---------------- MMA
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    bool ok = mbar_wait(aready, 0, abort);
    for (int i = 0; i < steps && ok; ++i) {
      const int nt = i / k_blocks, kb = i % k_blocks;
      const int st = i % R_NST;
      const uint32_t round = i / R_NST;
      const int buf = nt & 1;
      const uint32_t use = nt >> 1;
      if (!mbar_wait(&full[st], round & 1, abort) ||
          (kb == 0 && use > 0 && !mbar_wait(&acce[buf], (use - 1) & 1, abort))) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint8_t* ap = As + kb * 3 * A_BYTES;
      const uint8_t* bp = Bs + st * R_STAGE;
      const uint32_t d = tmem + buf * BN;
#pragma unroll
      for (int q = 5; q >= 0; --q) {   // smallest split products first
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk)
          mma_bf16(d, smem_desc(ap + kPA[q] * A_BYTES + kk * 32), smem_desc(bp + kPB[q] * B_BYTES + kk * 32), idesc,
                   (kb > 0 || q < 5 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&empty[st]);
      if (kb == k_blocks - 1) mma_commit(&accf[buf]);
    }
    if (!ok) {
      record_device_error(a.err, DEV_TIMEOUT);
      *abort = 1;
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (*abort) {
    if (warp == kProd && lane == 0)
      for (int q = 0; q < R_NST; ++q)
        if (last_round[q] >= 0) mbar_wait(&full[q], (uint32_t)last_round[q] & 1, never_abort);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN));
  }
}

// out[(e*3 + q)*N_pad + n][k] = part q of B_e[k][n] (zero outside K x N), with
// B_e[k][n] = U[e*es + k*ldu + n] (trans = 0) or U[e*es + n*ldu + k] (trans = 1).
__global__ void split_basis_kernel(const float* __restrict__ U, int n_el, int K, int N, long es, int ldu,
                                   int trans, float scale, int K_pad, int N_pad, __nv_bfloat16* __restrict__ out) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long total = (long)n_el * N_pad * K_pad;
  if (idx >= total) return;
  const int k = (int)(idx % K_pad);
  const int n = (int)((idx / K_pad) % N_pad);
  const int e = (int)(idx / ((long)K_pad * N_pad));
  float v = 0.f;
  if (k < K && n < N) v = scale * (trans ? U[e * es + (long)n * ldu + k] : U[e * es + (long)k * ldu + n]);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    out[((long)(e * 3 + q) * N_pad + n) * K_pad + k] = h;
    v = __fsub_rn(v, __bfloat162float(h));
  }
}

}  // namespace tcp

// K_pad, N_pad and bytes of the split basis for a K x N per-element map.
void proj_tc_dims(int K, int N, int* K_pad, int* N_pad) {
  *K_pad = std::max(2, (K + tcp::BK - 1) / tcp::BK) * tcp::BK;   // at least two K blocks
  *N_pad = (N + tcp::BN - 1) / tcp::BN * tcp::BN;
}

size_t proj_tc_basis_bytes(int n_el, int K, int N) {
  int kp, np;
  proj_tc_dims(K, N, &kp, &np);
  return (size_t)n_el * 3 * np * kp * 2;
}

int proj_tc_split_basis(const float* U, int n_el, int K, int N, long es, int ldu, bool trans, uint16_t* out,
                        cudaStream_t s, float scale) {
  int kp, np;
  proj_tc_dims(K, N, &kp, &np);
  const long total = (long)n_el * np * kp;
  tcp::split_basis_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
      U, n_el, K, N, es, ldu, trans ? 1 : 0, scale, kp, np, reinterpret_cast<__nv_bfloat16*>(out));
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

// C[row][n] = sum_k (sum_p A[p][row][k]) B_e[k][n] for the rows of each element.
int proj_tc_launch(const float* A, int lda, int K, int n_part, long a_part_stride, const uint16_t* basis, int N,
                   const int32_t* perm, const int32_t* elem_offsets, int n_atoms, int n_el, float* C, int ldc,
                   int zero_pad_to, cudaStream_t s) {
  using namespace tcp;
  int kp, np;
  proj_tc_dims(K, N, &kp, &np);
  CUtensorMap map;
  int rc = tc::make_map(&map, basis, kp, (long)n_el * 3 * np);
  if (rc) return rc;
  QMLR_CUDA_TRY(smem_attr_once((const void*)proj_tc_kernel, SMEM_BYTES));
  Args a{A, lda, K, n_part, a_part_stride, N, np, kp, perm, elem_offsets, n_el, C, ldc, zero_pad_to,
         device_error_ptr()};
  const int n_tiles = (std::max(N, zero_pad_to) + BN - 1) / BN;
  if (kp <= RK * BK && n_tiles > 1) {
    // short K, several column tiles: the CTA keeps its split rows and walks the tiles
    QMLR_CUDA_TRY(smem_attr_once((const void*)proj_tc_resident_kernel, R_SMEM_BYTES));
    proj_tc_resident_kernel<<<(n_atoms + BM - 1) / BM + n_el, kThreads, R_SMEM_BYTES, s>>>(map, a);
    QMLR_LAUNCH_CHECK();
    return QMLR_OK;
  }
  dim3 grid((n_atoms + BM - 1) / BM + n_el, n_tiles);
  proj_tc_kernel<<<grid, kThreads, SMEM_BYTES, s>>>(map, a);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

}  // namespace qmlr
