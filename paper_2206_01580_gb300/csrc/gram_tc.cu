// Split-BF16 tensor-core Gram G = Z^T Z on sm_103a (tcgen05 + TMA + TMEM).
//
// The normal equations' Z^T Z (RFF section of the paper; "the dominant
// term", built in FP32 with Kahan summation in the paper) is the one dense
// contraction of the method, so it runs on the 5th-generation tensor cores
// with a split-precision BF16 representation of Z:
//   2-way: Z = S0 + S1,       G ~= S0'S0 + S0'S1 + S1'S0                 (~2^-16 rel.)
//   3-way: Z = S0 + S1 + S2,  G ~= S0'S0 + S0'S1 + S1'S0 + S0'S2 + S2'S0 + S1'S1
//                                                                         (~2^-24 rel.)
// with S0 = bf16(Z), S1 = bf16(Z - S0), S2 = bf16(Z - S0 - S1) and FP32
// accumulation in tensor memory. Operands are the transposed splits
// St [N_F][K] (rows of Z contiguous: K-major), loaded by TMA into
// 128-byte-swizzled shared memory.
//
// One CTA computes a 128 x 128 tile of G for the upper triangle only: one
// thread issues TMA copies into a ring of shared-memory stages (full/empty
// mbarriers), one thread issues the split products (tcgen05.mma, 4 per 64-deep
// K block each) into one of two TMEM accumulators, and eight warps promote
// every K block's accumulator into FP32 Kahan sums in registers (the tensor
// cores' accumulator adds truncate; promoting per K block keeps their error
// to one block's worth), then write G[i][j] and its mirror G[j][i] for j >= i.
// Every mbarrier wait is bounded by a clock budget: on expiry the CTA records
// a device error, waits (bounded) for its own copies, frees TMEM and returns.
#include "tcgen05.cuh"

namespace qmlr {

namespace tc {

constexpr int BM = 128;          // tile rows (features i)
constexpr int BK = 64;           // K block: 64 bf16 = 128 bytes (one swizzle row)
constexpr int A_BYTES = BM * BK * 2;        // 16 KB per split part and 128 rows

template <int S>
struct Cfg {
  static constexpr int BN = 128;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = S * A_BYTES + S * B_BYTES;   // 64 KB (2-way), 96 KB (3-way)
  static constexpr int STAGES_N = S == 2 ? 3 : 2;
  static constexpr int SMEM_BYTES = STAGES_N * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
  // products (a-part, b-part) of the split expansion kept
  static constexpr int NP = S == 2 ? 3 : 6;
};
__device__ __constant__ int kProdA[6] = {0, 0, 1, 0, 2, 1};
__device__ __constant__ int kProdB[6] = {0, 1, 0, 2, 0, 1};
// Warp roles (576 threads): warps 0-15 drain the accumulators (warp w reads TMEM
// lanes 32*(w%4).. and columns 32*(w/4)..), warp 16 lane 0 issues TMA, warp 17
// lane 0 issues MMAs. Each 64-deep K block is accumulated into a fresh TMEM
// accumulator (two, used alternately) and promoted into FP32 Kahan sums held
// in the drain threads' registers, so that the tensor cores' accumulator adds
// only ever sum one K block.
constexpr int kDrainWarps = 16;
constexpr int kGroupRows = 16;   // tile rows per rasterization panel
constexpr int kDrainCols = 128 / (kDrainWarps / 4);   // columns per drain thread
constexpr int kThreads = 32 * (kDrainWarps + 2);

template <int S>
__global__ void __launch_bounds__(kThreads, 1)
gram_split_kernel(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1,
                  const __grid_constant__ CUtensorMap map2, int n_features, int k_blocks, int tiles_j,
                  float* __restrict__ G, int* err) {
  using C = Cfg<S>;
  constexpr int BN = C::BN, B_BYTES = C::B_BYTES, STAGE_BYTES = C::STAGE_BYTES, NST = C::STAGES_N;
  const CUtensorMap* maps[3] = {&map0, &map1, &map2};
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NST * STAGE_BYTES);
  uint64_t* empty = full + NST;
  uint64_t* accf = empty + NST;        // [2] accumulator ready (MMA -> drain)
  uint64_t* acce = accf + 2;           // [2] accumulator drained (drain -> MMA)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* never_abort = abort + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // Upper-triangle tiles in grouped order: panels of kGroupRows tile rows,
  // each walked column by column, so the CTAs resident at one time share a
  // few A and B panels (their K-block slices are then served from L2).
  int t = blockIdx.x, bi = 0, bj = 0;
  const int tiles_i = n_features / BM;
  for (int r0 = 0; r0 < tiles_i; r0 += kGroupRows) {
    const int r1 = min(r0 + kGroupRows, tiles_i);
    int cnt = 0;
    for (int c = r0; c < tiles_j; ++c) cnt += min(r1, c + 1) - r0;
    if (t >= cnt) {
      t -= cnt;
      continue;
    }
    for (int c = r0; c < tiles_j; ++c) {
      const int h = min(r1, c + 1) - r0;
      if (t < h) {
        bi = r0 + t;
        bj = c;
        break;
      }
      t -= h;
    }
    break;
  }
  const int i0 = bi * BM, j0 = bj * BN;

  if (threadIdx.x == 0) {
    for (int q = 0; q < NST; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&accf[q], 1);
      mbar_init(&acce[q], kDrainWarps);
    }
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

  if (warp == kDrainWarps && lane == 0) {
    // ---------------- TMA producer
    for (int kb = 0; kb < k_blocks; ++kb) {
      const int st = kb % NST;
      const uint32_t round = kb / NST;
      if (kb >= NST && !mbar_wait(&empty[st], (round - 1) & 1, abort)) {
        record_device_error(err, DEV_TIMEOUT);
        *abort = 1;
        break;
      }
      uint8_t* sp = smem + st * STAGE_BYTES;
      mbar_expect_tx(&full[st], STAGE_BYTES);
      const int k = kb * BK;
#pragma unroll
      for (int q = 0; q < S; ++q) {
        tma_load_2d(sp + q * A_BYTES, maps[q], &full[st], k, i0);
#pragma unroll
        for (int h = 0; h < BN / BM; ++h)
          tma_load_2d(sp + S * A_BYTES + q * B_BYTES + h * A_BYTES, maps[q], &full[st], k, j0 + h * BM);
      }
      last_round[st] = (int)round;
    }
  } else if (warp == kDrainWarps + 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    // descriptors of stage 0's split parts; a stage adds STAGE_BYTES >> 4 and a
    // 16-element K step adds 32 >> 4 = 2 to the start-address field
    uint64_t da[S], db[S];
#pragma unroll
    for (int q = 0; q < S; ++q) {
      da[q] = smem_desc(smem + q * A_BYTES);
      db[q] = smem_desc(smem + S * A_BYTES + q * B_BYTES);
    }
    for (int kb = 0; kb < k_blocks; ++kb) {
      const int st = kb % NST;
      const uint32_t round = kb / NST;
      const int buf = kb & 1;
      const uint32_t use = kb >> 1;
      if (!mbar_wait(&full[st], round & 1, abort) ||
          (use > 0 && !mbar_wait(&acce[buf], (use - 1) & 1, abort))) {
        record_device_error(err, DEV_TIMEOUT);
        *abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint64_t so = (uint64_t)(st * (STAGE_BYTES >> 4));
      const uint32_t d = tmem + buf * BN;
      // smallest split products first, S0'S0 last: every accumulator add
      // truncates relative to the running sum, so the many small terms are
      // added while that sum is still small (4 of the 4 * NP adds are large).
#pragma unroll
      for (int q = C::NP - 1; q >= 0; --q) {
        // (a-part, b-part) of product q: (0,0) (0,1) (1,0) (0,2) (2,0) (1,1), as compile-time indices
        const int qa = q == 2 ? 1 : (q == 4 ? 2 : (q == 5 ? 1 : 0));
        const int qb = q == 1 ? 1 : (q == 3 ? 2 : (q == 5 ? 1 : 0));
        const uint64_t a0 = da[qa] + so, b0 = db[qb] + so;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk)
          mma_bf16(d, a0 + 2 * kk, b0 + 2 * kk, idesc, (kk > 0 || q < C::NP - 1) ? 1u : 0u);
      }
      mma_commit(&empty[st]);   // frees the smem stage once these MMAs have read it
      mma_commit(&accf[buf]);   // accumulator of this K block is ready
    }
  } else if (warp < kDrainWarps) {
    // ---------------- drain: promote each K block into FP32 Kahan sums
    const int quarter = warp & 3, half = warp >> 2;
    float sum[kDrainCols], cmp[kDrainCols];
#pragma unroll
    for (int k = 0; k < kDrainCols; ++k) {
      sum[k] = 0.f;
      cmp[k] = 0.f;
    }
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    for (int kb = 0; kb < k_blocks; ++kb) {
      const int buf = kb & 1;
      const uint32_t use = kb >> 1;
      const bool ok = mbar_wait(&accf[buf], use & 1, abort);
      if (__any_sync(0xffffffffu, !ok)) {
        if (lane == 0) {
          record_device_error(err, DEV_TIMEOUT);
          *abort = 1;
        }
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int c4 = 0; c4 < kDrainCols / 16; ++c4) {
        float v[16];
        tmem_ld16(tmem + lane_base + buf * BN + half * kDrainCols + c4 * 16, v);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int e = c4 * 16 + k;
          const float y = v[k] - cmp[e];
          const float tt = sum[e] + y;
          cmp[e] = (tt - sum[e]) - y;
          sum[e] = tt;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[buf]);
    }
    if (!*abort) {
      const int row = i0 + quarter * 32 + lane;
      if (row < n_features) {
#pragma unroll
        for (int k = 0; k < kDrainCols; ++k) {
          const int col = j0 + half * kDrainCols + k;
          if (col >= row && col < n_features) {
            G[(long)row * n_features + col] = sum[k];
            G[(long)col * n_features + row] = sum[k];
          }
        }
      }
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (*abort) {
    // drain whatever is still in flight before the CTA exits (bounded waits)
    if (warp == kDrainWarps && lane == 0)
      for (int q = 0; q < NST; ++q)
        if (last_round[q] >= 0) mbar_wait(&full[q], (uint32_t)last_round[q] & 1, never_abort);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN));
  }
}

// ---------------------------------------------------------------------------
// Persistent Gram: one CTA per SM walks the tiles of the grouped order in
// waves (tile w * gridDim.x + blockIdx.x), and the TMA producers of all CTAs
// meet at the start of every wave (a counter each producer increments once it
// has issued its wave's loads; bounded wait). The tiles of a wave then stream
// their shared operand panels through the same K range at the same time, so
// fewer of their K-block slices have left L2 before the last tile of the wave
// reads them. Barrier phases and the two TMEM accumulators continue across a
// CTA's tiles; the drain warps write a tile's G block while the MMA thread
// already fills the other accumulator with the next tile's first K block.
//
// Forms (template): S split parts of BF16 (1, 2 or 3) or one e4m3 part with
// per-feature power-of-two scales (F8); tiles of 128 rows x BN columns (128
// or 256); the drain's register sums are Kahan sums (KAHAN) or plain FP32
// sums. Runtime: `promote` K blocks (128-byte lines of K: 64 bf16 or 128 e4m3
// values) are summed in the tensor cores' accumulator between promotions
// into the register sums; promote = 1 bounds the accumulator's truncating
// adds to one block (the accurate forms), promote = 0 keeps a tile's whole K
// range in TMEM (the drain then only runs at the end of a tile).
constexpr long long kWaveSpin = 1LL << 22;

template <int S, bool F8, int BN, bool KAHAN>
struct TcCfg {
  static_assert(S >= 1 && S <= 3 && (!F8 || S == 1), "unsupported split");
  static_assert(BN == 128 || BN == 256, "tile width must be 128 or 256");
  static_assert(!KAHAN || BN == 128, "Kahan register sums need the 128-wide tile");
  static constexpr int B_BYTES = BN * 128;                 // BN rows x one 128-byte line of K
  static constexpr int STAGE_BYTES = S * (A_BYTES + B_BYTES);
  static constexpr int STAGES_N = 196608 / STAGE_BYTES < 8 ? 196608 / STAGE_BYTES : 8;
  static constexpr int SMEM_BYTES = STAGES_N * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
  static constexpr int NP = S == 1 ? 1 : (S == 2 ? 3 : 6);  // split products kept
  static constexpr int COLS = BN / (kDrainWarps / 4);      // drain columns per thread
  static constexpr int KB_ELEMS = F8 ? 128 : 64;           // K values per 128-byte line
};

// Tile rows r (128 features each) that column c (BN features) meets in the upper triangle.
__host__ __device__ __forceinline__ int gram_col_rows(int c, int tiles_i, int bn) {
  const int h = (c + 1) * bn / BM;
  return h < tiles_i ? h : tiles_i;
}

// Tiles of the upper triangle in grouped order: panels of kGroupRows tile rows,
// each walked column by column.
__device__ __forceinline__ void gram_tile_of(int t, int tiles_i, int tiles_j, int bn, int& bi, int& bj) {
  bi = 0;
  bj = 0;
  for (int r0 = 0; r0 < tiles_i; r0 += kGroupRows) {
    const int r1 = min(r0 + kGroupRows, tiles_i);
    const int c0 = r0 * BM / bn;
    int cnt = 0;
    for (int c = c0; c < tiles_j; ++c) cnt += min(r1, gram_col_rows(c, tiles_i, bn)) - r0;
    if (t >= cnt) {
      t -= cnt;
      continue;
    }
    for (int c = c0; c < tiles_j; ++c) {
      const int h = min(r1, gram_col_rows(c, tiles_i, bn)) - r0;
      if (t < h) {
        bi = r0 + t;
        bj = c;
        return;
      }
      t -= h;
    }
    return;
  }
}

template <int S, bool F8, int BN, bool KAHAN>
__global__ void __launch_bounds__(kThreads, 1)
gram_persist_kernel(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1,
                    const __grid_constant__ CUtensorMap map2, int n_features, int k_blocks, int tiles_j,
                    int n_tiles, int promote, unsigned* wave_ctr, const float* __restrict__ inv_scale,
                    float* __restrict__ G, int* err) {
  using C = TcCfg<S, F8, BN, KAHAN>;
  constexpr int B_BYTES = C::B_BYTES, STAGE_BYTES = C::STAGE_BYTES, NST = C::STAGES_N, COLS = C::COLS;
  const CUtensorMap* maps[3] = {&map0, &map1, &map2};
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NST * STAGE_BYTES);
  uint64_t* empty = full + NST;
  uint64_t* accf = empty + NST;        // [2] accumulator ready (MMA -> drain)
  uint64_t* acce = accf + 2;           // [2] accumulator drained (drain -> MMA)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* never_abort = abort + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_i = n_features / BM;
  const int gsz = gridDim.x;
  const int waves = (n_tiles + gsz - 1) / gsz;
  const int P = (promote > 0 && promote < k_blocks) ? promote : k_blocks;   // K blocks per accumulation
  const int groups = (k_blocks + P - 1) / P;

  if (threadIdx.x == 0) {
    for (int q = 0; q < NST; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&accf[q], 1);
      mbar_init(&acce[q], kDrainWarps);
    }
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

  if (warp == kDrainWarps && lane == 0) {
    // ---------------- TMA producer
    int kg = 0;
    for (int w = 0; w < waves && !*abort; ++w) {
      if (w > 0) {   // every CTA has issued the loads of wave w - 1
        long long it = 0;
        const unsigned target = (unsigned)(w * gsz);
        while (*reinterpret_cast<volatile unsigned*>(wave_ctr) < target) {
          if (++it > kWaveSpin) break;
          __nanosleep(64);
        }
        if (*reinterpret_cast<volatile unsigned*>(wave_ctr) < target) {
          record_device_error(err, DEV_TIMEOUT);
          *abort = 1;
          break;
        }
      }
      const int t = w * gsz + blockIdx.x;
      if (t < n_tiles) {
        int bi, bj;
        gram_tile_of(t, tiles_i, tiles_j, BN, bi, bj);
        const int i0 = bi * BM, j0 = bj * BN;
        bool ok = true;
        for (int kb = 0; kb < k_blocks; ++kb, ++kg) {
          const int st = kg % NST;
          const uint32_t round = (uint32_t)(kg / NST);
          if (kg >= NST && !mbar_wait(&empty[st], (round - 1) & 1, abort)) {
            record_device_error(err, DEV_TIMEOUT);
            *abort = 1;
            ok = false;
            break;
          }
          uint8_t* sp = smem + st * STAGE_BYTES;
          mbar_expect_tx(&full[st], STAGE_BYTES);
          const int k = kb * C::KB_ELEMS;
#pragma unroll
          for (int q = 0; q < S; ++q) {
            tma_load_2d(sp + q * A_BYTES, maps[q], &full[st], k, i0);
#pragma unroll
            for (int h = 0; h < BN / BM; ++h)
              tma_load_2d(sp + S * A_BYTES + q * B_BYTES + h * A_BYTES, maps[q], &full[st], k, j0 + h * BM);
          }
          last_round[st] = (int)round;
        }
        if (!ok) break;
      }
      __threadfence();
      atomicAdd(wave_ctr, 1u);
    }
  } else if (warp == kDrainWarps + 1 && lane == 0) {
    // ---------------- MMA issuer: products smallest first; a fresh accumulator per group of P K blocks
    constexpr uint32_t idesc = F8 ? idesc_e4m3(BM, BN) : idesc_bf16(BM, BN);
    uint64_t da[S], db[S];
#pragma unroll
    for (int q = 0; q < S; ++q) {
      da[q] = smem_desc(smem + q * A_BYTES);
      db[q] = smem_desc(smem + S * A_BYTES + q * B_BYTES);
    }
    int kg = 0, gg = 0;
    bool ok = true;
    for (int w = 0; w < waves && ok; ++w) {
      if (w * gsz + blockIdx.x >= n_tiles) continue;
      for (int g = 0; g < groups && ok; ++g, ++gg) {
        const int buf = gg & 1;
        const uint32_t use = (uint32_t)(gg >> 1);
        const int kb0 = g * P, kb1 = min(kb0 + P, k_blocks);
        for (int kb = kb0; kb < kb1; ++kb, ++kg) {
          const int st = kg % NST;
          const uint32_t round = (uint32_t)(kg / NST);
          if (!mbar_wait(&full[st], round & 1, abort) ||
              (kb == kb0 && use > 0 && !mbar_wait(&acce[buf], (use - 1) & 1, abort))) {
            record_device_error(err, DEV_TIMEOUT);
            *abort = 1;
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint64_t so = (uint64_t)(st * (STAGE_BYTES >> 4));
          const uint32_t d = tmem + buf * BN;
          // smallest split products first, S0'S0 last: every accumulator add
          // truncates relative to the running sum, so the many small terms are
          // added while that sum is still small.
#pragma unroll
          for (int q = C::NP - 1; q >= 0; --q) {
            // (a-part, b-part) of product q: (0,0) (0,1) (1,0) (0,2) (2,0) (1,1), as compile-time indices
            const int qa = q == 2 ? 1 : (q == 4 ? 2 : (q == 5 ? 1 : 0));
            const int qb = q == 1 ? 1 : (q == 3 ? 2 : (q == 5 ? 1 : 0));
            const uint64_t a0 = da[qa] + so, b0 = db[qb] + so;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t acc = (kb > kb0 || kk > 0 || q < C::NP - 1) ? 1u : 0u;
              if constexpr (F8)
                mma_e4m3(d, a0 + 2 * kk, b0 + 2 * kk, idesc, acc);
              else
                mma_bf16(d, a0 + 2 * kk, b0 + 2 * kk, idesc, acc);
            }
          }
          mma_commit(&empty[st]);   // frees the smem stage once these MMAs have read it
        }
        if (ok) mma_commit(&accf[buf]);   // the group's accumulator is ready
      }
    }
  } else if (warp < kDrainWarps) {
    // ---------------- drain: per tile, FP32 register sums of the groups, then the G block
    const int quarter = warp & 3, half = warp >> 2;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    int gg = 0;
    bool ok = true;
    for (int w = 0; w < waves && ok; ++w) {
      const int t = w * gsz + blockIdx.x;
      if (t >= n_tiles) continue;
      float sum[COLS], cmp[KAHAN ? COLS : 1];
#pragma unroll
      for (int k = 0; k < COLS; ++k) sum[k] = 0.f;
#pragma unroll
      for (int k = 0; k < (KAHAN ? COLS : 1); ++k) cmp[k] = 0.f;
      for (int g = 0; g < groups; ++g, ++gg) {
        const int buf = gg & 1;
        const uint32_t use = (uint32_t)(gg >> 1);
        const bool got = mbar_wait(&accf[buf], use & 1, abort);
        if (__any_sync(0xffffffffu, !got)) {
          if (lane == 0) {
            record_device_error(err, DEV_TIMEOUT);
            *abort = 1;
          }
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
        for (int c4 = 0; c4 < COLS / 16; ++c4) {
          float v[16];
          tmem_ld16(tmem + lane_base + buf * BN + half * COLS + c4 * 16, v);
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int e = c4 * 16 + k;
            if constexpr (KAHAN) {
              const float y = v[k] - cmp[e];
              const float tt = sum[e] + y;
              cmp[e] = (tt - sum[e]) - y;
              sum[e] = tt;
            } else {
              sum[e] += v[k];
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[buf]);
      }
      if (!ok) break;
      int bi, bj;
      gram_tile_of(t, tiles_i, tiles_j, BN, bi, bj);
      const int i0 = bi * BM, j0 = bj * BN;
      const int row = i0 + quarter * 32 + lane;
      if (row < n_features) {
        const float rs = F8 ? __ldg(inv_scale + row) : 1.0f;
#pragma unroll
        for (int k = 0; k < COLS; ++k) {
          const int col = j0 + half * COLS + k;
          if (col >= row && col < n_features) {
            const float val = F8 ? sum[k] * rs * __ldg(inv_scale + col) : sum[k];
            G[(long)row * n_features + col] = val;
            G[(long)col * n_features + row] = val;
          }
        }
      }
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (*abort) {
    if (warp == kDrainWarps && lane == 0)
      for (int q = 0; q < NST; ++q)
        if (last_round[q] >= 0) mbar_wait(&full[q], (uint32_t)last_round[q] & 1, never_abort);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN));
  }
}

// (hi + lo) - w for a float pair: Knuth's two-sum of hi and -w, its error
// folded into lo, and the pair renormalised by a second two-sum.
__device__ __forceinline__ float2 pair_sub(float2 a, float w) {
  const float s = __fsub_rn(a.x, w);
  const float bb = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(-w, bb));
  const float lo = __fadd_rn(a.y, e);
  const float h = __fadd_rn(s, lo);
  const float b2 = __fsub_rn(h, s);
  return make_float2(h, __fadd_rn(__fsub_rn(s, __fsub_rn(h, b2)), __fsub_rn(lo, b2)));
}

// ---------------------------------------------------------------------------
// Trailing update of the mixed-precision Cholesky factor on the tensor cores:
//   A[i][j] -= sum_k P[i][k] P[j][k],  i >= j,  P = the factored 256-column
// panel below its diagonal block (FP64), given as its 3-way BF16 split
// [3][m][256] (K-major). Each CTA takes one 128 x 128 lower tile, runs the six
// split products per 64-deep K block into TMEM, promotes every K block into
// FP32 register sums (four blocks: K = 256), and subtracts the result from the
// trailing matrix, held as float pairs (hi, lo) in FP32 arithmetic. The epilogue transposes each drain warp's 32 x 32 block
// through its own slice of the (then idle) stage memory so that the
// read-modify-write runs along rows.
constexpr int kPanelK = 256;

__global__ void __launch_bounds__(kThreads, 1)
syrk_tc_kernel(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1,
               const __grid_constant__ CUtensorMap map2, int m, double* __restrict__ A, long lda, int part,
               int* err) {
  using C = Cfg<3>;
  constexpr int BN = C::BN, B_BYTES = C::B_BYTES, STAGE_BYTES = C::STAGE_BYTES, NST = C::STAGES_N;
  constexpr int k_blocks = kPanelK / BK;
  const CUtensorMap* maps[3] = {&map0, &map1, &map2};
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NST * STAGE_BYTES);
  uint64_t* empty = full + NST;
  uint64_t* accf = empty + NST;
  uint64_t* acce = accf + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* never_abort = abort + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // lower-triangle tile (bi >= bj) of this CTA: part 0 = all tiles, part 1 =
  // the first two tile columns (the next panel's columns), part 2 = the rest
  const int T = (m + BM - 1) / BM;
  int bi, bj;
  if (part == 1) {
    const int t = blockIdx.x;
    if (t < T) {
      bi = t;
      bj = 0;
    } else {
      bi = 1 + (t - T);
      bj = 1;
    }
  } else {
    const int t = blockIdx.x;
    bi = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while (bi * (bi + 1) / 2 > t) --bi;
    while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
    bj = t - bi * (bi + 1) / 2;
    if (part == 2) {
      bi += 2;
      bj += 2;
    }
  }
  const int i0 = bi * BM, j0 = bj * BN;

  if (threadIdx.x == 0) {
    for (int q = 0; q < NST; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&accf[q], 1);
      mbar_init(&acce[q], kDrainWarps);
    }
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

  if (warp == kDrainWarps && lane == 0) {
    // ---------------- TMA producer
    for (int kb = 0; kb < k_blocks; ++kb) {
      const int st = kb % NST;
      const uint32_t round = kb / NST;
      if (kb >= NST && !mbar_wait(&empty[st], (round - 1) & 1, abort)) {
        record_device_error(err, DEV_TIMEOUT);
        *abort = 1;
        break;
      }
      uint8_t* sp = smem + st * STAGE_BYTES;
      mbar_expect_tx(&full[st], STAGE_BYTES);
      const int k = kb * BK;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        tma_load_2d(sp + q * A_BYTES, maps[q], &full[st], k, i0);
        tma_load_2d(sp + 3 * A_BYTES + q * B_BYTES, maps[q], &full[st], k, j0);
      }
      last_round[st] = (int)round;
    }
  } else if (warp == kDrainWarps + 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    for (int kb = 0; kb < k_blocks; ++kb) {
      const int st = kb % NST;
      const uint32_t round = kb / NST;
      const int buf = kb & 1;
      const uint32_t use = kb >> 1;
      if (!mbar_wait(&full[st], round & 1, abort) ||
          (use > 0 && !mbar_wait(&acce[buf], (use - 1) & 1, abort))) {
        record_device_error(err, DEV_TIMEOUT);
        *abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint8_t* sp = smem + st * STAGE_BYTES;
      const uint32_t d = tmem + buf * BN;
#pragma unroll
      for (int q = C::NP - 1; q >= 0; --q) {   // smallest products first (see the Gram)
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const int off = kk * 32;
          const uint8_t* a = sp + kProdA[q] * A_BYTES + off;
          const uint8_t* b = sp + 3 * A_BYTES + kProdB[q] * B_BYTES + off;
          mma_bf16(d, smem_desc(a), smem_desc(b), idesc, (kk > 0 || q < C::NP - 1) ? 1u : 0u);
        }
      }
      mma_commit(&empty[st]);
      mma_commit(&accf[buf]);
    }
  } else if (warp < kDrainWarps) {
    // ---------------- drain and FP64 subtraction
    const int quarter = warp & 3, half = warp >> 2;
    float sum[kDrainCols];
#pragma unroll
    for (int k = 0; k < kDrainCols; ++k) sum[k] = 0.f;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    bool done = true;
    for (int kb = 0; kb < k_blocks; ++kb) {
      const int buf = kb & 1;
      const uint32_t use = kb >> 1;
      const bool ok = mbar_wait(&accf[buf], use & 1, abort);
      if (__any_sync(0xffffffffu, !ok)) {
        if (lane == 0) {
          record_device_error(err, DEV_TIMEOUT);
          *abort = 1;
        }
        done = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int c4 = 0; c4 < kDrainCols / 16; ++c4) {
        float v[16];
        tmem_ld16(tmem + lane_base + buf * BN + half * kDrainCols + c4 * 16, v);
#pragma unroll
        for (int k = 0; k < 16; ++k) sum[c4 * 16 + k] += v[k];
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[buf]);
    }
    // This warp saw the last K block's accumulator, so every MMA (and every
    // TMA copy they consumed) has completed and the stage memory is idle.
    if (done && (bi > bj || half <= quarter)) {
      float* W = reinterpret_cast<float*>(smem) + warp * (32 * 33);
#pragma unroll
      for (int k = 0; k < kDrainCols; ++k) W[lane * 33 + k] = sum[k];
      __syncwarp();
      // 16 rows at a time: all loads in flight before the first store
      float2* P = reinterpret_cast<float2*>(A);
      const int j = j0 + half * 32 + lane;
#pragma unroll
      for (int r0 = 0; r0 < 32; r0 += 16) {
        float2 old[16];
#pragma unroll
        for (int rr = 0; rr < 16; ++rr) {
          const int i = i0 + quarter * 32 + r0 + rr;
          old[rr] = (i < m && j <= i) ? P[(long)i * lda + j] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int rr = 0; rr < 16; ++rr) {
          const int i = i0 + quarter * 32 + r0 + rr;
          if (i < m && j <= i) P[(long)i * lda + j] = pair_sub(old[rr], W[(r0 + rr) * 33 + lane]);
        }
      }
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (*abort) {
    if (warp == kDrainWarps && lane == 0)
      for (int q = 0; q < NST; ++q)
        if (last_round[q] >= 0) mbar_wait(&full[q], (uint32_t)last_round[q] & 1, never_abort);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN));
  }
}

// Persistent launch of gram_persist_kernel<S, F8, BN, KAHAN>: one CTA per SM
// (or per tile when there are fewer tiles), cooperative so that the wave
// counter's producers are all resident.
template <int S, bool F8, int BN, bool KAHAN>
static int launch_persist(const void* zt, long k_pad, int n_features, int promote, const float* inv_scale,
                          float* G, cudaStream_t s) {
  using C = TcCfg<S, F8, BN, KAHAN>;
  constexpr int eb = F8 ? 1 : 2;
  CUtensorMap m[3];
  for (int q = 0; q < 3; ++q) {
    const uint8_t* part = static_cast<const uint8_t*>(zt) + (size_t)std::min(q, S - 1) * n_features * k_pad * eb;
    int rc = make_map(&m[q], part, k_pad, n_features, 128, eb);
    if (rc) return rc;
  }
  const int tiles_i = n_features / BM;
  const int tiles_j = n_features / BN;
  int n_tiles = 0;
  for (int c = 0; c < tiles_j; ++c) n_tiles += gram_col_rows(c, tiles_i, BN);
  int coop = 0, dev = 0;
  QMLR_CUDA_TRY(cudaGetDevice(&dev));
  QMLR_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  QMLR_REQUIRE(coop, "the tensor-core Gram needs cooperative launch");
  const void* fn = (const void*)gram_persist_kernel<S, F8, BN, KAHAN>;
  QMLR_CUDA_TRY(smem_attr_once(fn, C::SMEM_BYTES));
  int per_sm = 0;
  QMLR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gram_persist_kernel<S, F8, BN, KAHAN>,
                                                              kThreads, C::SMEM_BYTES));
  QMLR_REQUIRE(per_sm >= 1, "the tensor-core Gram kernel does not fit on an SM");
  const int grid = std::min(sm_count(), n_tiles);
  // a counter of this launch's own (stream-ordered), so that Gram launches
  // on different streams never share one
  void* ctr = nullptr;
  QMLR_CUDA_TRY(cudaMallocAsync(&ctr, sizeof(unsigned), s));
  QMLR_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(unsigned), s));
  unsigned* wave_ctr = static_cast<unsigned*>(ctr);
  int kbl = (int)(k_pad / C::KB_ELEMS);
  int* err = device_error_ptr();
  void* args[] = {(void*)&m[0], (void*)&m[1], (void*)&m[2], (void*)&n_features, (void*)&kbl,
                  (void*)&tiles_j, (void*)&n_tiles, (void*)&promote, (void*)&wave_ctr, (void*)&inv_scale,
                  (void*)&G, (void*)&err};
  const cudaError_t le = cudaLaunchCooperativeKernel(fn, grid, kThreads, args, C::SMEM_BYTES, s);
  QMLR_CUDA_TRY(cudaFreeAsync(ctr, s));
  QMLR_CUDA_TRY(le);
  count_launch();
  return QMLR_OK;
}

template <int S>
static int launch_split(const uint16_t* zt, long k_pad, int n_features, float* G, cudaStream_t s) {
  using namespace tc;
  using C = Cfg<S>;
  const int tiles_i = n_features / BM;
  const int tiles_j = (n_features + C::BN - 1) / C::BN;
  int n_tiles = 0;
  for (int bi = 0; bi < tiles_i; ++bi) n_tiles += tiles_j - (bi * BM) / C::BN;
  if (n_tiles >= 4 * sm_count()) {
    // persistent form: one CTA per SM, producers meet at every wave; the same
    // per-tile arithmetic (Kahan promotion of every K block) as the kernel below
    return launch_persist<S, false, 128, true>(zt, k_pad, n_features, 1, nullptr, G, s);
  }
  CUtensorMap m[3];
  for (int q = 0; q < 3; ++q) {
    const uint16_t* part = zt + (size_t)std::min(q, S - 1) * n_features * k_pad;
    int rc = make_map(&m[q], part, k_pad, n_features);
    if (rc) return rc;
  }
  QMLR_CUDA_TRY(smem_attr_once((const void*)gram_split_kernel<S>, C::SMEM_BYTES));
  gram_split_kernel<S><<<n_tiles, kThreads, C::SMEM_BYTES, s>>>(m[0], m[1], m[2], n_features, (int)(k_pad / BK),
                                                            tiles_j, G, device_error_ptr());
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

static int launch_syrk(const uint16_t* parts, long part_elems, int m, double* A, long lda, int part,
                       cudaStream_t s) {
  using C = Cfg<3>;
  const int T = (m + BM - 1) / BM;
  QMLR_REQUIRE(part_elems >= (long)T * BM * kPanelK, "panel operand smaller than its padded rows");
  CUtensorMap mp[3];
  for (int q = 0; q < 3; ++q) {   // all T * 128 rows are in the buffer (zero beyond m)
    int rc = make_map(&mp[q], parts + (size_t)q * part_elems, kPanelK, T * BM);
    if (rc) return rc;
  }
  QMLR_CUDA_TRY(smem_attr_once((const void*)syrk_tc_kernel, C::SMEM_BYTES));
  int tiles = T * (T + 1) / 2;
  if (part == 1) tiles = T >= 2 ? 2 * T - 1 : T;
  if (part == 2) tiles = T > 2 ? (T - 2) * (T - 1) / 2 : 0;
  if (tiles == 0) return QMLR_OK;
  syrk_tc_kernel<<<tiles, kThreads, C::SMEM_BYTES, s>>>(mp[0], mp[1], mp[2], m, A, lda, part,
                                                        device_error_ptr());
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

}  // namespace tc

int gram_split_tc(int n_split, const uint16_t* zt, long k_pad, int n_features, float* G, cudaStream_t s) {
  if (k_pad == 0) {
    QMLR_CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(float) * (size_t)n_features * n_features, s));
    return QMLR_OK;
  }
  return n_split == 2 ? tc::launch_split<2>(zt, k_pad, n_features, G, s)
                      : tc::launch_split<3>(zt, k_pad, n_features, G, s);
}

// The configurable forms (qmlr_gram_tc): form 1 = 1-part BF16, 2 = 2-way split,
// 3 = 3-way split, 4 = e4m3 with per-feature scales.
int gram_tc_form(int form, int tile_n, int promote, const void* zt, long k_pad, int n_features,
                 const float* inv_scale, float* G, cudaStream_t s) {
  using namespace tc;
  if (k_pad == 0) {
    QMLR_CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(float) * (size_t)n_features * n_features, s));
    return QMLR_OK;
  }
  if (form == 1 && tile_n == 256) return launch_persist<1, false, 256, false>(zt, k_pad, n_features, promote, nullptr, G, s);
  if (form == 1 && tile_n == 128) return launch_persist<1, false, 128, false>(zt, k_pad, n_features, promote, nullptr, G, s);
  if (form == 2 && tile_n == 256) return launch_persist<2, false, 256, false>(zt, k_pad, n_features, promote, nullptr, G, s);
  if (form == 2 && tile_n == 128) return launch_persist<2, false, 128, true>(zt, k_pad, n_features, promote, nullptr, G, s);
  if (form == 3 && tile_n == 128) return launch_persist<3, false, 128, true>(zt, k_pad, n_features, promote, nullptr, G, s);
  if (form == 4 && tile_n == 256) return launch_persist<1, true, 256, false>(zt, k_pad, n_features, promote, inv_scale, G, s);
  if (form == 4 && tile_n == 128) return launch_persist<1, true, 128, false>(zt, k_pad, n_features, promote, inv_scale, G, s);
  set_error("unsupported tensor-core Gram form %d with %d-wide tiles", form, tile_n);
  return QMLR_EINVAL;
}

int syrk_tc(const uint16_t* parts, long part_elems, int m, double* A, long lda, int part, cudaStream_t s) {
  if (m <= 0) return QMLR_OK;
  return tc::launch_syrk(parts, part_elems, m, A, lda, part, s);
}

}  // namespace qmlr
