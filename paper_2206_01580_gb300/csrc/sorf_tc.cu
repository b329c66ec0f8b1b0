// SORF energies and gradients on the tensor cores (sm_103a: tcgen05 + TMA + TMEM).
//
// SORF section of the paper: each stack s maps x (d = 128) to
//   u_s = c * M_s x + b_s,   M_s = H D_{s,T} ... H D_{s,1},   c = (sqrt(d)/sigma) / d^{T/2},
// with H the unnormalised Walsh-Hadamard matrix and D the Rademacher signs;
// the atomic energy is eps = sqrt(2/N_F) sum_s alpha_s . cos(u_s) (RFF section,
// atomic energy partition) and its gradient
//   d eps / dx = -sqrt(2/N_F) c sum_s M_s^T (alpha_s * sin(u_s)).
// The fast transform needs 2 T log2(d) FP32 adds per feature and direction on
// the CUDA cores; here both directions run as dense products on the tensor
// cores instead. M_s has integer entries bounded by d^{T/2} (1448 for d = 128,
// T = 3), which FP16 holds exactly, so the chain itself carries no rounding:
//   forward : D_s = X M_s^T  with X = 2^-k (Xh + Xl) split into two FP16 parts
//             per atom (row scale 2^k puts the row maximum in [2^14, 2^15),
//             each part keeps 11 bits: 2^-22 relative per element);
//   backward: G = sum_s Y_s M_s with Y_s = S alpha_s * sin(u_s) split the same
//             way (S: one power of two for all features, max |alpha| S in
//             [2^14, 2^15)).
// Four FP16 products of 128 x 64 x 128 per half stack, FP32 accumulation in
// tensor memory; the backward accumulator is promoted into FP32 register sums
// every few half stacks (the accumulator adds truncate; short runs keep their
// error small).
//
// Kernel layout: persistent, one CTA per SM, tiles of 128 atoms (one TMEM lane
// per atom). A unit is half a stack (64 features). Warp 16 issues TMA (the
// tile's two X parts once, then per unit the forward tile of M_s, the backward
// tile of M_s^T and the unit's 64 phases and weights), warp 17 issues the MMAs
// (forward of unit n, then backward of unit n - 1), warps 0-15 run the
// epilogue (four per SM sub-partition, to hide the latency of the sin/cos
// chains): each reads 16 columns of the unit's accumulator for its atom, forms the
// phases, sin and cos, the energy partial and the two FP16 parts of Y, and
// writes them 128-byte swizzled for the backward MMA. Every wait is bounded:
// on expiry the CTA records DEV_TIMEOUT, stops, waits (bounded) for its own
// copies and MMAs in flight, frees TMEM and returns.
#include "model_internal.cuh"
#include "sorf_math.cuh"
#include "tcgen05.cuh"

#include <cuda_fp16.h>

namespace qmlr {
namespace stc {

using namespace tc;

constexpr int D = 128;        // projected dimension = features per stack
constexpr int TM = 128;       // atoms per tile
constexpr int UN = 64;        // features per unit (half a stack)
constexpr int NS = 7;         // ring of 16 KB operand tiles (forward and backward, in MMA order)
constexpr int NDB = 4;        // forward accumulators (64 TMEM columns each)
constexpr int NYS = 1;        // Y slots
constexpr int NBA = 8;        // phase / weight slots
constexpr int LA = 1;         // the backward of unit n is issued after the forward of unit n + LA
constexpr int kEpiWarps = 16;   // four per SM sub-partition
constexpr int CQ = kEpiWarps / 4;   // column groups (warps sharing a TMEM lane quarter)
constexpr int CW = 64 / CQ;         // accumulator columns of a unit per epilogue thread
constexpr int GW = 128 / CQ;        // gradient dimensions per epilogue thread
constexpr int kThreads = 32 * (kEpiWarps + 2);

constexpr int X_BYTES = 2 * TM * D * 2;     // two FP16 parts x two 64-wide K blocks
constexpr int TILE_BYTES = 16384;           // one operand tile
constexpr int Y_BYTES = 2 * TM * UN * 2;    // two FP16 parts of one unit
constexpr int BA_FLOATS = 2 * UN;           // 64 phases, 64 weights
constexpr int OFF_X = 0;
constexpr int OFF_B = OFF_X + X_BYTES;
constexpr int OFF_Y = OFF_B + NS * TILE_BYTES;
constexpr int OFF_BA = OFF_Y + NYS * Y_BYTES;
constexpr int OFF_RED = OFF_BA + NBA * BA_FLOATS * 4;    // double [2 tile parities][CQ - 1][TM]
constexpr int OFF_BAR = OFF_RED + 2 * (CQ - 1) * TM * 8;
constexpr int N_BARS = 2 + 2 * NS + 2 * NBA + 2 * NDB + 2 * NYS + 2 * 2 + 2 * 4 + 1;
constexpr int SMEM_BYTES = OFF_BAR + N_BARS * 8 + 64 + 1024;
constexpr int TMEM_COLS = 512;   // NDB x 64 forward + 2 x 128 backward

static_assert(NDB * UN + 2 * D <= TMEM_COLS, "TMEM budget");
static_assert((CW == 16 || CW == 32) && GW % 32 == 0, "epilogue TMEM loads: 16 or 32 unit columns, gradient in 32s");
static_assert(SMEM_BYTES <= 227 * 1024, "shared-memory budget");

struct Args {
  const float* kx;       // [n_pad] 2^-k of each atom's row scale
  const float* b;        // [N_F] phases, natural order (stack-major)
  const float* alpha;    // [N_F] weights times S, natural order
  const float* ys;       // [2]: S, a power of two with max |alpha| S in [2^14, 2^15), and 1/S
  double* atom_e;        // [n_atoms]
  float* gx;             // [n_atoms][D]
  int n_atoms, n_pad, n_tiles, n_stack, period_log2;   // backward promotion every 2^period_log2 units
  float cscale;          // (sqrt(d)/sigma) / d^{T/2}
  float pref;            // sqrt(2/N_F)
  int* err;
};

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void tmem_ldn(uint32_t taddr, float (&v)[16]) { tmem_ld16(taddr, v); }
__device__ __forceinline__ void tmem_ldn(uint32_t taddr, float (&v)[32]) { tmem_ld32(taddr, v); }

// kind::f16 instruction descriptor with FP16 A and B (format code 0), FP32 D, K-major.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t h2_bits(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }

__global__ void __launch_bounds__(kThreads, 1)
sorf_tc_kernel(const __grid_constant__ CUtensorMap mapx, const __grid_constant__ CUtensorMap mapf,
               const __grid_constant__ CUtensorMap mapb, Args a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sx = smem + OFF_X;
  uint8_t* sb = smem + OFF_B;
  uint8_t* sy = smem + OFF_Y;
  float* sba = reinterpret_cast<float*>(smem + OFF_BA);
  double* red = reinterpret_cast<double*>(smem + OFF_RED);
  uint64_t* xfull = reinterpret_cast<uint64_t*>(smem + OFF_BAR);
  uint64_t* xempty = xfull + 1;
  uint64_t* bfull = xempty + 1;
  uint64_t* bempty = bfull + NS;
  uint64_t* bafull = bempty + NS;
  uint64_t* baempty = bafull + NBA;
  uint64_t* dfull = baempty + NBA;
  uint64_t* dempty = dfull + NDB;
  uint64_t* yfull = dempty + NDB;
  uint64_t* yempty = yfull + NYS;
  uint64_t* gfull = yempty + NYS;
  uint64_t* gempty = gfull + 2;
  uint64_t* efull = gempty + 2;     // [2 parities][4 quarters]: energy partials of column groups 1.. written
  uint64_t* mdone = efull + 8;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mdone + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* never_abort = abort + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int U = 2 * a.n_stack, PL = a.period_log2, P = 1 << PL, PM = P - 1;

  if (threadIdx.x == 0) {
    mbar_init(xfull, 1);
    mbar_init(xempty, 1);
    for (int q = 0; q < NS; ++q) {
      mbar_init(&bfull[q], 1);
      mbar_init(&bempty[q], 1);
    }
    for (int q = 0; q < NBA; ++q) {
      mbar_init(&bafull[q], 1);
      mbar_init(&baempty[q], kEpiWarps);
    }
    for (int q = 0; q < NDB; ++q) {
      mbar_init(&dfull[q], 1);
      mbar_init(&dempty[q], kEpiWarps);
    }
    for (int q = 0; q < NYS; ++q) {
      mbar_init(&yfull[q], kEpiWarps);
      mbar_init(&yempty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&gfull[q], 1);
      mbar_init(&gempty[q], kEpiWarps);
    }
    for (int q = 0; q < 8; ++q) mbar_init(&efull[q], CQ - 1);
    mbar_init(mdone, 1);
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
  const float S = __ldg(a.ys), inv_s = __ldg(a.ys + 1);

  int last_x = -1, last_b[NS], last_ba[NBA];
#pragma unroll
  for (int q = 0; q < NS; ++q) last_b[q] = -1;
#pragma unroll
  for (int q = 0; q < NBA; ++q) last_ba[q] = -1;

  if (warp == kEpiWarps && lane == 0) {
    // ------------------------------------------------------------ TMA producer
    int q = 0, n = 0;
    int k = 0;
    bool ok = true;
    // every CTA walks the stacks in the same order: an atom's energy and gradient
    // sums then do not depend on the CTA (or batch) that computes it
    const int s0 = 0;
    for (int tile = blockIdx.x; ok && tile < a.n_tiles; tile += gridDim.x, ++k, n += U) {
      if (k > 0 && !mbar_wait(xempty, (k - 1) & 1, abort)) {
        ok = false;
        break;
      }
      mbar_expect_tx(xfull, X_BYTES);
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int kb = 0; kb < 2; ++kb)
          tma_load_2d(sx + p * (X_BYTES / 2) + kb * (X_BYTES / 4), &mapx, xfull, kb * 64, p * a.n_pad + tile * TM);
      last_x = k;
      for (int j = 0; ok && j < U + LA; ++j) {
        if (j < U) {
          const int un = n + j;
          int s = (j >> 1) + s0;
          if (s >= a.n_stack) s -= a.n_stack;
          const int h = j & 1;
          const int bs = (int)(un % NBA);
          if (un >= NBA && !mbar_wait(&baempty[bs], (uint32_t)((un / NBA) - 1) & 1, abort)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&bafull[bs], BA_FLOATS * 4);
          bulk_load(sba + bs * BA_FLOATS, a.b + (long)s * D + h * UN, UN * 4, &bafull[bs]);
          bulk_load(sba + bs * BA_FLOATS + UN, a.alpha + (long)s * D + h * UN, UN * 4, &bafull[bs]);
          last_ba[bs] = (int)(un / NBA);
          const int st = (int)(q % NS);
          if (q >= NS && !mbar_wait(&bempty[st], (uint32_t)((q / NS) - 1) & 1, abort)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&bfull[st], TILE_BYTES);
          tma_load_2d(sb + st * TILE_BYTES, &mapf, &bfull[st], 0, s * D + h * UN);
          tma_load_2d(sb + st * TILE_BYTES + TILE_BYTES / 2, &mapf, &bfull[st], 64, s * D + h * UN);
          last_b[st] = (int)(q / NS);
          ++q;
        }
        if (j >= LA) {
          const int jm = j - LA, h = jm & 1;
          int s = (jm >> 1) + s0;
          if (s >= a.n_stack) s -= a.n_stack;
          const int st = (int)(q % NS);
          if (q >= NS && !mbar_wait(&bempty[st], (uint32_t)((q / NS) - 1) & 1, abort)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&bfull[st], TILE_BYTES);
          tma_load_2d(sb + st * TILE_BYTES, &mapb, &bfull[st], h * UN, s * D);
          last_b[st] = (int)(q / NS);
          ++q;
        }
      }
    }
    if (!ok) {
      record_device_error(a.err, DEV_TIMEOUT);
      *abort = 1;
    }
  } else if (warp == kEpiWarps + 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    constexpr uint32_t idf = idesc_f16(TM, UN), idb = idesc_f16(TM, D);
    int q = 0, n = 0;
    int k = 0;
    bool ok = true;
    for (int tile = blockIdx.x; ok && tile < a.n_tiles; tile += gridDim.x, ++k, n += U) {
      if (!mbar_wait(xfull, k & 1, abort)) {
        ok = false;
        break;
      }
      for (int j = 0; ok && j < U + LA; ++j) {
        if (j < U) {
          const int un = n + j;
          const int st = q % NS, db = un % NDB;
          if (!mbar_wait(&bfull[st], (uint32_t)(q / NS) & 1, abort) ||
              (un >= NDB && !mbar_wait(&dempty[db], (uint32_t)((un / NDB) - 1) & 1, abort))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t d = tmem + db * UN;
          // low part first: its small terms are added while the accumulator is small
#pragma unroll
          for (int p = 1; p >= 0; --p)
#pragma unroll
            for (int kk = 0; kk < D / 16; ++kk) {
              const uint64_t da = smem_desc(sx + p * (X_BYTES / 2) + (kk >> 2) * (X_BYTES / 4)) + 2 * (kk & 3);
              const uint64_t dbd = smem_desc(sb + st * TILE_BYTES + (kk >> 2) * (TILE_BYTES / 2)) + 2 * (kk & 3);
              mma_bf16(d, da, dbd, idf, (p == 1 && kk == 0) ? 0u : 1u);
            }
          mma_commit(&bempty[st]);
          mma_commit(&dfull[db]);
          if (j == U - 1) mma_commit(xempty);
          ++q;
        }
        if (j >= LA) {
          const int um = n + j - LA;
          const int st = q % NS, ys = um % NYS;
          const int gp = um >> PL;
          const int gb = gp & 1;
          const bool first = (um & PM) == 0;
          if (!mbar_wait(&bfull[st], (uint32_t)(q / NS) & 1, abort) ||
              !mbar_wait(&yfull[ys], (uint32_t)(um / NYS) & 1, abort) ||
              (first && gp >= 2 && !mbar_wait(&gempty[gb], (uint32_t)((gp / 2) - 1) & 1, abort))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t g = tmem + NDB * UN + gb * D;
#pragma unroll
          for (int p = 1; p >= 0; --p)
#pragma unroll
            for (int kk = 0; kk < UN / 16; ++kk) {
              const uint64_t da = smem_desc(sy + ys * Y_BYTES + p * (Y_BYTES / 2)) + 2 * kk;
              const uint64_t dbd = smem_desc(sb + st * TILE_BYTES) + 2 * kk;
              mma_bf16(g, da, dbd, idb, (first && p == 1 && kk == 0) ? 0u : 1u);
            }
          mma_commit(&bempty[st]);
          mma_commit(&yempty[ys]);
          if ((um & PM) == PM) mma_commit(&gfull[gb]);
          ++q;
        }
      }
    }
    if (!ok) {
      record_device_error(a.err, DEV_TIMEOUT);
      *abort = 1;
    }
    // every MMA issued above has completed before TMEM is released
    mma_commit(mdone);
    mbar_wait(mdone, 0, never_abort);
  } else if (warp < kEpiWarps) {
    // ------------------------------------------------------------ epilogue
    // warp = (column group cg, lane quarter): TMEM lanes 32*quarter.., unit
    // columns cg*CW.., gradient dimensions cg*GW..
    const int quarter = warp & 3, cg = warp >> 2;
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    const float gscale = -a.pref * a.cscale * inv_s;
    float g[GW];
    int n = 0;
    int k = 0;
    bool ok = true;
    auto fail = [&]() {
      if (lane == 0) {
        record_device_error(a.err, DEV_TIMEOUT);
        *abort = 1;
      }
      ok = false;
    };
    // add the backward accumulator of period gp into the register sums
    auto promote = [&](int gp) {
      const int gb = gp & 1;
      const bool w = mbar_wait(&gfull[gb], (uint32_t)(gp / 2) & 1, abort);
      if (__any_sync(0xffffffffu, !w)) {
        fail();
        return;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int c2 = 0; c2 < GW / 32; ++c2) {
        float t[32];
        tmem_ld32(tmem + lane_base + NDB * UN + gb * D + cg * GW + c2 * 32, t);
#pragma unroll
        for (int i = 0; i < 32; ++i) g[c2 * 32 + i] += t[i];
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(&gempty[gb]);
    };
    for (int tile = blockIdx.x; ok && tile < a.n_tiles; tile += gridDim.x, ++k, n += U) {
      const int atom = tile * TM + row;
      const bool valid = atom < a.n_atoms;
      const float cs = a.cscale * __ldg(a.kx + atom);   // atom < n_pad always
#pragma unroll
      for (int i = 0; i < GW; ++i) g[i] = 0.f;
      double e_tile = 0.0;
      float e_f = 0.f;
      for (int j = 0; j < U; ++j) {
        const int un = n + j;
        if (j >= P && (j & PM) == 1) {
          promote((un >> PL) - 1);
          if (!ok) break;
        }
        const int db = un % NDB, bs = un % NBA, ys = un % NYS;
        bool w = mbar_wait(&dfull[db], (uint32_t)(un / NDB) & 1, abort);
        if (__any_sync(0xffffffffu, !w)) {
          fail();
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        float v[CW];
        tmem_ldn(tmem + lane_base + db * UN + cg * CW, v);
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) mbar_arrive(&dempty[db]);
        w = mbar_wait(&bafull[bs], (uint32_t)(un / NBA) & 1, abort);
        if (__any_sync(0xffffffffu, !w)) {
          fail();
          break;
        }
        const float4* b4 = reinterpret_cast<const float4*>(sba + bs * BA_FLOATS + cg * CW);
        const float4* a4 = reinterpret_cast<const float4*>(sba + bs * BA_FLOATS + UN + cg * CW);
#pragma unroll
        for (int c = 0; c < CW / 4; ++c) {
          const float4 bb = b4[c], aa = a4[c];
          const float bv[4] = {bb.x, bb.y, bb.z, bb.w}, av[4] = {aa.x, aa.y, aa.z, aa.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            float sn, cn;
            fast_sincos(fmaf(v[4 * c + e], cs, bv[e]), &sn, &cn);
            e_f = fmaf(av[e], cn, e_f);
            v[4 * c + e] = av[e] * sn;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&baempty[bs]);
        if (un >= NYS) {
          w = mbar_wait(&yempty[ys], (uint32_t)((un / NYS) - 1) & 1, abort);
          if (__any_sync(0xffffffffu, !w)) {
            fail();
            break;
          }
        }
        // Y parts: row `row`, K offset cg*CW of the unit, 128-byte swizzle
        uint8_t* yrow = sy + ys * Y_BYTES + (row >> 3) * 1024 + (row & 7) * 128;
#pragma unroll
        for (int cc = 0; cc < CW / 8; ++cc) {
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int i = cc * 8 + 2 * t;
            const __half2 hi = __floats2half2_rn(v[i], v[i + 1]);
            const float2 hf = __half22float2(hi);
            const __half2 lo = __floats2half2_rn(v[i] - hf.x, v[i + 1] - hf.y);
            hw[t] = h2_bits(hi);
            lw[t] = h2_bits(lo);
          }
          const int chunk = ((cg * (CW / 8) + cc) ^ (row & 7)) * 16;
          *reinterpret_cast<uint4*>(yrow + chunk) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *reinterpret_cast<uint4*>(yrow + Y_BYTES / 2 + chunk) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&yfull[ys]);
        if ((j & PM) == PM) {
          e_tile += (double)e_f;
          e_f = 0.f;
        }
      }
      if (!ok) break;
      promote((n + U - 1) >> PL);
      if (!ok) break;
      if (valid) {
        float4* o = reinterpret_cast<float4*>(a.gx + (long)atom * D + cg * GW);
#pragma unroll
        for (int c = 0; c < GW / 4; ++c)
          o[c] = make_float4(g[4 * c] * gscale, g[4 * c + 1] * gscale, g[4 * c + 2] * gscale, g[4 * c + 3] * gscale);
      }
      // energy: column group 0 adds the other groups' partials (written to red) in order
      double* rb = red + (k & 1) * (CQ - 1) * TM;
      uint64_t* eb = &efull[(k & 1) * 4 + quarter];
      if (cg > 0) {
        rb[(cg - 1) * TM + row] = e_tile;
        __syncwarp();
        if (lane == 0) mbar_arrive(eb);
      } else {
        const bool w = mbar_wait(eb, (uint32_t)(k / 2) & 1, abort);
        if (__any_sync(0xffffffffu, !w)) {
          fail();
          break;
        }
        double e = e_tile;
#pragma unroll
        for (int c = 0; c < CQ - 1; ++c) e += rb[c * TM + row];
        if (valid) a.atom_e[atom] = e * (double)a.pref * (double)inv_s;
      }
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (*abort && warp == kEpiWarps && lane == 0) {
    // copies still in flight land before the CTA exits (bounded waits)
    if (last_x >= 0) mbar_wait(xfull, (uint32_t)last_x & 1, never_abort);
    for (int q = 0; q < NS; ++q)
      if (last_b[q] >= 0) mbar_wait(&bfull[q], (uint32_t)last_b[q] & 1, never_abort);
    for (int q = 0; q < NBA; ++q)
      if (last_ba[q] >= 0) mbar_wait(&bafull[q], (uint32_t)last_ba[q] & 1, never_abort);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// Row-scaled two-part FP16 split of x (one warp per atom, lanes own 4 dims):
// xs = x 2^k with max |xs| in [2^14, 2^15), Xh = fp16(xs), Xl = fp16(xs - Xh),
// kx = 2^-k; rows n_atoms .. n_pad-1 are zero. Also the phase-reduction range
// check of the SORF kernels (|x|^2 <= x2max, else DEV_RANGE).
__global__ void split_x_kernel(const float* __restrict__ x, int n_atoms, int n_pad, float x2max,
                               __half* __restrict__ xh, float* __restrict__ kx, int* err) {
  const int atom = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (atom >= n_pad) return;
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (atom < n_atoms) v = __ldg(reinterpret_cast<const float4*>(x + (long)atom * D) + lane);
  float m = fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)));
  float q = v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    q += __shfl_xor_sync(0xffffffffu, q, o);
  }
  if (lane == 0 && atom < n_atoms && !(q <= x2max)) record_device_error(err, DEV_RANGE);
  int e = 0;
  frexpf(m, &e);
  const int k = (m > 0.f && m < 1e30f) ? min(max(15 - e, -100), 100) : 0;
  const float f[4] = {ldexpf(v.x, k), ldexpf(v.y, k), ldexpf(v.z, k), ldexpf(v.w, k)};
  __half hi[4], lo[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    hi[t] = __float2half_rn(f[t]);
    lo[t] = __float2half_rn(f[t] - __half2float(hi[t]));
  }
  __half* ph = xh + (long)atom * D + 4 * lane;
  __half* pl = xh + ((long)n_pad + atom) * D + 4 * lane;
  *reinterpret_cast<uint2*>(ph) = make_uint2(h2_bits(__halves2half2(hi[0], hi[1])), h2_bits(__halves2half2(hi[2], hi[3])));
  *reinterpret_cast<uint2*>(pl) = make_uint2(h2_bits(__halves2half2(lo[0], lo[1])), h2_bits(__halves2half2(lo[2], lo[3])));
  if (lane == 0) kx[atom] = ldexpf(1.f, -k);
}

// S = 2^(15 - e) for max |alpha| = m 2^e, m in [0.5, 1) (so max |alpha| S lies in
// [2^14, 2^15), the range of the backward operand's FP16 parts), 1/S, and
// alpha_sc = alpha S (exact: a power-of-two scale). One CTA.
__global__ void __launch_bounds__(1024) alpha_scale_kernel(const float* __restrict__ alpha, int n,
                                                           float* __restrict__ ys, float* __restrict__ alpha_sc) {
  __shared__ float wmax[32];
  __shared__ float s_sc;
  float m = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, fabsf(alpha[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float mm = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmaxf(mm, wmax[w]);
    int ex = 0;
    frexpf(mm, &ex);
    const int k = (mm > 0.f && mm < 1e30f) ? min(max(15 - ex, -100), 100) : 0;
    s_sc = ldexpf(1.f, k);
    ys[0] = s_sc;
    ys[1] = ldexpf(1.f, -k);
  }
  __syncthreads();
  const float sc = s_sc;
  for (int i = threadIdx.x; i < n; i += blockDim.x) alpha_sc[i] = alpha[i] * sc;
}

// Forward and backward operand tables of the chains (exact integers in FP16):
// mf[s][i][j] = (M_s)_{ij} (rows = features, K = dims) and mb[s][j][i] = (M_s)_{ij}
// (rows = dims, K = features). One thread per (stack, column j): the chain of
// e_j in FP32 (exact: |entries| <= d^{T/2} < 2^24).
__global__ void __launch_bounds__(D) chain_tables_kernel(const uint32_t* __restrict__ sign_bits, int T,
                                                         __half* __restrict__ mf, __half* __restrict__ mb) {
  constexpr int W = D / 32;
  const int s = blockIdx.x, j = threadIdx.x;
  float v[D];
#pragma unroll
  for (int i = 0; i < D; ++i) v[i] = i == j ? 1.f : 0.f;
  for (int t = 0; t < T; ++t) {
    uint32_t w[W];
#pragma unroll
    for (int q = 0; q < W; ++q) w[q] = __ldg(sign_bits + ((long)s * T + t) * W + q);
    flip<D>(v, w);
    fwht<D>(v);
  }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const __half h = __float2half_rn(v[i]);
    mf[((long)s * D + i) * D + j] = h;
    mb[((long)s * D + j) * D + i] = h;
  }
}


// ---------------------------------------------------------------------------
// Segment sums Z_m = sqrt(2/N_F) sum_{I in m} cos(u(x_I)) on the tensor cores:
// the energy rows of the normal equations (SORF and RFF sections). Forward
// chains only (two FP16 products per unit, as above); the epilogue writes
// cos(c D + b) of its 16 columns to a padded shared-memory tile, and reader
// threads (one feature column and one molecule slot each) add each molecule's
// rows in atom order. Each CTA owns a contiguous range of whole molecules
// (split at molecule starts, balanced by atom count) and walks it in tiles of
// 128 atoms from the range's first atom; a molecule that crosses a tile
// boundary is carried to the next tile through a per-CTA row in global memory,
// always by the same thread. Every row of Z is written exactly once (empty
// molecules as zeros); the order of every sum is fixed: deterministic.
namespace zc {
constexpr int NSZ = 5;               // ring of forward operand tiles
constexpr int NBZ = 8;               // phase slots (64 floats each)
constexpr int CLD = UN + 4;          // padded row of the cos tile (floats)
constexpr int C_BYTES = TM * CLD * 4;
constexpr int OFF_X = 0;
constexpr int OFF_B = OFF_X + X_BYTES;
constexpr int OFF_C = OFF_B + NSZ * TILE_BYTES;
constexpr int OFF_BZ = OFF_C + 2 * C_BYTES;
constexpr int OFF_BAR = OFF_BZ + NBZ * UN * 4;
constexpr int N_BARS = 2 + 2 * NSZ + 2 * NBZ + 2 * NDB + 2 * 2 + 1;
constexpr int SMEM_BYTES = OFF_BAR + N_BARS * 8 + 64 + 1024;
constexpr int TMEM_COLS = 256;
constexpr int kSlots = kEpiWarps * 32 / UN;   // molecule slots of the reader threads
static_assert(SMEM_BYTES <= 227 * 1024, "shared-memory budget");
static_assert(NDB * UN <= TMEM_COLS, "TMEM budget");
static_assert(kSlots >= 3, "reader slots");
}  // namespace zc

struct ZArgs {
  const float* kx;          // [n_pad] row scales of the FP16 parts
  const float* b;           // [N_F] phases
  const int32_t* mol_ptr;   // [n_mol + 1]
  float* Z;                 // [n_mol][ldz]
  long ldz;
  float* carry;             // [gridDim.x][N_F] raw sums of molecules crossing a tile boundary
  int n_atoms, n_mol, n_pad, n_stack;
  float cscale, pref;
  int* err;
};

// first m in [0, n] with p[m] >= v (p non-decreasing)
__device__ __forceinline__ int lower_bound_i(const int32_t* p, int n, long v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(p + mid) < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
// first m in [0, n] with p[m] > v
__device__ __forceinline__ int upper_bound_i(const int32_t* p, int n, long v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(p + mid) <= v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Rows [a0, a1) of one tile and the molecules [mf, mf + nm) that own them; sin:
// the first molecule started in an earlier tile, sout: the last one continues.
struct ZTile {
  int a0, a1, mf, nm;
  bool sin, sout;
};

__device__ __forceinline__ ZTile z_tile(const int32_t* mol_ptr, int n_mol, int A0, int A1, int M0, int M1, int k,
                                        int n_tiles) {
  ZTile t;
  t.a0 = A0 + k * TM;
  t.a1 = min(t.a0 + TM, A1);
  const bool last = k == n_tiles - 1;
  int mf;
  if (k == 0) {
    mf = M0;
    t.sin = false;
  } else {
    const int mc = upper_bound_i(mol_ptr, n_mol + 1, t.a0) - 1;   // the molecule holding atom a0
    t.sin = __ldg(mol_ptr + mc) < t.a0;
    mf = t.sin ? mc : lower_bound_i(mol_ptr, n_mol + 1, t.a0);
  }
  const int me = last ? M1 : lower_bound_i(mol_ptr, n_mol + 1, t.a1);
  t.mf = mf;
  t.nm = me - mf;
  t.sout = !last && t.nm > 0 && __ldg(mol_ptr + me) > t.a1;
  return t;
}

__global__ void __launch_bounds__(kThreads, 1)
sorf_z_tc_kernel(const __grid_constant__ CUtensorMap mapx, const __grid_constant__ CUtensorMap mapf, ZArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sx = smem + zc::OFF_X;
  uint8_t* sb = smem + zc::OFF_B;
  float* sc = reinterpret_cast<float*>(smem + zc::OFF_C);
  float* sbz = reinterpret_cast<float*>(smem + zc::OFF_BZ);
  uint64_t* xfull = reinterpret_cast<uint64_t*>(smem + zc::OFF_BAR);
  uint64_t* xempty = xfull + 1;
  uint64_t* bfull = xempty + 1;
  uint64_t* bempty = bfull + zc::NSZ;
  uint64_t* bzfull = bempty + zc::NSZ;
  uint64_t* bzempty = bzfull + zc::NBZ;
  uint64_t* dfull = bzempty + zc::NBZ;
  uint64_t* dempty = dfull + NDB;
  uint64_t* cfull = dempty + NDB;
  uint64_t* cempty = cfull + 2;
  uint64_t* mdone = cempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mdone + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* never_abort = abort + 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int U = 2 * a.n_stack, NF = a.n_stack * D;
  // this CTA's molecules [M0, M1) and atoms [A0, A1)
  const int M0 = blockIdx.x == 0 ? 0 : lower_bound_i(a.mol_ptr, a.n_mol + 1, (long)blockIdx.x * a.n_atoms / gridDim.x);
  const int M1 = blockIdx.x == gridDim.x - 1
                     ? a.n_mol
                     : lower_bound_i(a.mol_ptr, a.n_mol + 1, (long)(blockIdx.x + 1) * a.n_atoms / gridDim.x);
  const int A0 = __ldg(a.mol_ptr + M0), A1 = __ldg(a.mol_ptr + M1);
  const int n_tiles = (A1 - A0 + TM - 1) / TM;
  const int s0 = (int)(((long)blockIdx.x * a.n_stack) / gridDim.x);

  if (threadIdx.x == 0) {
    mbar_init(xfull, 1);
    mbar_init(xempty, 1);
    for (int q = 0; q < zc::NSZ; ++q) {
      mbar_init(&bfull[q], 1);
      mbar_init(&bempty[q], 1);
    }
    for (int q = 0; q < zc::NBZ; ++q) {
      mbar_init(&bzfull[q], 1);
      mbar_init(&bzempty[q], kEpiWarps);
    }
    for (int q = 0; q < NDB; ++q) {
      mbar_init(&dfull[q], 1);
      mbar_init(&dempty[q], kEpiWarps);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&cfull[q], kEpiWarps);
      mbar_init(&cempty[q], kEpiWarps);
    }
    mbar_init(mdone, 1);
    *abort = 0;
    *never_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(zc::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;

  int last_x = -1, last_b[zc::NSZ], last_bz[zc::NBZ];
#pragma unroll
  for (int q = 0; q < zc::NSZ; ++q) last_b[q] = -1;
#pragma unroll
  for (int q = 0; q < zc::NBZ; ++q) last_bz[q] = -1;

  if (warp == kEpiWarps && lane == 0) {
    // ------------------------------------------------------------ TMA producer
    int q = 0, n = 0;
    bool ok = true;
    for (int k = 0; ok && k < n_tiles; ++k, n += U) {
      if (k > 0 && !mbar_wait(xempty, (k - 1) & 1, abort)) {
        ok = false;
        break;
      }
      mbar_expect_tx(xfull, X_BYTES);
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int kb = 0; kb < 2; ++kb)
          tma_load_2d(sx + p * (X_BYTES / 2) + kb * (X_BYTES / 4), &mapx, xfull, kb * 64, p * a.n_pad + A0 + k * TM);
      last_x = k;
      for (int j = 0; ok && j < U; ++j) {
        const int un = n + j;
        int s = (j >> 1) + s0;
        if (s >= a.n_stack) s -= a.n_stack;
        const int h = j & 1;
        const int bs = un % zc::NBZ;
        if (un >= zc::NBZ && !mbar_wait(&bzempty[bs], (uint32_t)((un / zc::NBZ) - 1) & 1, abort)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&bzfull[bs], UN * 4);
        bulk_load(sbz + bs * UN, a.b + (long)s * D + h * UN, UN * 4, &bzfull[bs]);
        last_bz[bs] = un / zc::NBZ;
        // the stack's chain tile, one 64-wide K block (all 128 features) per ring slot
        const int st = q % zc::NSZ;
        if (q >= zc::NSZ && !mbar_wait(&bempty[st], (uint32_t)((q / zc::NSZ) - 1) & 1, abort)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&bfull[st], TILE_BYTES);
        tma_load_2d(sb + st * TILE_BYTES, &mapf, &bfull[st], h * 64, s * D);
        last_b[st] = q / zc::NSZ;
        ++q;
      }
    }
    if (!ok) {
      record_device_error(a.err, DEV_TIMEOUT);
      *abort = 1;
    }
  } else if (warp == kEpiWarps + 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    constexpr uint32_t idf2 = idesc_f16(TM, 2 * UN);
    int q = 0, n = 0;
    bool ok = true;
    for (int k = 0; ok && k < n_tiles; ++k, n += U) {
      if (!mbar_wait(xfull, k & 1, abort)) {
        ok = false;
        break;
      }
      // one N = 128 product per stack (two units: adjacent accumulators)
      for (int j = 0; j < U; j += 2) {
        const int un = n + j;
        const int st0 = q % zc::NSZ, st1 = (q + 1) % zc::NSZ, db = un % NDB;
        if (!mbar_wait(&bfull[st0], (uint32_t)(q / zc::NSZ) & 1, abort) ||
            !mbar_wait(&bfull[st1], (uint32_t)((q + 1) / zc::NSZ) & 1, abort) ||
            (un >= NDB && !mbar_wait(&dempty[db], (uint32_t)((un / NDB) - 1) & 1, abort)) ||
            (un + 1 >= NDB && !mbar_wait(&dempty[db + 1], (uint32_t)(((un + 1) / NDB) - 1) & 1, abort))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t d = tmem + db * UN;
#pragma unroll
        for (int p = 1; p >= 0; --p)
#pragma unroll
          for (int kk = 0; kk < D / 16; ++kk) {
            const uint64_t da = smem_desc(sx + p * (X_BYTES / 2) + (kk >> 2) * (X_BYTES / 4)) + 2 * (kk & 3);
            const uint64_t dbd = smem_desc(sb + ((kk >> 2) ? st1 : st0) * TILE_BYTES) + 2 * (kk & 3);
            mma_bf16(d, da, dbd, idf2, (p == 1 && kk == 0) ? 0u : 1u);
          }
        mma_commit(&bempty[st0]);
        mma_commit(&bempty[st1]);
        mma_commit(&dfull[db]);
        mma_commit(&dfull[db + 1]);
        if (j == U - 2) mma_commit(xempty);
        q += 2;
      }
    }
    if (!ok) {
      record_device_error(a.err, DEV_TIMEOUT);
      *abort = 1;
    }
    mma_commit(mdone);
    mbar_wait(mdone, 0, never_abort);
  } else if (warp < kEpiWarps) {
    // ------------------------------------------------------------ epilogue
    const int quarter = warp & 3, cg = warp >> 2;
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    // reader role: feature column f of a unit, molecule slot
    const int t = warp * 32 + lane, f = t % UN, slot = t / UN;
    float* carry = a.carry + (long)blockIdx.x * NF;
    bool ok = true;
    auto fail = [&]() {
      if (lane == 0) {
        record_device_error(a.err, DEV_TIMEOUT);
        *abort = 1;
      }
      ok = false;
    };
    if (n_tiles == 0) {
      // molecules without atoms only: zero rows
      for (int m = M0; m < M1; ++m)
        for (int i = t; i < NF; i += kEpiWarps * 32) a.Z[(long)m * a.ldz + i] = 0.f;
    }
    // sum0 plus one molecule's rows [r0, r1) of column f of the cos tile, in row
    // order (a molecule carried across tiles is summed exactly as if in one)
    auto col_sum = [&](const float* cbuf, int r0, int r1, float sum0) {
      float sum = sum0;
      for (int r = r0; r < r1; ++r) sum += cbuf[r * zc::CLD + f];
      return sum;
    };
    // this thread's molecules of a tile (row bounds cached per tile): slot 0 the
    // first molecule (carried in or not), the last slot the one carried out,
    // the slots between the molecules that start and end in the tile, in turn
    // (more than two: bounds loaded when read)
    struct ZSlot {
      int m[2], r0[2], r1[2], cnt;
      bool more;
    };
    auto slot_of = [&](const ZTile& tt) {
      ZSlot z;
      z.cnt = 0;
      z.more = false;
      if (slot == 0) {
        z.m[0] = tt.mf;
        z.r0[0] = max(__ldg(a.mol_ptr + tt.mf), tt.a0) - tt.a0;
        z.r1[0] = min(__ldg(a.mol_ptr + tt.mf + 1), tt.a1) - tt.a0;
        z.cnt = 1;
      } else if (slot == zc::kSlots - 1) {
        if (tt.sout && tt.nm > 1) {
          z.m[0] = tt.mf + tt.nm - 1;
          z.r0[0] = __ldg(a.mol_ptr + z.m[0]) - tt.a0;
          z.r1[0] = tt.a1 - tt.a0;
          z.cnt = 1;
        }
      } else {
        const int n_own = tt.nm - (tt.sout && tt.nm > 1 ? 1 : 0);   // molecules ending in this tile
        for (int i = slot; i < n_own; i += zc::kSlots - 2) {
          if (z.cnt == 2) {
            z.more = true;
            break;
          }
          const int m = tt.mf + i;
          z.m[z.cnt] = m;
          z.r0[z.cnt] = __ldg(a.mol_ptr + m) - tt.a0;
          z.r1[z.cnt] = __ldg(a.mol_ptr + m + 1) - tt.a0;
          ++z.cnt;
        }
      }
      return z;
    };
    // feature index of a tile's unit j for this reader thread
    auto feat_of = [&](int j) {
      int st = (j >> 1) + s0;
      if (st >= a.n_stack) st -= a.n_stack;
      return st * D + (j & 1) * UN + f;
    };
    // the reader pass for unit un (local index j of a tile with info tt);
    // cin: the carried sum of the first molecule (prefetched), if tt.sin
    auto read_unit = [&](int un, int j, const ZTile& tt, const ZSlot& z, float cin) {
      const int cb = un & 1;
      const bool w = mbar_wait(&cfull[cb], (uint32_t)(un >> 1) & 1, abort);
      if (__any_sync(0xffffffffu, !w)) {
        fail();
        return;
      }
      const float* cbuf = sc + cb * (zc::C_BYTES / 4);
      const int fi = feat_of(j);
      if (slot == 0) {
        const float sum = col_sum(cbuf, z.r0[0], z.r1[0], tt.sin ? cin : 0.f);
        if (tt.nm == 1 && tt.sout) carry[fi] = sum;
        else a.Z[(long)z.m[0] * a.ldz + fi] = a.pref * sum;
      } else if (slot == zc::kSlots - 1) {
        // the molecule carried out: read back by slot 0 of this feature one tile
        // later (the mbarrier phases in between order the accesses)
        if (z.cnt == 1) carry[fi] = col_sum(cbuf, z.r0[0], z.r1[0], 0.f);
      } else {
        for (int c = 0; c < z.cnt; ++c) a.Z[(long)z.m[c] * a.ldz + fi] = a.pref * col_sum(cbuf, z.r0[c], z.r1[c], 0.f);
        if (z.more) {
          const int n_own = tt.nm - (tt.sout && tt.nm > 1 ? 1 : 0);
          for (int i = slot + 2 * (zc::kSlots - 2); i < n_own; i += zc::kSlots - 2) {
            const int m = tt.mf + i;
            const int r0 = __ldg(a.mol_ptr + m) - tt.a0, r1 = __ldg(a.mol_ptr + m + 1) - tt.a0;
            a.Z[(long)m * a.ldz + fi] = a.pref * col_sum(cbuf, r0, r1, 0.f);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&cempty[cb]);
    };
    int n = 0;
    ZTile prev{};
    ZSlot zprev{};
    for (int k = 0; ok && k < n_tiles; ++k, n += U) {
      const ZTile tt = z_tile(a.mol_ptr, a.n_mol, A0, A1, M0, M1, k, n_tiles);
      const ZSlot zs = slot_of(tt);
      const float cs = a.cscale * __ldg(a.kx + tt.a0 + row);   // a0 + row < n_pad
      for (int j = 0; j < U; ++j) {
        const int un = n + j;
        // the carried sum the reader of unit un - 1 needs, loaded ahead of the writer work
        const ZTile& tr = j > 0 ? tt : prev;
        const float cin = (un > 0 && slot == 0 && tr.sin) ? carry[feat_of(j > 0 ? j - 1 : U - 1)] : 0.f;
        const int db = un % NDB, bs = un % zc::NBZ, cb = un & 1;
        bool w = mbar_wait(&dfull[db], (uint32_t)(un / NDB) & 1, abort);
        if (__any_sync(0xffffffffu, !w)) {
          fail();
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        float v[CW];
        tmem_ldn(tmem + lane_base + db * UN + cg * CW, v);
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) mbar_arrive(&dempty[db]);
        w = mbar_wait(&bzfull[bs], (uint32_t)(un / zc::NBZ) & 1, abort);
        if (__any_sync(0xffffffffu, !w)) {
          fail();
          break;
        }
        const float4* b4 = reinterpret_cast<const float4*>(sbz + bs * UN + cg * CW);
#pragma unroll
        for (int c = 0; c < CW / 4; ++c) {
          const float4 bb = b4[c];
          v[4 * c] = fast_cos(fmaf(v[4 * c], cs, bb.x));
          v[4 * c + 1] = fast_cos(fmaf(v[4 * c + 1], cs, bb.y));
          v[4 * c + 2] = fast_cos(fmaf(v[4 * c + 2], cs, bb.z));
          v[4 * c + 3] = fast_cos(fmaf(v[4 * c + 3], cs, bb.w));
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&bzempty[bs]);
        if (un >= 2) {
          w = mbar_wait(&cempty[cb], (uint32_t)((un >> 1) - 1) & 1, abort);
          if (__any_sync(0xffffffffu, !w)) {
            fail();
            break;
          }
        }
        float4* crow = reinterpret_cast<float4*>(sc + cb * (zc::C_BYTES / 4) + row * zc::CLD + cg * CW);
#pragma unroll
        for (int c = 0; c < CW / 4; ++c) crow[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
        __syncwarp();
        if (lane == 0) mbar_arrive(&cfull[cb]);
        if (un > 0) {
          read_unit(un - 1, j > 0 ? j - 1 : U - 1, tr, j > 0 ? zs : zprev, cin);
          if (!ok) break;
        }
      }
      prev = tt;
      zprev = zs;
    }
    if (ok && n_tiles > 0) read_unit(n - 1, U - 1, prev, zprev, slot == 0 && prev.sin ? carry[feat_of(U - 1)] : 0.f);
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (*abort && warp == kEpiWarps && lane == 0) {
    if (last_x >= 0) mbar_wait(xfull, (uint32_t)last_x & 1, never_abort);
    for (int q = 0; q < zc::NSZ; ++q)
      if (last_b[q] >= 0) mbar_wait(&bfull[q], (uint32_t)last_b[q] & 1, never_abort);
    for (int q = 0; q < zc::NBZ; ++q)
      if (last_bz[q] >= 0) mbar_wait(&bzfull[q], (uint32_t)last_bz[q] & 1, never_abort);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(zc::TMEM_COLS));
  }
}

}  // namespace stc

size_t sorf_tc_table_bytes(int n_features) { return (size_t)2 * n_features * stc::D * sizeof(__half); }

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t sorf_tc_work_bytes(int n_atoms, int n_features) {
  const size_t n_pad = (size_t)((std::max(n_atoms, 1) + stc::TM - 1) / stc::TM) * stc::TM;
  return align256(2 * n_pad * stc::D * sizeof(__half)) + align256(n_pad * sizeof(float)) + 256 +
         align256((size_t)std::max(n_features, 1) * sizeof(float));
}

bool sorf_tc_supported(int d, int T, int n_features) {
  return d == stc::D && T >= 1 && T <= 3 && n_features >= d && n_features % d == 0;
}

int sorf_tc_tables(const uint32_t* sign_bits, int T, int n_features, void* tables, cudaStream_t s) {
  QMLR_REQUIRE(T >= 1 && T <= 3, "tensor-core SORF needs T in 1..3 (entries of the chain exact in FP16)");
  QMLR_REQUIRE(n_features >= stc::D && n_features % stc::D == 0, "n_features must be a multiple of 128");
  const int n_stack = n_features / stc::D;
  __half* mf = static_cast<__half*>(tables);
  __half* mb = mf + (size_t)n_features * stc::D;
  stc::chain_tables_kernel<<<n_stack, stc::D, 0, s>>>(sign_bits, T, mf, mb);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

// Per-atom energies (atom_e [n_atoms]) and gradients (gx [n_atoms][128]) of the
// SORF energy for tables built by sorf_tc_tables; work holds sorf_tc_work_bytes.
int sorf_tc_energy_grad(const float* x, int n_atoms, const void* tables, int T, const float* b,
                        const float* alpha, int n_features, double sigma, double* atom_e, float* gx, void* work,
                        size_t work_bytes, cudaStream_t s) {
  using namespace stc;
  QMLR_REQUIRE(n_atoms >= 0, "negative sizes");
  if (n_atoms == 0) return QMLR_OK;
  QMLR_REQUIRE(x && tables && b && alpha && atom_e && gx && work, "NULL pointer argument");
  QMLR_REQUIRE(work_bytes >= sorf_tc_work_bytes(n_atoms, n_features), "SORF workspace too small (%zu < %zu bytes)",
               work_bytes, sorf_tc_work_bytes(n_atoms, n_features));
  QMLR_REQUIRE((reinterpret_cast<uintptr_t>(x) & 15) == 0 && (reinterpret_cast<uintptr_t>(b) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(alpha) & 15) == 0 && (reinterpret_cast<uintptr_t>(gx) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(tables) & 15) == 0 && (reinterpret_cast<uintptr_t>(work) & 255) == 0,
               "x, b, alpha, gx, tables must be 16-byte and work 256-byte aligned");
  const int n_stack = n_features / D;
  const int n_tiles = (n_atoms + TM - 1) / TM, n_pad = n_tiles * TM;
  __half* xh = static_cast<__half*>(work);
  float* kx = reinterpret_cast<float*>(static_cast<uint8_t*>(work) + align256((size_t)2 * n_pad * D * sizeof(__half)));
  float* ys = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(kx) + align256((size_t)n_pad * sizeof(float)));
  float* alpha_sc = ys + 64;
  int* err = device_error_ptr();
  alpha_scale_kernel<<<1, 1024, 0, s>>>(alpha, n_features, ys, alpha_sc);
  QMLR_LAUNCH_CHECK();
  split_x_kernel<<<(n_pad + 7) / 8, 256, 0, s>>>(x, n_atoms, n_pad, sorf_x2max(D, sigma), xh, kx, err);
  QMLR_LAUNCH_CHECK();
  const __half* mf = static_cast<const __half*>(tables);
  const __half* mb = mf + (size_t)n_features * D;
  CUtensorMap mx, mapf, mapb;
  int rc;
  if ((rc = make_map(&mx, xh, D, 2L * n_pad, TM))) return rc;
  if ((rc = make_map(&mapf, mf, D, (long)n_stack * D, UN))) return rc;
  if ((rc = make_map(&mapb, mb, D, (long)n_stack * D, D))) return rc;
  Args a;
  a.kx = kx;
  a.b = b;
  a.alpha = alpha_sc;
  a.ys = ys;
  a.atom_e = atom_e;
  a.gx = gx;
  a.n_atoms = n_atoms;
  a.n_pad = n_pad;
  a.n_tiles = n_tiles;
  a.n_stack = n_stack;
  const int U = 2 * n_stack;
  a.period_log2 = U % 8 == 0 ? 3 : (U % 4 == 0 ? 2 : 1);
  a.cscale = (float)(sqrt((double)D) / sigma / pow((double)D, 0.5 * T));
  a.pref = (float)sqrt(2.0 / n_features);
  a.err = err;
  QMLR_CUDA_TRY(smem_attr_once((const void*)sorf_tc_kernel, SMEM_BYTES));
  const int grid = std::min(n_tiles, sm_count());
  sorf_tc_kernel<<<grid, kThreads, SMEM_BYTES, s>>>(mx, mapf, mapb, a);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

// Z rows [n_mol][ldz] of the SORF segment sums for tables built by
// sorf_tc_tables; work holds sorf_tc_z_work_bytes.
constexpr int kZMaxCtas = 256;

static size_t z_pad(int n_atoms) { return ((size_t)(std::max(n_atoms, 0) + stc::TM - 1) / stc::TM + 1) * stc::TM; }

size_t sorf_tc_z_work_bytes(int n_atoms, int n_features) {
  const size_t n_pad = z_pad(n_atoms);
  return align256(2 * n_pad * stc::D * sizeof(__half)) + align256(n_pad * sizeof(float)) +
         align256((size_t)kZMaxCtas * std::max(n_features, 1) * sizeof(float));
}

int sorf_tc_segment_sum(const float* x, int n_atoms, const int32_t* mol_ptr, int n_mol, const void* tables, int T,
                        const float* b, int n_features, double sigma, float* Z, long ldz, void* work,
                        size_t work_bytes, cudaStream_t s) {
  using namespace stc;
  QMLR_REQUIRE(n_atoms >= 0 && n_mol >= 0, "negative sizes");
  QMLR_REQUIRE(ldz >= n_features, "ldz must be >= n_features");
  if (n_mol == 0) return QMLR_OK;
  QMLR_REQUIRE(mol_ptr && Z, "NULL pointer argument");
  if (n_atoms == 0) {
    QMLR_CUDA_TRY(cudaMemset2DAsync(Z, (size_t)ldz * sizeof(float), 0, (size_t)n_features * sizeof(float),
                                    (size_t)n_mol, s));
    return QMLR_OK;
  }
  QMLR_REQUIRE(x && tables && b && work, "NULL pointer argument");
  QMLR_REQUIRE(work_bytes >= sorf_tc_z_work_bytes(n_atoms, n_features), "SORF workspace too small (%zu < %zu bytes)",
               work_bytes, sorf_tc_z_work_bytes(n_atoms, n_features));
  QMLR_REQUIRE((reinterpret_cast<uintptr_t>(x) & 15) == 0 && (reinterpret_cast<uintptr_t>(b) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(tables) & 15) == 0 && (reinterpret_cast<uintptr_t>(work) & 255) == 0,
               "x, b, tables must be 16-byte and work 256-byte aligned");
  const int n_stack = n_features / D;
  const int n_pad = (int)z_pad(n_atoms);
  __half* xh = static_cast<__half*>(work);
  float* kx = reinterpret_cast<float*>(static_cast<uint8_t*>(work) + align256((size_t)2 * n_pad * D * sizeof(__half)));
  float* carry = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(kx) + align256((size_t)n_pad * sizeof(float)));
  int* err = device_error_ptr();
  split_x_kernel<<<(n_pad + 7) / 8, 256, 0, s>>>(x, n_atoms, n_pad, sorf_x2max(D, sigma), xh, kx, err);
  QMLR_LAUNCH_CHECK();
  CUtensorMap mx, mapf;
  int rc;
  if ((rc = make_map(&mx, xh, D, 2L * n_pad, TM))) return rc;
  if ((rc = make_map(&mapf, tables, D, (long)n_stack * D, TM))) return rc;
  ZArgs a;
  a.kx = kx;
  a.b = b;
  a.mol_ptr = mol_ptr;
  a.Z = Z;
  a.ldz = ldz;
  a.carry = carry;
  a.n_atoms = n_atoms;
  a.n_mol = n_mol;
  a.n_pad = n_pad;
  a.n_stack = n_stack;
  a.cscale = (float)(sqrt((double)D) / sigma / pow((double)D, 0.5 * T));
  a.pref = (float)sqrt(2.0 / n_features);
  a.err = err;
  QMLR_CUDA_TRY(smem_attr_once((const void*)sorf_z_tc_kernel, zc::SMEM_BYTES));
  const int grid = std::max(1, std::min(std::min(sm_count(), kZMaxCtas), (n_atoms + 255) / 256));
  sorf_z_tc_kernel<<<grid, kThreads, zc::SMEM_BYTES, s>>>(mx, mapf, a);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

}  // namespace qmlr

using namespace qmlr;

extern "C" int64_t qmlr_sorf_tc_table_bytes(int32_t n_features) {
  return n_features > 0 ? (int64_t)sorf_tc_table_bytes(n_features) : 0;
}

extern "C" int64_t qmlr_sorf_tc_workspace_bytes(int32_t n_atoms, int32_t n_features) {
  return n_atoms >= 0 && n_features > 0 ? (int64_t)sorf_tc_work_bytes(n_atoms, n_features) : 0;
}

extern "C" int qmlr_sorf_tc_tables(const uint32_t* sign_bits, int32_t d, int32_t T, int32_t n_features,
                                   void* tables, void* stream) {
  QMLR_REQUIRE(sorf_tc_supported(d, T, n_features),
               "tensor-core SORF needs d = 128, T in 1..3 and n_features a multiple of 128 (got %d, %d, %d)", d,
               T, n_features);
  QMLR_REQUIRE(sign_bits && tables, "NULL pointer argument");
  QMLR_REQUIRE((reinterpret_cast<uintptr_t>(tables) & 15) == 0, "tables must be 16-byte aligned");
  return sorf_tc_tables(sign_bits, T, n_features, tables, as_stream(stream));
}

extern "C" int qmlr_sorf_grad_tc(const float* x, int32_t d, const int32_t* mol_ptr, int32_t n_mol,
                                 int32_t n_atoms, const void* tables, int32_t T, const float* b,
                                 int32_t n_features, double sigma, const float* alpha, double* atom_energy,
                                 double* energies, float* gx, void* work, int64_t work_bytes, void* stream) {
  QMLR_REQUIRE(sorf_tc_supported(d, T, n_features),
               "tensor-core SORF needs d = 128, T in 1..3 and n_features a multiple of 128 (got %d, %d, %d)", d,
               T, n_features);
  QMLR_REQUIRE(sigma > 0, "sigma must be > 0");
  QMLR_REQUIRE(n_mol >= 0 && n_atoms >= 0 && work_bytes >= 0, "negative sizes");
  if (n_mol == 0) return QMLR_OK;
  QMLR_REQUIRE(mol_ptr && energies && atom_energy, "NULL pointer argument");
  cudaStream_t s = as_stream(stream);
  int rc = sorf_tc_energy_grad(x, n_atoms, tables, T, b, alpha, n_features, sigma, atom_energy, gx, work,
                               (size_t)work_bytes, s);
  if (rc) return rc;
  return sorf_segment_energy(atom_energy, 1, n_atoms, mol_ptr, n_mol, energies, s);
}

extern "C" int64_t qmlr_sorf_tc_segment_workspace_bytes(int32_t n_atoms, int32_t n_features) {
  return n_atoms >= 0 && n_features > 0 ? (int64_t)sorf_tc_z_work_bytes(n_atoms, n_features) : 0;
}

extern "C" int qmlr_sorf_segment_sum_tc(const float* x, int32_t d, const int32_t* mol_ptr, int32_t n_mol,
                                        int32_t n_atoms, const void* tables, int32_t T, const float* b,
                                        int32_t n_features, double sigma, float* Z, int64_t ldz, void* work,
                                        int64_t work_bytes, void* stream) {
  QMLR_REQUIRE(sorf_tc_supported(d, T, n_features),
               "tensor-core SORF needs d = 128, T in 1..3 and n_features a multiple of 128 (got %d, %d, %d)", d,
               T, n_features);
  QMLR_REQUIRE(sigma > 0, "sigma must be > 0");
  QMLR_REQUIRE(work_bytes >= 0, "negative sizes");
  return sorf_tc_segment_sum(x, n_atoms, mol_ptr, n_mol, tables, T, b, n_features, sigma, Z, ldz, work,
                             (size_t)work_bytes, as_stream(stream));
}
