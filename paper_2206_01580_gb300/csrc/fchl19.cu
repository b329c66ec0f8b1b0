// FCHL19 representation: forward and vector-Jacobian product (sm_103a).
//
// Representation section of the paper: two-body log-normal radial terms with
// cutoff and r^-N2 decay; three-body terms = ATM weight x Gaussian radial in
// (r_ij + r_ik)/2 x Fourier angular [cos, sin] x three cutoffs.
//
// Design (GB300): one warp per centre atom. The warp builds its neighbour list
// from staged coordinates with a ballot / popc compaction (no HBM neighbour
// list); every sum has a fixed order (deterministic, no atomics).
// Forward (fchl19_forward_reg_kernel, up to 5 elements and 32-point grids):
// lane k owns radial bin k; two-body sums in registers element by element;
// three-body pairs are counting-sorted by element-pair type per block of up to
// 256 pairs (lane-parallel geometry), then each type's run is walked in pair
// order and its two columns stored. Larger parameter sets take
// fchl19_forward_kernel (shared-memory rows).
// VJP: lanes over neighbour pairs, each lane loops over its pair's radial
// bins (no per-pair warp reductions); the pair contributions reach the atoms'
// accumulators in a fixed order (segmented scans over lanes), summed per atom
// in a fixed order.
#include "common.cuh"

namespace qmlr {

constexpr int kMaxGrid = 64;     // n2, n3 <= 64
constexpr int kWarpsFwd = 4;
constexpr int kWarpsVjp = 4;

struct Fchl19Consts {
  int n_el, n2, n3, rep_dim, base3;
  float rcut, rcut2, pi_over_rcut, inv_rcut;
  float eta2, eta3, N2, N3;
  float w3;          // c3 * sqrt(eta3/pi)
  float ang2;        // 2 exp(-zeta^2/2): G^cos = ang2 cos(th), G^sin = ang2 sin(th) for n = 1
  float inv_sqrt_2pi;
  float sq_eta3;      // sqrt(eta3 log2(e)): three-body Gaussians as 2^-(y - y_k)^2, y = xbar sq_eta3
  float rs2_log[kMaxGrid], rs2_inv[kMaxGrid], rs3[kMaxGrid], ys3[kMaxGrid];
};

static Fchl19Consts make_consts(const qmlr_fchl19_params& p) {
  Fchl19Consts c{};
  c.n_el = p.n_el;
  c.n2 = p.n2;
  c.n3 = p.n3;
  c.rep_dim = rep_dim_of(p);
  c.base3 = p.n_el * p.n2;
  c.rcut = (float)p.rcut;
  c.rcut2 = (float)(p.rcut * p.rcut);
  c.pi_over_rcut = (float)(M_PI / p.rcut);
  c.inv_rcut = (float)(1.0 / p.rcut);
  c.eta2 = (float)p.eta2;
  c.eta3 = (float)p.eta3;
  c.N2 = (float)p.N2;
  c.N3 = (float)p.N3;
  c.w3 = (float)(p.c3 * sqrt(p.eta3 / M_PI));
  c.ang2 = (float)(2.0 * exp(-p.zeta * p.zeta / 2.0));
  c.inv_sqrt_2pi = (float)(1.0 / sqrt(2.0 * M_PI));
  for (int k = 0; k < p.n2; ++k) {
    double R = p.rcut * (k + 1) / p.n2;
    c.rs2_log[k] = (float)log(R);
    c.rs2_inv[k] = (float)(1.0 / R);
  }
  c.sq_eta3 = (float)sqrt(p.eta3 / log(2.0));
  for (int k = 0; k < p.n3; ++k) {
    c.rs3[k] = (float)(p.rcut * (k + 1) / p.n3);
    c.ys3[k] = (float)(p.rcut * (k + 1) / p.n3 * sqrt(p.eta3 / log(2.0)));
  }
  return c;
}

int validate_params(const qmlr_fchl19_params* p) {
  QMLR_REQUIRE(p != nullptr, "params is NULL");
  QMLR_REQUIRE(p->n_el >= 1 && p->n_el <= 8, "n_el must be in 1..8 (got %d)", p->n_el);
  QMLR_REQUIRE(p->n2 >= 1 && p->n2 <= kMaxGrid, "n2 must be in 1..64 (got %d)", p->n2);
  QMLR_REQUIRE(p->n3 >= 1 && p->n3 <= kMaxGrid, "n3 must be in 1..64 (got %d)", p->n3);
  QMLR_REQUIRE(p->nfourier == 1, "only nfourier = 1 is supported (got %d)", p->nfourier);
  QMLR_REQUIRE(p->rcut > 0 && p->eta2 > 0 && p->eta3 > 0, "rcut, eta2, eta3 must be > 0");
  return QMLR_OK;
}

__device__ __forceinline__ float cutoff_f(float r, const Fchl19Consts& c) {
  return r < c.rcut ? 0.5f * (cospif(r / c.rcut) + 1.0f) : 0.0f;
}
__device__ __forceinline__ float cutoff_df(float r, const Fchl19Consts& c) {
  return r < c.rcut ? -0.5f * c.pi_over_rcut * sinpif(r / c.rcut) : 0.0f;
}

__device__ __forceinline__ int pair_index(int a, int b, int n_el) {
  int lo = min(a, b), hi = max(a, b);
  return lo * n_el - lo * (lo - 1) / 2 + (hi - lo);
}

__device__ __forceinline__ int find_molecule(const int32_t* mol_ptr, int n_mol, int atom) {
  int lo = 0, hi = n_mol;  // mol_ptr[lo] <= atom < mol_ptr[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(mol_ptr + mid) <= atom) lo = mid; else hi = mid;
  }
  return lo;
}

// Decode a flat index q over the pairs (j < k) of n items.
__device__ __forceinline__ void decode_pair(int q, int n, int& j, int& k) {
  float t = (float)(2 * n - 1);
  int jj = (int)floorf((t - sqrtf(t * t - 8.0f * (float)q)) * 0.5f);
  jj = max(0, min(jj, n - 2));
  // fix rounding: first index of row jj is jj*(2n-jj-1)/2
  while (jj > 0 && jj * (2 * n - jj - 1) / 2 > q) --jj;
  while (jj < n - 2 && (jj + 1) * (2 * n - jj - 2) / 2 <= q) ++jj;
  j = jj;
  k = q - jj * (2 * n - jj - 1) / 2 + jj + 1;
}

// ---------------------------------------------------------------------------
// Shared-memory staging and neighbour lists.

// Positions of the molecule's atoms: pos[j] = (x, y, z, element bits).
__device__ void stage_molecule(const float* __restrict__ coords, const int32_t* __restrict__ elem,
                               int a0, int M, int n_el, float4* pos, int tid, int nthreads,
                               int* err) {
  for (int j = tid; j < M; j += nthreads) {
    int e = __ldg(elem + a0 + j);
    if (e < 0 || e >= n_el) {
      record_device_error(err, DEV_BAD_ELEMENT);
      e = 0;
    }
    pos[j] = make_float4(__ldg(coords + 3 * (a0 + j)), __ldg(coords + 3 * (a0 + j) + 1),
                         __ldg(coords + 3 * (a0 + j) + 2), __int_as_float(e));
  }
}

// Neighbour list of local atom il (ballot/popc compaction, ascending j).
//   nb_u[s]  = unit vector i->j and r_ij; nb_2b[s] = (mu, 1/(2 s^2), two-body prefactor, f_cut)
//   nb_el[s] = element of j; nb_idx[s] = local index j (nullable)
// Returns the neighbour count (warp-uniform).
__device__ int neighbour_list(const float4* pos, int M, int il, const Fchl19Consts& c,
                              float4* nb_u, float4* nb_2b, int* nb_el, int* nb_idx, int lane) {
  const float4 ri = pos[il];
  int n = 0;
  for (int base = 0; base < M; base += 32) {
    const int j = base + lane;
    bool ok = false;
    float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f, wj = 0.f;
    if (j < M && j != il) {
      const float4 pj = pos[j];
      dx = pj.x - ri.x;
      dy = pj.y - ri.y;
      dz = pj.z - ri.z;
      wj = pj.w;
      r2 = dx * dx + dy * dy + dz * dz;
      ok = r2 < c.rcut2;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, ok);
    if (ok) {
      const int slot = n + __popc(mask & ((1u << lane) - 1u));
      const float r = sqrtf(r2);
      const float inv = 1.0f / r;
      nb_u[slot] = make_float4(dx * inv, dy * inv, dz * inv, r);
      nb_el[slot] = __float_as_int(wj);
      if (nb_idx) nb_idx[slot] = j;
      const float fc = cutoff_f(r, c);
      const float s2 = log1pf(c.eta2 * inv * inv);   // sigma^2 = ln(1 + eta2 / r^2)
      const float s = sqrtf(s2);
      nb_2b[slot] = make_float4(logf(r) - 0.5f * s2,                       // mu = ln(r / sqrt(1 + eta2/r^2))
                                0.5f / s2,                                  // 1 / (2 s^2)
                                fc * expf(-c.N2 * logf(r)) * c.inv_sqrt_2pi / s,
                                fc);
    }
    n += __popc(mask);
  }
  __syncwarp();
  return n;
}

// Per-warp shared memory of the forward kernel (16-byte aligned pieces).
struct FwdWarp {
  float4* pos;    // [mxp]
  float4* nb_u;   // [mxp]
  float4* nb_2b;  // [mxp]
  float4* pairs;  // [32] w*G^cos, w*G^sin, xbar, bin offset (bits)
  float* acc;     // [rp]
  int* nb_el;     // [mxp]
};
__host__ __device__ __forceinline__ size_t fwd_warp_bytes(int mxp, int rp) {
  return (size_t)mxp * 52 + (size_t)rp * 4 + 512;
}
__device__ __forceinline__ FwdWarp carve_fwd(char* base, int mxp, int rp) {
  FwdWarp s;
  s.pos = reinterpret_cast<float4*>(base);
  s.nb_u = s.pos + mxp;
  s.nb_2b = s.nb_u + mxp;
  s.pairs = s.nb_2b + mxp;
  s.acc = reinterpret_cast<float*>(s.pairs + 32);
  s.nb_el = reinterpret_cast<int*>(s.acc + rp);
  return s;
}

__global__ void __launch_bounds__(32 * kWarpsFwd)
fchl19_forward_kernel(const float* __restrict__ coords, const int32_t* __restrict__ elem,
                      const int32_t* __restrict__ mol_ptr, int n_mol, int n_atoms, int mx,
                      int mxp, int rp, Fchl19Consts c, float* __restrict__ rep, int rep_ld,
                      int* err) {
  extern __shared__ __align__(16) char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int atom = blockIdx.x * kWarpsFwd + warp;
  if (atom >= n_atoms) return;
  FwdWarp s = carve_fwd(smem_raw + warp * fwd_warp_bytes(mxp, rp), mxp, rp);

  const int m = find_molecule(mol_ptr, n_mol, atom);
  const int a0 = __ldg(mol_ptr + m);
  const int M = __ldg(mol_ptr + m + 1) - a0;
  float* out = rep + (size_t)atom * rep_ld;
  if (M > mx) {
    if (lane == 0) record_device_error(err, DEV_MOL_TOO_LARGE);
    for (int k = lane; k < rep_ld; k += 32) out[k] = 0.0f;
    return;
  }
  for (int k = lane; k < rp; k += 32) s.acc[k] = 0.0f;
  stage_molecule(coords, elem, a0, M, c.n_el, s.pos, lane, 32, err);
  __syncwarp();
  const int n = neighbour_list(s.pos, M, atom - a0, c, s.nb_u, s.nb_2b, s.nb_el, nullptr, lane);

  // two-body: lanes over radial bins, neighbours in order
  for (int jn = 0; jn < n; ++jn) {
    const float4 t = s.nb_2b[jn];
    float* dst = s.acc + s.nb_el[jn] * c.n2;
    for (int k = lane; k < c.n2; k += 32) {
      const float a = c.rs2_log[k] - t.x;
      dst[k] += t.z * c.rs2_inv[k] * expf(-a * a * t.y);
    }
  }
  __syncwarp();

  // three-body: pair geometry lane-parallel over flat pairs (j < k), then lanes over bins
  const int n_pairs = n * (n - 1) / 2;
  for (int q0 = 0; q0 < n_pairs; q0 += 32) {
    const int q = q0 + lane;
    bool ok = false;
    float wc = 0.f, ws = 0.f, xbar = 0.f;
    int bin = 0;
    if (q < n_pairs) {
      int jn, kn;
      decode_pair(q, n, jn, kn);
      const float4 uj = s.nb_u[jn], uk = s.nb_u[kn];
      const float vx = uk.x * uk.w - uj.x * uj.w;
      const float vy = uk.y * uk.w - uj.y * uj.w;
      const float vz = uk.z * uk.w - uj.z * uj.w;
      const float rjk2 = vx * vx + vy * vy + vz * vz;
      if (rjk2 < c.rcut2) {
        ok = true;
        const float rjk = sqrtf(rjk2);
        const float inv_rjk = 1.0f / rjk;
        const float ci = uj.x * uk.x + uj.y * uk.y + uj.z * uk.z;
        const float cx = uj.y * uk.z - uj.z * uk.y;
        const float cy = uj.z * uk.x - uj.x * uk.z;
        const float cz = uj.x * uk.y - uj.y * uk.x;
        const float si = sqrtf(cx * cx + cy * cy + cz * cz);
        const float cj = -(uj.x * vx + uj.y * vy + uj.z * vz) * inv_rjk;
        const float ck = (uk.x * vx + uk.y * vy + uk.z * vz) * inv_rjk;
        const float atm = (1.0f + 3.0f * ci * cj * ck) * expf(-c.N3 * logf(uj.w * uk.w * rjk));
        const float w = c.w3 * atm * s.nb_2b[jn].w * s.nb_2b[kn].w * cutoff_f(rjk, c);
        wc = w * c.ang2 * ci;
        ws = w * c.ang2 * si;
        xbar = 0.5f * (uj.w + uk.w);
        bin = c.base3 + pair_index(s.nb_el[jn], s.nb_el[kn], c.n_el) * c.n3 * 2;
      }
    }
    const unsigned mask = __ballot_sync(0xffffffffu, ok);
    if (ok) s.pairs[__popc(mask & ((1u << lane) - 1u))] = make_float4(wc, ws, xbar, __int_as_float(bin));
    __syncwarp();
    const int cnt = __popc(mask);
    for (int t = 0; t < cnt; ++t) {
      const float4 pr = s.pairs[t];
      float* dst = s.acc + __float_as_int(pr.w);
      for (int k = lane; k < c.n3; k += 32) {
        const float a = pr.z - c.rs3[k];
        const float g = expf(-c.eta3 * a * a);
        dst[2 * k] += g * pr.x;
        dst[2 * k + 1] += g * pr.y;
      }
    }
    __syncwarp();
  }
  for (int k = lane; k < rep_ld; k += 32) out[k] = k < c.rep_dim ? s.acc[k] : 0.0f;
}

// Register-accumulating forward for up to 5 elements (15 element pairs) and
// radial grids of at most 32 points: lane k owns radial bin k of every element
// (two-body) and of every element pair (three-body, cos and sin), so the
// accumulation is a warp-uniform switch on the element or pair index into
// registers instead of a shared-memory read-modify-write; the row is written
// straight from registers at the end.
//
// Work layout: a CTA takes a contiguous range of `range` atoms (32 for large
// batches, 4 - one atom per warp - for small ones, where the range would
// otherwise leave most SMs idle and serialise the atoms of a molecule); thread 0
// finds the molecules at its two ends (two binary searches per CTA instead of
// one per atom), the CTA stages the positions of every molecule the range
// touches once, and each warp takes every kWarpsFwd-th atom of the range. The
// Gaussians of the radial grids are evaluated as 2^(-c t^2) with the
// hardware base-2 exponential (the constants carry the log2(e) factor), one
// special-function instruction per (neighbour or triplet, bin); the per-pair
// geometry uses the hardware cosine for the third cutoff factor and base-2
// log / exponential for the ATM power. Summation order per bin: neighbours,
// then triplets, in the same order as the shared-memory kernel.
constexpr int kFwdRange = 32;          // atoms per CTA for large batches
constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Per-warp shared memory of the register kernel: neighbour data and one block
// of triplets, sorted by element-pair type.
constexpr int kPairBlock = 256;   // neighbour pairs staged per walk (8 sweeps of 32 lanes)
struct RegWarp {
  float4* nb_u;   // [mxp] unit vector i->j, r_ij
  float4* nb_2b;  // [mxp] mu, log2(e)/(2 s^2), two-body prefactor, f_cut(r_ij)
  float4* pairs;  // [kPairBlock] w G^cos, w G^sin, xbar sqrt(eta3 log2 e), 0 (the block's triplets, by type)
  int* run;       // [16] first entry of each type's run in `pairs` (entry 15: end of type 14)
  int* nb_el;     // [mxp]
};
__host__ __device__ __forceinline__ size_t reg_warp_bytes(int mxp) {
  return (size_t)mxp * 36 + (size_t)kPairBlock * 16 + 64;
}
__device__ __forceinline__ RegWarp carve_reg(char* base, int mxp) {
  RegWarp s;
  s.nb_u = reinterpret_cast<float4*>(base);
  s.nb_2b = s.nb_u + mxp;
  s.pairs = s.nb_2b + mxp;
  s.run = reinterpret_cast<int*>(s.pairs + kPairBlock);
  s.nb_el = s.run + 16;
  return s;
}
__host__ __device__ __forceinline__ int reg_stage_atoms(int mx, int range) { return range + 2 * (mx - 1); }


// Per-lane constants of the register forward (lane = radial bin).
struct BinConsts {
  bool has2, has3;
  float r2log, r2inv, y3;   // y3 = R_k sqrt(eta3 log2 e) of this lane's bin
  int np;
};
__device__ __forceinline__ BinConsts bin_consts(const Fchl19Consts& c, int lane) {
  BinConsts k;
  k.has2 = lane < c.n2;
  k.has3 = lane < c.n3;
  k.r2log = k.has2 ? c.rs2_log[lane] : 0.f;
  k.r2inv = k.has2 ? c.rs2_inv[lane] : 0.f;
  k.y3 = k.has3 ? c.ys3[lane] : 0.f;
  k.np = c.n_el * (c.n_el + 1) / 2;
  return k;
}

// One neighbour of the register forward at `slot`: displacement (dx, dy, dz)
// from the centre, r2 = its squared length (0 < r2 < rcut^2), element e.
__device__ __forceinline__ void store_neighbour(const RegWarp& s, int slot, float dx, float dy, float dz, float r2,
                                                int e, const Fchl19Consts& c) {
  const float inv = rsqrt_approx(r2);
  const float r = r2 * inv;
  s.nb_u[slot] = make_float4(dx * inv, dy * inv, dz * inv, r);
  s.nb_el[slot] = e;
  const float fc = 0.5f * (cospif(r * c.inv_rcut) + 1.0f);   // r < rcut
  const float s2 = log1pf(c.eta2 * inv * inv);   // sigma^2 = ln(1 + eta2 / r^2)
  const float lr = logf(r);
  s.nb_2b[slot] = make_float4(lr - 0.5f * s2,                              // mu = ln(r / sqrt(1 + eta2/r^2))
                              kLog2e * 0.5f / s2,                          // log2(e) / (2 sigma^2)
                              fc * ex2_approx(-c.N2 * kLog2e * lr) * c.inv_sqrt_2pi * rsqrtf(s2),
                              fc);
}

// Flat index q over the pairs (j < k) of n items, row-major: the row from an
// approximate square root, then one correction step each way.
__device__ __forceinline__ void decode_pair_fast(int q, int n, int& j, int& k) {
  const float t = (float)(2 * n - 1);
  float sq;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sq) : "f"(fmaf(t, t, -8.0f * (float)q)));
  int jj = max(0, min((int)((t - sq) * 0.5f), n - 2));
  if (jj * (2 * n - jj - 1) / 2 > q) --jj;
  else if ((jj + 1) * (2 * n - jj - 2) / 2 <= q) ++jj;
  j = jj;
  k = q - jj * (2 * n - jj - 1) / 2 + jj + 1;
}

// Lanes whose 4-bit type equals t, from the ballots b0..b3 of the types' bits.
__device__ __forceinline__ unsigned type_lanes(int t, unsigned b0, unsigned b1, unsigned b2, unsigned b3) {
  return ((t & 1) ? b0 : ~b0) & ((t & 2) ? b1 : ~b1) & ((t & 4) ? b2 : ~b2) & ((t & 8) ? b3 : ~b3);
}

// The representation row of a centre from its n staged neighbours (one warp);
// columns rep_dim..rep_ld-1 are written as zeros.
__device__ __forceinline__ void fwd_row(const RegWarp& s, int n, const Fchl19Consts& c, const BinConsts& kb,
                                        float* __restrict__ out, int rep_ld, int lane) {
  const bool has2 = kb.has2, has3 = kb.has3;
  const float r2log = kb.r2log, r2inv = kb.r2inv, y3 = kb.y3;
  const int np = kb.np;
  // two-body: lanes over bins; per block of 32 neighbours, element by element
  // (a compile-time accumulator index), neighbours in order
  float a2[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int ej = j0 + lane < n ? s.nb_el[j0 + lane] : -1;
#pragma unroll
    for (int e = 0; e < 5; ++e) {
      unsigned m = __ballot_sync(0xffffffffu, ej == e);
      while (m) {
        const int jn = j0 + __ffs(m) - 1;
        m &= m - 1u;
        const float4 t = s.nb_2b[jn];
        const float d = r2log - t.x;
        a2[e] = fmaf(t.z * r2inv, ex2_approx(-(d * d) * t.y), a2[e]);
      }
    }
  }

  if (has2)   // two-body columns (written before the three-body sums take the registers)
#pragma unroll
    for (int e = 0; e < 5; ++e)
      if (e < c.n_el) out[e * c.n2 + lane] = a2[e];

  // three-body, per block of up to kPairBlock neighbour pairs (j < k, row-major):
  //  1. lanes over pairs: each pair's element-pair type (15: no term, r_jk >= r_cut),
  //     4 bits per 32-lane sweep in `keys`, and the count of each type (lane t counts type t);
  //  2. lanes over pairs: the pair geometry, written to its type's run in pair
  //     order (rank among the sweep's lanes of the same type from four bit ballots);
  //  3. lanes over bins: type by type, the run in pair order with four
  //     Gaussians in flight; each type's (cos, sin) sums are stored at the end
  //     of its run.
  // Every type's triplets are summed in pair order within a block; a block's
  // sums are added to the earlier blocks' in the row (one block in most rows).
  const unsigned lt_mask = (1u << lane) - 1u;
  const int n_pairs = n * (n - 1) / 2;
  for (int p0 = 0; p0 == 0 || p0 < n_pairs; p0 += kPairBlock) {   // one (empty) block when n_pairs = 0
    const int p1 = min(p0 + kPairBlock, n_pairs);
    unsigned keys = 0u;
    int cnt = 0;
    for (int r = 0, q0 = p0; q0 < p1; ++r, q0 += 32) {
      const int q = q0 + lane;
      int key = 15;
      if (q < p1) {
        int jn, kn;
        decode_pair_fast(q, n, jn, kn);
        const float4 uj = s.nb_u[jn], uk = s.nb_u[kn];
        const float vx = uk.x * uk.w - uj.x * uj.w;
        const float vy = uk.y * uk.w - uj.y * uj.w;
        const float vz = uk.z * uk.w - uj.z * uj.w;
        if (vx * vx + vy * vy + vz * vz < c.rcut2) key = pair_index(s.nb_el[jn], s.nb_el[kn], c.n_el);
      }
      keys |= (unsigned)key << (4 * r);
      const unsigned b0 = __ballot_sync(0xffffffffu, key & 1), b1 = __ballot_sync(0xffffffffu, key & 2);
      const unsigned b2 = __ballot_sync(0xffffffffu, key & 4), b3 = __ballot_sync(0xffffffffu, key & 8);
      cnt += __popc(type_lanes(lane, b0, b1, b2, b3));
    }
    // exclusive scan of the counts over lanes 0..15: each type's first entry
    if (lane >= 16) cnt = 0;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    int run = incl - cnt;
    if (lane < 16) s.run[lane] = run;
    for (int r = 0, q0 = p0; q0 < p1; ++r, q0 += 32) {
      const int q = q0 + lane;
      const int key = (int)((keys >> (4 * r)) & 15u);
      const unsigned b0 = __ballot_sync(0xffffffffu, key & 1), b1 = __ballot_sync(0xffffffffu, key & 2);
      const unsigned b2 = __ballot_sync(0xffffffffu, key & 4), b3 = __ballot_sync(0xffffffffu, key & 8);
      const int slot = __shfl_sync(0xffffffffu, run, key) + __popc(type_lanes(key, b0, b1, b2, b3) & lt_mask);
      run += __popc(type_lanes(lane, b0, b1, b2, b3));
      if (key < 15) {   // q < p1 and r_jk < r_cut
        int jn, kn;
        decode_pair_fast(q, n, jn, kn);
        const float4 uj = s.nb_u[jn], uk = s.nb_u[kn];
        const float vx = uk.x * uk.w - uj.x * uj.w;
        const float vy = uk.y * uk.w - uj.y * uj.w;
        const float vz = uk.z * uk.w - uj.z * uj.w;
        const float rjk2 = vx * vx + vy * vy + vz * vz;
        const float inv_rjk = rsqrtf(rjk2);
        const float rjk = rjk2 * inv_rjk;
        const float ci = uj.x * uk.x + uj.y * uk.y + uj.z * uk.z;
        const float cx = uj.y * uk.z - uj.z * uk.y;
        const float cy = uj.z * uk.x - uj.x * uk.z;
        const float cz = uj.x * uk.y - uj.y * uk.x;
        const float s2i = cx * cx + cy * cy + cz * cz;
        const float si = s2i > 0.0f ? s2i * rsqrt_approx(s2i) : 0.0f;
        const float cj = -(uj.x * vx + uj.y * vy + uj.z * vz) * inv_rjk;
        const float ck = (uk.x * vx + uk.y * vy + uk.z * vz) * inv_rjk;
        // (r_ij r_ik r_jk)^-N3 = 2^(-N3 log2(r_ij r_ik r_jk))
        const float atm = (1.0f + 3.0f * ci * cj * ck) * ex2_approx(-c.N3 * lg2_approx(uj.w * uk.w * rjk));
        const float fcjk = 0.5f * (__cosf(rjk * c.pi_over_rcut) + 1.0f);
        const float w = c.w3 * atm * s.nb_2b[jn].w * s.nb_2b[kn].w * fcjk;
        s.pairs[slot] = make_float4(w * c.ang2 * ci, w * c.ang2 * si, 0.5f * (uj.w + uk.w) * c.sq_eta3, 0.f);
      }
    }
    __syncwarp();
    // one copy of the walk for all types (the sums are two scalars per type, so
    // nothing needs a compile-time index; a small body stays in the instruction cache)
    int lo = s.run[0];
#pragma unroll 1
    for (int b = 0; b < 15; ++b) {
      const int hi = s.run[b + 1];
      int t = lo;
      lo = hi;
      float ac = 0.f, as = 0.f;
      for (; t + 3 < hi; t += 4) {   // four triplets' Gaussians in flight, summed in order
        float g[4];
        float4 e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          e[u] = s.pairs[t + u];
          const float d = e[u].z - y3;
          g[u] = ex2_approx(-(d * d));
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          ac = fmaf(g[u], e[u].x, ac);
          as = fmaf(g[u], e[u].y, as);
        }
      }
      for (; t < hi; ++t) {
        const float4 e0 = s.pairs[t];
        const float d0 = e0.z - y3;
        const float g0 = ex2_approx(-(d0 * d0));
        ac = fmaf(g0, e0.x, ac);
        as = fmaf(g0, e0.y, as);
      }
      if (has3 && b < np) {   // the type's two columns at this lane's bin
        float* o = out + c.base3 + (b * c.n3 + lane) * 2;
        if (p0 > 0) {
          ac += o[0];
          as += o[1];
        }
        o[0] = ac;
        o[1] = as;
      }
    }
    __syncwarp();
  }
  for (int k = c.rep_dim + lane; k < rep_ld; k += 32) out[k] = 0.0f;   // padding columns
}

#ifndef QMLR_FWD_MIN_BLOCKS
#define QMLR_FWD_MIN_BLOCKS 8   // resident CTAs per SM the register budget is sized for (64 registers)
#endif
__global__ void __launch_bounds__(32 * kWarpsFwd, QMLR_FWD_MIN_BLOCKS)
fchl19_forward_reg_kernel(const float* __restrict__ coords, const int32_t* __restrict__ elem,
                          const int32_t* __restrict__ mol_ptr, int n_mol, int n_atoms, int mx, int mxp, int range,
                          Fchl19Consts c, float* __restrict__ rep, int rep_ld, int* err) {
  extern __shared__ __align__(16) char smem_raw[];
  __shared__ int s_m0, s_m1, s_base, s_end;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a_lo = blockIdx.x * range;
  const int a_hi = min(a_lo + range, n_atoms) - 1;
  if (threadIdx.x == 0) {
    const int m0 = find_molecule(mol_ptr, n_mol, a_lo);
    const int m1 = find_molecule(mol_ptr, n_mol, a_hi);
    s_m0 = m0;
    s_m1 = m1;
    // every atom of a molecule of at most mx atoms that owns an atom of the
    // range lies in [a_lo - (mx - 1), a_hi + mx): the staged window
    s_base = max(__ldg(mol_ptr + m0), a_lo - (mx - 1));
    s_end = min(__ldg(mol_ptr + m1 + 1), a_hi + mx);
  }
  __syncthreads();
  const int m0 = s_m0, m1 = s_m1, base = s_base;
  const int stage_n = s_end - base;   // <= range + 2 (mx - 1)
  float4* pos = reinterpret_cast<float4*>(smem_raw);
  for (int j = threadIdx.x; j < stage_n; j += blockDim.x) {
    int e = __ldg(elem + base + j);
    if (e < 0 || e >= c.n_el) {
      record_device_error(err, DEV_BAD_ELEMENT);
      e = 0;
    }
    const float* q = coords + 3 * (size_t)(base + j);
    pos[j] = make_float4(__ldg(q), __ldg(q + 1), __ldg(q + 2), __int_as_float(e));
  }
  __syncthreads();
  const RegWarp s = carve_reg(smem_raw + (size_t)reg_stage_atoms(mx, range) * 16 + warp * reg_warp_bytes(mxp), mxp);

  const BinConsts kb = bin_consts(c, lane);   // per-lane radial constants (lane = bin)

  for (int atom = a_lo + warp; atom <= a_hi; atom += kWarpsFwd) {
    // molecule of this atom: mol_ptr[mi] <= atom < mol_ptr[mi + 1], mi in [m0, m1]
    int lo = m0, hi = m1 + 1;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(mol_ptr + mid) <= atom) lo = mid; else hi = mid;
    }
    const int a0 = __ldg(mol_ptr + lo), M = __ldg(mol_ptr + lo + 1) - a0;
    float* out = rep + (size_t)atom * rep_ld;
    if (M > mx) {
      if (lane == 0) record_device_error(err, DEV_MOL_TOO_LARGE);
      for (int k = lane; k < rep_ld; k += 32) out[k] = 0.0f;
      continue;
    }
    const float4* mpos = pos + (a0 - base);
    const float4 ri = mpos[atom - a0];
    // neighbour list (ballot compaction, ascending j)
    int n = 0;
    for (int b0 = 0; b0 < M; b0 += 32) {
      const int j = b0 + lane;
      bool ok = false;
      float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f, wj = 0.f;
      if (j < M && j != atom - a0) {
        const float4 pj = mpos[j];
        dx = pj.x - ri.x;
        dy = pj.y - ri.y;
        dz = pj.z - ri.z;
        wj = pj.w;
        r2 = dx * dx + dy * dy + dz * dz;
        ok = r2 < c.rcut2;
      }
      const unsigned mask = __ballot_sync(0xffffffffu, ok);
      if (ok) store_neighbour(s, n + __popc(mask & ((1u << lane) - 1u)), dx, dy, dz, r2, __float_as_int(wj), c);
      n += __popc(mask);
    }
    __syncwarp();

    fwd_row(s, n, c, kb, out, rep_ld, lane);
    __syncwarp();
  }
}
// ---------------------------------------------------------------------------
// VJP: one CTA per molecule, warps over centre atoms.

struct VjpWarp {
  float4* stage;  // [64] one chunk of pair contributions (atom index bits, gradient)
  float4* nb_u;   // [mxp]
  float4* nb_2b;  // [mxp]
  float* g;       // [rp]   gradient row of the centre
  float* facc;    // [3 mxp] gradient with respect to the molecule's positions
  int* nb_el;     // [mxp]
  int* nb_idx;    // [mxp]
};
__host__ __device__ __forceinline__ size_t vjp_warp_bytes(int mxp, int rp) {
  return 64 * 16 + (size_t)mxp * (16 + 16 + 12 + 4 + 4) + (size_t)(rp + 4) * 4;
}

// The centre's gradient row in the warp's buffer, the three-body columns moved
// up by one float when they start at an odd column so that each (cos, sin)
// pair is one 8-byte load (grad3() points at them).
__device__ __forceinline__ void load_grad_row(float* g, const float* __restrict__ grow, const Fchl19Consts& c,
                                              int lane) {
  const int sh = c.base3 & 1;
  for (int k = lane; k < c.rep_dim; k += 32) g[k + (k >= c.base3 ? sh : 0)] = __ldg(grow + k);
}
__device__ __forceinline__ const float2* grad3(const float* g, const Fchl19Consts& c) {
  return reinterpret_cast<const float2*>(g + c.base3 + (c.base3 & 1));
}
__device__ __forceinline__ VjpWarp carve_vjp(char* base, int mxp, int rp) {
  VjpWarp s;
  s.stage = reinterpret_cast<float4*>(base);
  s.nb_u = s.stage + 64;
  s.nb_2b = s.nb_u + mxp;
  s.g = reinterpret_cast<float*>(s.nb_2b + mxp);
  s.facc = s.g + rp + 4;
  s.nb_el = reinterpret_cast<int*>(s.facc + 3 * mxp);
  s.nb_idx = s.nb_el + mxp;
  return s;
}

// Adjoint of one centre: accumulates d(sum_b g_b rho_il,b)/d r_k into facc[3k..3k+2]
// for every atom k of the molecule (the centre's own entry included). One warp.
// Gaussians as 2^(-c t^2) with the hardware base-2 exponential.
//
// Three-body contributions are computed lane-parallel over flat neighbour
// pairs (j < k, row-major), 32 at a time, and reach the atoms' accumulators in
// a fixed order without atomics: the j-side values of a chunk share their row
// index j along contiguous lanes, so a segmented scan over lanes (keyed by j)
// sums each row's run and the run's last lane adds it; the k-side values of one
// row name distinct atoms, so the rows of the chunk add theirs one row at a time.
// The body of the adjoint for n staged neighbours (nb_u, nb_2b in the
// neighbour_list format, nb_el, nb_idx naming each neighbour's accumulator) and
// the centre's gradient row in s.g; the centre's own gradient goes to
// accumulator il.
__device__ void vjp_from_neighbours(int n, int il, const Fchl19Consts& c, VjpWarp& s, int lane);

__device__ void vjp_centre(const float4* pos, int M, int il, const Fchl19Consts& c, const float* __restrict__ grow,
                           VjpWarp& s, int lane) {
  load_grad_row(s.g, grow, c, lane);
  const int n = neighbour_list(pos, M, il, c, s.nb_u, s.nb_2b, s.nb_el, s.nb_idx, lane);
  vjp_from_neighbours(n, il, c, s, lane);
}

__device__ void vjp_from_neighbours(int n, int il, const Fchl19Consts& c, VjpWarp& s, int lane) {
  float gi_x = 0.f, gi_y = 0.f, gi_z = 0.f;   // gradient on the centre (per-lane partials)

  // two-body: lanes over neighbours (distinct atoms per lane); reciprocals
  // and the cutoff's sine from the hardware approximations (a few ulp)
  for (int jn = lane; jn < n; jn += 32) {
    const float4 u = s.nb_u[jn];
    const float r = u.w;
    const float4 t = s.nb_2b[jn];   // mu, 1/(2s^2), fc r^-N2/(s sqrt(2pi)), fc
    const float inv_r = rcp_approx(r);
    const float inv_s2 = 2.0f * t.y;                           // 1 / sigma^2
    const float inv_sd = inv_s2 * rsqrt_approx(inv_s2);        // 1 / sigma
    const float inv_rr = rcp_approx(fmaf(r, r, c.eta2));       // 1 / (r^2 + eta2)
    const float ds = -c.eta2 * inv_sd * inv_r * inv_rr;        // d sigma / dr
    const float dmu = inv_r + c.eta2 * inv_r * inv_rr;         // d mu / dr
    const float fc = t.w;
    const float dfc = -0.5f * c.pi_over_rcut * __sinf(r * c.pi_over_rcut);
    const float rN = ex2_approx(-c.N2 * lg2_approx(r));
    const float P = fc * rN;
    const float dP = rN * (dfc - c.N2 * fc * inv_r);
    const float negc = -t.y * kLog2e;
    const float pre = c.inv_sqrt_2pi * inv_sd;
    const float k1 = -ds * inv_sd, k2 = dmu * inv_s2, k3 = ds * inv_s2 * inv_sd;
    const float* gb = s.g + s.nb_el[jn] * c.n2;
    // dE/dr = sum_k g_k L_k (dP + P dlnL_k), dlnL_k = k1 + a_k k2 + a_k^2 k3, with
    // L_k = pre e_k: the sums of g_k e_k a_k^p (p = 0, 1, 2) over the bins, then combined
    float S0 = 0.f, S1 = 0.f, S2 = 0.f;
    for (int k = 0; k < c.n2; ++k) {
      const float a = c.rs2_log[k] - t.x;
      const float ge = gb[k] * (c.rs2_inv[k] * ex2_approx(a * (a * negc)));
      const float gea = ge * a;
      S0 += ge;
      S1 += gea;
      S2 = fmaf(gea, a, S2);
    }
    const float dEdr = pre * (dP * S0 + P * (k1 * S0 + k2 * S1 + k3 * S2));
    const int jl = s.nb_idx[jn];
    s.facc[3 * jl + 0] += dEdr * u.x;
    s.facc[3 * jl + 1] += dEdr * u.y;
    s.facc[3 * jl + 2] += dEdr * u.z;
    gi_x -= dEdr * u.x;
    gi_y -= dEdr * u.y;
    gi_z -= dEdr * u.z;
  }
  __syncwarp();

  // three-body
  const int n_pairs = n * (n - 1) / 2;
  for (int q0 = 0; q0 < n_pairs; q0 += 32) {
    const int q = q0 + lane;
    float gj0 = 0.f, gj1 = 0.f, gj2 = 0.f, gk0 = 0.f, gk1 = 0.f, gk2 = 0.f;
    int jn = n, kn = n;   // lanes past the last pair: key n (no atom)
    if (q < n_pairs) {
      decode_pair(q, n, jn, kn);
      const float4 uj = s.nb_u[jn], uk = s.nb_u[kn];
      const float a = uj.w, b = uk.w;
      const float vx = uk.x * b - uj.x * a, vy = uk.y * b - uj.y * a, vz = uk.z * b - uj.z * a;
      const float c2 = vx * vx + vy * vy + vz * vz;
      if (c2 < c.rcut2) {
        // reciprocals, square roots, the ATM power and the cutoffs from the
        // hardware approximations (a few ulp; the gradient's tolerance is 1e-4)
        const float inv_c = rsqrt_approx(c2);
        const float cc = c2 * inv_c;
        const float inv_a = rcp_approx(a), inv_b = rcp_approx(b);
        const float ux = vx * inv_c, uy = vy * inv_c, uz = vz * inv_c;   // unit j -> k
        const float ci = uj.x * uk.x + uj.y * uk.y + uj.z * uk.z;
        const float crx = uj.y * uk.z - uj.z * uk.y;
        const float cry = uj.z * uk.x - uj.x * uk.z;
        const float crz = uj.x * uk.y - uj.y * uk.x;
        const float s2i = crx * crx + cry * cry + crz * crz;
        const float si = s2i > 0.0f ? s2i * rsqrt_approx(s2i) : 0.0f;
        const float cj = -(uj.x * ux + uj.y * uy + uj.z * uz);
        const float ck = (uk.x * ux + uk.y * uy + uk.z * uz);
        // cosines as functions of the sides a = r_ij, b = r_ik, cc = r_jk
        const float iab = inv_a * inv_b, iac = inv_a * inv_c, ibc = inv_b * inv_c;
        const float dci_da = (a - b * ci) * iab, dci_db = (b - a * ci) * iab, dci_dc = -cc * iab;
        const float dcj_da = (a - cc * cj) * iac, dcj_dc = (cc - a * cj) * iac, dcj_db = -b * iac;
        const float dck_db = (b - cc * ck) * ibc, dck_dc = (cc - b * ck) * ibc, dck_da = -a * ibc;
        const float Q = 1.0f + 3.0f * ci * cj * ck;
        const float dQ_da = 3.0f * (dci_da * cj * ck + ci * dcj_da * ck + ci * cj * dck_da);
        const float dQ_db = 3.0f * (dci_db * cj * ck + ci * dcj_db * ck + ci * cj * dck_db);
        const float dQ_dc = 3.0f * (dci_dc * cj * ck + ci * dcj_dc * ck + ci * cj * dck_dc);
        const float R3 = ex2_approx(-c.N3 * lg2_approx(a * b * cc));   // (r_ij r_ik r_jk)^-N3
        const float fa = s.nb_2b[jn].w, fb = s.nb_2b[kn].w;
        float sin_c, cos_c;
        __sincosf(cc * c.pi_over_rcut, &sin_c, &cos_c);
        const float hp = -0.5f * c.pi_over_rcut;
        const float fcc = 0.5f * (cos_c + 1.0f), dfcc = hp * sin_c;
        const float dfa = hp * __sinf(a * c.pi_over_rcut), dfb = hp * __sinf(b * c.pi_over_rcut);
        const float F3 = fa * fb * fcc;
        const float WR = c.w3 * R3;
        const float W = WR * Q * F3;
        const float QFN = Q * F3 * c.N3;
        const float dW_da = WR * (dQ_da * F3 - QFN * inv_a + Q * dfa * fb * fcc);
        const float dW_db = WR * (dQ_db * F3 - QFN * inv_b + Q * fa * dfb * fcc);
        const float dW_dc = WR * (dQ_dc * F3 - QFN * inv_c + Q * fa * fb * dfcc);
        const float Ac = c.ang2 * ci, As = c.ang2 * si;
        const float dsi_dci = si > 1e-7f ? -ci * rcp_approx(si) : 0.0f;   // collinear guard
        // radial Gaussians rad_k = 2^-(y - y_k)^2, y = xbar sqrt(eta3 log2 e);
        // S = sum_k g_k rad_k and S1 = sum_k g_k (y - y_k) rad_k, with
        // d rad_k / d xbar = -2 eta3 (xbar - R_k) rad_k = -2 eta3 / sqrt(eta3 log2 e) (y - y_k) rad_k
        const float y = 0.5f * (a + b) * c.sq_eta3;
        const float2* gb = grad3(s.g, c) + pair_index(s.nb_el[jn], s.nb_el[kn], c.n_el) * c.n3;
        float Sc = 0.f, Ss = 0.f, Sc1 = 0.f, Ss1 = 0.f;
        for (int k = 0; k < c.n3; ++k) {
          const float d = y - c.ys3[k];
          const float rad = ex2_approx(-(d * d));
          const float td = d * rad;
          const float2 g = gb[k];
          Sc = fmaf(g.x, rad, Sc);
          Ss = fmaf(g.y, rad, Ss);
          Sc1 = fmaf(g.x, td, Sc1);
          Ss1 = fmaf(g.y, td, Ss1);
        }
        const float kd = -2.0f * c.eta3 / c.sq_eta3;
        Sc1 *= kd;
        Ss1 *= kd;
        const float AS = Ac * Sc + As * Ss;
        const float AS1 = Ac * Sc1 + As * Ss1;
        const float dA = c.ang2 * (Sc + dsi_dci * Ss);   // d(A.S)/d cos(th_i) at fixed S
        const float dE_da = dW_da * AS + W * dA * dci_da + W * AS1 * 0.5f;
        const float dE_db = dW_db * AS + W * dA * dci_db + W * AS1 * 0.5f;
        const float dE_dc = dW_dc * AS + W * dA * dci_dc;
        // a = |r_j - r_i|, b = |r_k - r_i|, cc = |r_k - r_j|
        gi_x -= dE_da * uj.x + dE_db * uk.x;
        gi_y -= dE_da * uj.y + dE_db * uk.y;
        gi_z -= dE_da * uj.z + dE_db * uk.z;
        gj0 = dE_da * uj.x - dE_dc * ux;
        gj1 = dE_da * uj.y - dE_dc * uy;
        gj2 = dE_da * uj.z - dE_dc * uz;
        gk0 = dE_db * uk.x + dE_dc * ux;
        gk1 = dE_db * uk.y + dE_dc * uy;
        gk2 = dE_db * uk.z + dE_dc * uz;
      }
    }
    // j side: segmented inclusive scan over lanes with equal jn (runs are contiguous)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float t0 = __shfl_up_sync(0xffffffffu, gj0, o);
      const float t1 = __shfl_up_sync(0xffffffffu, gj1, o);
      const float t2 = __shfl_up_sync(0xffffffffu, gj2, o);
      const int kk = __shfl_up_sync(0xffffffffu, jn, o);
      if (lane >= o && kk == jn) {
        gj0 += t0;
        gj1 += t1;
        gj2 += t2;
      }
    }
    const int next = __shfl_down_sync(0xffffffffu, jn, 1);
    if (jn < n && (lane == 31 || next != jn)) {
      const int jl = s.nb_idx[jn];
      s.facc[3 * jl + 0] += gj0;
      s.facc[3 * jl + 1] += gj1;
      s.facc[3 * jl + 2] += gj2;
    }
    __syncwarp();
    // k side: one row at a time (distinct atoms within a row)
    const int r_first = __shfl_sync(0xffffffffu, jn, 0);
    const int r_last = __reduce_max_sync(0xffffffffu, jn < n ? jn : -1);
    for (int r = r_first; r <= r_last; ++r) {
      if (jn == r) {
        const int kl = s.nb_idx[kn];
        s.facc[3 * kl + 0] += gk0;
        s.facc[3 * kl + 1] += gk1;
        s.facc[3 * kl + 2] += gk2;
      }
      __syncwarp();
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gi_x += __shfl_xor_sync(0xffffffffu, gi_x, o);
    gi_y += __shfl_xor_sync(0xffffffffu, gi_y, o);
    gi_z += __shfl_xor_sync(0xffffffffu, gi_z, o);
  }
  if (lane == 0) {
    s.facc[3 * il + 0] += gi_x;
    s.facc[3 * il + 1] += gi_y;
    s.facc[3 * il + 2] += gi_z;
  }
  __syncwarp();
}

__global__ void __launch_bounds__(32 * kWarpsVjp)
fchl19_vjp_kernel(const float* __restrict__ coords, const int32_t* __restrict__ elem,
                  const int32_t* __restrict__ mol_ptr, int n_mol, int mx, int mxp, int rp,
                  Fchl19Consts c, const float* __restrict__ grad_rep, int rep_ld,
                  float* __restrict__ grad_coords, int accumulate, int* err) {
  extern __shared__ __align__(16) char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = blockIdx.x;
  const int a0 = __ldg(mol_ptr + m);
  const int M = __ldg(mol_ptr + m + 1) - a0;
  if (M > mx) {
    if (threadIdx.x == 0) record_device_error(err, DEV_MOL_TOO_LARGE);
    return;
  }
  float4* pos = reinterpret_cast<float4*>(smem_raw);
  VjpWarp s = carve_vjp(smem_raw + (size_t)mxp * 16 + warp * vjp_warp_bytes(mxp, rp), mxp, rp);
  stage_molecule(coords, elem, a0, M, c.n_el, pos, threadIdx.x, blockDim.x, err);
  for (int k = lane; k < 3 * mxp; k += 32) s.facc[k] = 0.0f;
  __syncthreads();

  for (int il = warp; il < M; il += kWarpsVjp) {
    vjp_centre(pos, M, il, c, grad_rep + (size_t)(a0 + il) * rep_ld, s, lane);
  }
  __syncthreads();
  // fixed-order reduction over the warps' buffers
  for (int k = threadIdx.x; k < 3 * M; k += blockDim.x) {
    float sum = 0.f;
    for (int w = 0; w < kWarpsVjp; ++w)
      sum += carve_vjp(smem_raw + (size_t)mxp * 16 + w * vjp_warp_bytes(mxp, rp), mxp, rp).facc[k];
    float* dst = grad_coords + 3 * (size_t)a0 + k;
    *dst = accumulate ? *dst + sum : sum;
  }
}

// ---------------------------------------------------------------------------
// Jacobian blocks (forward mode): for centre I and atom k of the same molecule,
// the three rows d rho_I / d r_{k,x} (x = 0, 1, 2). Neighbour blocks are formed
// from the two-body term of the pair (I, k) and every three-body term in which
// k is one of the two neighbours (recomputed here); atoms beyond the cutoff
// give zero rows; the centre's own block is minus the sum of its neighbours'
// blocks (translation invariance), summed in neighbour order.
//   row index = jac_ptr[m] + (I_local * M + k_local) * 3 + x

struct JacWarp {
  float4* pos;    // [mxp]
  float4* nb_u;   // [mxp]
  float4* nb_2b;  // [mxp]
  float4* pairs;  // [32][4]: cA (cos, sin), hA (cos, sin) | cC (cos, sin), xbar, bin | uC, -
  float* blk;     // [3][rp]
  float* cblk;    // [3][rp]
  int* nb_el;     // [mxp]
  int* nb_idx;    // [mxp]
};
__host__ __device__ __forceinline__ size_t jac_warp_bytes(int mxp, int rp) {
  return (size_t)mxp * 56 + (size_t)rp * 24 + 32 * 64;
}
__device__ __forceinline__ JacWarp carve_jac(char* base, int mxp, int rp) {
  JacWarp s;
  s.pos = reinterpret_cast<float4*>(base);
  s.nb_u = s.pos + mxp;
  s.nb_2b = s.nb_u + mxp;
  s.pairs = s.nb_2b + mxp;
  s.blk = reinterpret_cast<float*>(s.pairs + 32 * 4);
  s.cblk = s.blk + 3 * rp;
  s.nb_el = reinterpret_cast<int*>(s.cblk + 3 * rp);
  s.nb_idx = s.nb_el + mxp;
  return s;
}

__global__ void __launch_bounds__(32 * kWarpsFwd)
fchl19_jac_kernel(const float* __restrict__ coords, const int32_t* __restrict__ elem,
                  const int32_t* __restrict__ mol_ptr, int n_mol, int n_atoms, int mx, int mxp, int rp,
                  Fchl19Consts c, const int64_t* __restrict__ jac_ptr, float* __restrict__ jac,
                  int rep_ld, int32_t* __restrict__ row_elem, int* err) {
  extern __shared__ __align__(16) char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int atom = blockIdx.x * kWarpsFwd + warp;
  if (atom >= n_atoms) return;
  JacWarp s = carve_jac(smem_raw + warp * jac_warp_bytes(mxp, rp), mxp, rp);
  const int m = find_molecule(mol_ptr, n_mol, atom);
  const int a0 = __ldg(mol_ptr + m);
  const int M = __ldg(mol_ptr + m + 1) - a0;
  const int il = atom - a0;
  if (M > mx) {
    if (lane == 0) record_device_error(err, DEV_MOL_TOO_LARGE);
    return;
  }
  const long base_row = jac_ptr[m] + (long)il * M * 3;
  const int ei = __ldg(elem + atom);
  for (int r = lane; r < 3 * M; r += 32) row_elem[base_row + r] = (ei >= 0 && ei < c.n_el) ? ei : 0;
  stage_molecule(coords, elem, a0, M, c.n_el, s.pos, lane, 32, err);
  for (int k = lane; k < 3 * rp; k += 32) s.cblk[k] = 0.f;
  __syncwarp();
  const int n = neighbour_list(s.pos, M, il, c, s.nb_u, s.nb_2b, s.nb_el, s.nb_idx, lane);
  const float neg_eta3 = -c.eta3 * kLog2e;

  int next_nb = 0;
  for (int kl = 0; kl < M; ++kl) {
    float* out = jac + (base_row + (long)kl * 3) * rep_ld;
    if (kl == il) continue;                                   // written last
    if (next_nb >= n || s.nb_idx[next_nb] != kl) {            // beyond the cutoff: zero rows
      for (int q = lane; q < 3 * rep_ld; q += 32) out[q] = 0.f;
      continue;
    }
    const int kn = next_nb++;
    for (int q = lane; q < 3 * rp; q += 32) s.blk[q] = 0.f;
    __syncwarp();
    const float4 uA = s.nb_u[kn];
    const float A = uA.w;
    // two-body term of the pair (I, k): d G / d r_k = G'(A) uA
    {
      // reciprocals, the power and the cutoff's sine from the hardware approximations
      const float4 t = s.nb_2b[kn];
      const float inv_r = rcp_approx(A);
      const float inv_s2 = 2.0f * t.y;                           // 1 / sigma^2
      const float inv_sd = inv_s2 * rsqrt_approx(inv_s2);        // 1 / sigma
      const float inv_rr = rcp_approx(fmaf(A, A, c.eta2));       // 1 / (r^2 + eta2)
      const float ds = -c.eta2 * inv_sd * inv_r * inv_rr;        // d sigma / dr
      const float dmu = inv_r + c.eta2 * inv_r * inv_rr;         // d mu / dr
      const float fc = t.w;
      const float dfc = -0.5f * c.pi_over_rcut * __sinf(A * c.pi_over_rcut);
      const float rN = ex2_approx(-c.N2 * lg2_approx(A));
      const float P = fc * rN;
      const float dP = rN * (dfc - c.N2 * fc * inv_r);
      const float pre = c.inv_sqrt_2pi * inv_sd, negc = -t.y * kLog2e;
      const float k1 = -ds * inv_sd, k2 = dmu * inv_s2, k3 = ds * inv_s2 * inv_sd;
      const int b0 = s.nb_el[kn] * c.n2;
      for (int q = lane; q < c.n2; q += 32) {
        const float a = c.rs2_log[q] - t.x;
        const float L = c.rs2_inv[q] * pre * ex2_approx(a * (a * negc));
        const float dlnL = k1 + a * k2 + a * a * k3;
        const float g = L * (dP + P * dlnL);
        s.blk[0 * rp + b0 + q] += g * uA.x;
        s.blk[1 * rp + b0 + q] += g * uA.y;
        s.blk[2 * rp + b0 + q] += g * uA.z;
      }
    }
    __syncwarp();
    // three-body terms with k as one of the two neighbours, the other neighbour j
    for (int j0 = 0; j0 < n; j0 += 32) {
      const int jn = j0 + lane;
      bool ok = false;
      float4 q0 = make_float4(0, 0, 0, 0), q1 = q0, q2 = q0;
      if (jn < n && jn != kn) {
        const float4 uB = s.nb_u[jn];
        const float B = uB.w;
        const float vx = uB.x * B - uA.x * A, vy = uB.y * B - uA.y * A, vz = uB.z * B - uA.z * A;
        const float C2 = vx * vx + vy * vy + vz * vz;
        if (C2 < c.rcut2) {
          ok = true;
          // reciprocals, square roots, the ATM power and the cutoffs from the
          // hardware approximations (a few ulp)
          const float icc = rsqrt_approx(C2);
          const float C = C2 * icc;
          const float ux = vx * icc, uy = vy * icc, uz = vz * icc;   // unit k -> j
          const float ci = uA.x * uB.x + uA.y * uB.y + uA.z * uB.z;
          const float crx = uA.y * uB.z - uA.z * uB.y;
          const float cry = uA.z * uB.x - uA.x * uB.z;
          const float crz = uA.x * uB.y - uA.y * uB.x;
          const float s2i = crx * crx + cry * cry + crz * crz;
          const float si = s2i > 0.0f ? s2i * rsqrt_approx(s2i) : 0.0f;
          const float ck = -(uA.x * ux + uA.y * uy + uA.z * uz);   // angle at k (first neighbour)
          const float cj = (uB.x * ux + uB.y * uy + uB.z * uz);    // angle at j (second neighbour)
          // sides: a = A (I-k), b = B (I-j), cc = C (k-j); "first" = k, "second" = j
          const float a = A, b = B, cc = C;
          const float ia = rcp_approx(a), ib = rcp_approx(b);
          const float iab = ia * ib, iac = ia * icc, ibc = ib * icc;
          const float dci_da = (a - b * ci) * iab, dci_dc = -cc * iab;
          const float dcf_da = (a - cc * ck) * iac, dcf_dc = (cc - a * ck) * iac;
          const float dcs_da = -a * ibc, dcs_dc = (cc - b * cj) * ibc;
          const float Q = 1.0f + 3.0f * ci * ck * cj;
          const float dQ_da = 3.0f * (dci_da * ck * cj + ci * dcf_da * cj + ci * ck * dcs_da);
          const float dQ_dc = 3.0f * (dci_dc * ck * cj + ci * dcf_dc * cj + ci * ck * dcs_dc);
          const float R3 = ex2_approx(-c.N3 * lg2_approx(a * b * cc));
          const float fa = s.nb_2b[kn].w, fb = s.nb_2b[jn].w;
          float sin_c, cos_c;
          __sincosf(cc * c.pi_over_rcut, &sin_c, &cos_c);
          const float hp = -0.5f * c.pi_over_rcut;
          const float fcc = 0.5f * (cos_c + 1.0f), dfcc = hp * sin_c;
          const float dfa = hp * __sinf(a * c.pi_over_rcut);
          const float F3 = fa * fb * fcc;
          const float WR = c.w3 * R3;
          const float W = WR * Q * F3;
          const float QFN = Q * F3 * c.N3;
          const float dW_da = WR * (dQ_da * F3 - QFN * ia + Q * dfa * fb * fcc);
          const float dW_dc = WR * (dQ_dc * F3 - QFN * icc + Q * fa * fb * dfcc);
          const float Ac = c.ang2 * ci, As = c.ang2 * si;
          const float dAc = c.ang2, dAs = si > 1e-7f ? -c.ang2 * ci * rcp_approx(si) : 0.0f;
          const int bin = c.base3 + pair_index(s.nb_el[kn], s.nb_el[jn], c.n_el) * c.n3 * 2;
          q0 = make_float4(dW_da * Ac + W * dAc * dci_da, dW_da * As + W * dAs * dci_da, 0.5f * W * Ac,
                           0.5f * W * As);
          q1 = make_float4(dW_dc * Ac + W * dAc * dci_dc, dW_dc * As + W * dAs * dci_dc, 0.5f * (a + b),
                           __int_as_float(bin));
          q2 = make_float4(ux, uy, uz, 0.f);
        }
      }
      const unsigned mask = __ballot_sync(0xffffffffu, ok);
      if (ok) {
        const int slot = __popc(mask & ((1u << lane) - 1u));
        s.pairs[4 * slot + 0] = q0;
        s.pairs[4 * slot + 1] = q1;
        s.pairs[4 * slot + 2] = q2;
      }
      __syncwarp();
      const int cnt = __popc(mask);
      for (int t = 0; t < cnt; ++t) {
        const float4 p0 = s.pairs[4 * t], p1 = s.pairs[4 * t + 1], p2 = s.pairs[4 * t + 2];
        const int bin = __float_as_int(p1.w);
        for (int q = lane; q < c.n3; q += 32) {
          const float d = p1.z - c.rs3[q];
          const float rad = ex2_approx(d * (d * neg_eta3));
          const float drad = -2.0f * c.eta3 * d * rad;
          // d v / d r_k = dv/da * uA - dv/dc * uC   (C = |r_j - r_k|)
          const float da_c = rad * p0.x + drad * p0.z, da_s = rad * p0.y + drad * p0.w;
          const float dc_c = rad * p1.x, dc_s = rad * p1.y;
          const int bc = bin + 2 * q;
          s.blk[0 * rp + bc] += da_c * uA.x - dc_c * p2.x;
          s.blk[1 * rp + bc] += da_c * uA.y - dc_c * p2.y;
          s.blk[2 * rp + bc] += da_c * uA.z - dc_c * p2.z;
          s.blk[0 * rp + bc + 1] += da_s * uA.x - dc_s * p2.x;
          s.blk[1 * rp + bc + 1] += da_s * uA.y - dc_s * p2.y;
          s.blk[2 * rp + bc + 1] += da_s * uA.z - dc_s * p2.z;
        }
      }
      __syncwarp();
    }
    // write the block; accumulate minus it into the centre's block
    for (int x = 0; x < 3; ++x)
      for (int q = lane; q < rep_ld; q += 32) {
        const float v = q < c.rep_dim ? s.blk[x * rp + q] : 0.f;
        out[(long)x * rep_ld + q] = v;
        if (q < c.rep_dim) s.cblk[x * rp + q] -= v;
      }
    __syncwarp();
  }
  float* outc = jac + (base_row + (long)il * 3) * rep_ld;
  for (int x = 0; x < 3; ++x)
    for (int q = lane; q < rep_ld; q += 32) outc[(long)x * rep_ld + q] = q < c.rep_dim ? s.cblk[x * rp + q] : 0.f;
}

// jac_ptr[m] = sum_{m' < m} 3 M_{m'}^2 (one CTA, sequential over chunks of 1024 molecules)
__global__ void jac_offsets_kernel(const int32_t* __restrict__ mol_ptr, int n_mol, int64_t* __restrict__ out) {
  __shared__ long long part[1024];
  long long carry = 0;
  for (int base = 0; base < n_mol; base += 1024) {
    const int m = base + threadIdx.x;
    long long v = 0;
    if (m < n_mol) {
      const long long M = mol_ptr[m + 1] - mol_ptr[m];
      v = 3 * M * M;
    }
    part[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const long long t = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += t;
      __syncthreads();
    }
    if (m < n_mol) out[m] = carry + part[threadIdx.x] - v;
    carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n_mol] = carry;
}

// VJP with one warp per centre atom (the atoms of a molecule run in parallel):
// each warp writes its centre's contributions to every atom of the molecule
// into contrib[pair_ptr[m] + (I*M + k)*3 + x]; vjp_reduce_kernel then sums
// them over the centres I in order.
__global__ void __launch_bounds__(32 * kWarpsFwd)
fchl19_vjp_centre_kernel(const float* __restrict__ coords, const int32_t* __restrict__ elem,
                         const int32_t* __restrict__ mol_ptr, int n_mol, int n_atoms, int mx, int mxp, int rp,
                         Fchl19Consts c, const float* __restrict__ grad_rep, int rep_ld,
                         const int64_t* __restrict__ pair_ptr, float* __restrict__ contrib, int* err) {
  extern __shared__ __align__(16) char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int atom = blockIdx.x * kWarpsFwd + warp;
  if (atom >= n_atoms) return;
  char* base = smem_raw + warp * ((size_t)mxp * 16 + vjp_warp_bytes(mxp, rp));
  float4* pos = reinterpret_cast<float4*>(base);
  VjpWarp s = carve_vjp(base + (size_t)mxp * 16, mxp, rp);
  const int m = find_molecule(mol_ptr, n_mol, atom);
  const int a0 = __ldg(mol_ptr + m);
  const int M = __ldg(mol_ptr + m + 1) - a0;
  const int il = atom - a0;
  if (M > mx) {
    if (lane == 0) record_device_error(err, DEV_MOL_TOO_LARGE);
    return;
  }
  stage_molecule(coords, elem, a0, M, c.n_el, pos, lane, 32, err);
  for (int k = lane; k < 3 * M; k += 32) s.facc[k] = 0.0f;
  __syncwarp();
  vjp_centre(pos, M, il, c, grad_rep + (size_t)atom * rep_ld, s, lane);
  __syncwarp();
  float* out = contrib + pair_ptr[m] + (long)il * M * 3;
  for (int k = lane; k < 3 * M; k += 32) out[k] = s.facc[k];
}

// grad[k][x] = scale * sum_{I = 0..M-1} contrib[pair_ptr[m] + (I*M + k_local)*3 + x] (+ grad if accumulate)
__global__ void vjp_reduce_kernel(const int32_t* __restrict__ mol_ptr, int n_mol, int n_atoms,
                                  const int64_t* __restrict__ pair_ptr, const float* __restrict__ contrib,
                                  float scale, int accumulate, float* __restrict__ grad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * n_atoms) return;
  const int atom = t / 3, x = t % 3;
  int lo = 0, hi = n_mol;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (mol_ptr[mid] <= atom) lo = mid; else hi = mid;
  }
  const int a0 = mol_ptr[lo], M = mol_ptr[lo + 1] - a0, kl = atom - a0;
  const float* cp = contrib + pair_ptr[lo] + (long)kl * 3 + x;
  float sum = 0.f;
  for (int I = 0; I < M; ++I) sum += cp[(long)I * M * 3];
  grad[t] = accumulate ? grad[t] + scale * sum : scale * sum;
}

// ---------------------------------------------------------------------------
// Periodic systems (the paper's periodic MOF and water rows): the environment of
// centre i is its list of lattice images (j, n) within r_cut, from the host
// cell list (qmlr_periodic_environment), at R_j + n . cell. A warp per centre
// builds its neighbour list from that list (the displacement R_j + n . cell -
// R_i formed in FP64, then rounded, so that the lattice shift does not cost
// FP32 precision), then runs the molecular kernels' row or adjoint arithmetic.

struct Cell9 {
  double a[9];   // lattice vectors as rows
};

__device__ __forceinline__ bool periodic_entry(const float* __restrict__ coords, const int32_t* __restrict__ elem,
                                               int n_atoms, const Cell9& cell, const int32_t* __restrict__ env_atom,
                                               const int32_t* __restrict__ env_shift, long e, double xi, double yi,
                                               double zi, int n_el, float rcut2, float& dx, float& dy, float& dz,
                                               float& r2, int& el, int* err) {
  const int j = __ldg(env_atom + e);
  if (j < 0 || j >= n_atoms) {
    record_device_error(err, DEV_BAD_INDEX);
    return false;
  }
  const double n0 = __ldg(env_shift + 3 * e), n1 = __ldg(env_shift + 3 * e + 1), n2 = __ldg(env_shift + 3 * e + 2);
  const double px = (double)__ldg(coords + 3 * (size_t)j) + n0 * cell.a[0] + n1 * cell.a[3] + n2 * cell.a[6];
  const double py = (double)__ldg(coords + 3 * (size_t)j + 1) + n0 * cell.a[1] + n1 * cell.a[4] + n2 * cell.a[7];
  const double pz = (double)__ldg(coords + 3 * (size_t)j + 2) + n0 * cell.a[2] + n1 * cell.a[5] + n2 * cell.a[8];
  dx = (float)(px - xi);
  dy = (float)(py - yi);
  dz = (float)(pz - zi);
  r2 = dx * dx + dy * dy + dz * dz;
  el = __ldg(elem + j);
  if (el < 0 || el >= n_el) {
    record_device_error(err, DEV_BAD_ELEMENT);
    el = 0;
  }
  return r2 < rcut2 && r2 > 0.f;
}

__global__ void __launch_bounds__(32 * kWarpsFwd, 6)
fchl19_periodic_kernel(const float* __restrict__ coords, const int32_t* __restrict__ elem, int n_atoms, Cell9 cell,
                       const int64_t* __restrict__ env_ptr, const int32_t* __restrict__ env_atom,
                       const int32_t* __restrict__ env_shift, int max_env, int envp, Fchl19Consts c,
                       float* __restrict__ rep, int rep_ld, int* err) {
  extern __shared__ __align__(16) char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarpsFwd + warp;
  if (i >= n_atoms) return;
  const RegWarp s = carve_reg(smem_raw + warp * reg_warp_bytes(envp), envp);
  const BinConsts kb = bin_consts(c, lane);
  float* out = rep + (size_t)i * rep_ld;
  const long e0 = __ldg(env_ptr + i), e1 = __ldg(env_ptr + i + 1);
  if (e1 - e0 > max_env || e1 < e0) {
    if (lane == 0) record_device_error(err, DEV_MOL_TOO_LARGE);
    for (int k = lane; k < rep_ld; k += 32) out[k] = 0.0f;
    return;
  }
  const double xi = __ldg(coords + 3 * (size_t)i), yi = __ldg(coords + 3 * (size_t)i + 1),
               zi = __ldg(coords + 3 * (size_t)i + 2);
  int n = 0;
  for (long b0 = e0; b0 < e1; b0 += 32) {
    const long e = b0 + lane;
    bool ok = false;
    float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
    int el = 0;
    if (e < e1)
      ok = periodic_entry(coords, elem, n_atoms, cell, env_atom, env_shift, e, xi, yi, zi, c.n_el, c.rcut2, dx, dy,
                          dz, r2, el, err);
    const unsigned mask = __ballot_sync(0xffffffffu, ok);
    if (ok) store_neighbour(s, n + __popc(mask & ((1u << lane) - 1u)), dx, dy, dz, r2, el, c);
    n += __popc(mask);
  }
  __syncwarp();
  fwd_row(s, n, c, kb, out, rep_ld, lane);
}

// Adjoint: warp per centre i; the contribution of every environment entry e
// goes to contrib[e] (the gradient with respect to the image, which is the
// gradient with respect to R_j), the centre's own to contrib[E + i]. Entries
// beyond the cutoff in FP32 get zero.
__global__ void __launch_bounds__(32 * kWarpsVjp)
fchl19_periodic_vjp_kernel(const float* __restrict__ coords, const int32_t* __restrict__ elem, int n_atoms,
                           Cell9 cell, const int64_t* __restrict__ env_ptr, const int32_t* __restrict__ env_atom,
                           const int32_t* __restrict__ env_shift, int max_env, int envp, Fchl19Consts c,
                           const float* __restrict__ grad_rep, int rep_ld, float* __restrict__ contrib,
                           int* err) {
  extern __shared__ __align__(16) char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarpsVjp + warp;
  if (i >= n_atoms) return;
  const int rp = (c.rep_dim + 3) & ~3;
  VjpWarp s = carve_vjp(smem_raw + warp * vjp_warp_bytes(envp + 4, rp), envp + 4, rp);
  const long E = __ldg(env_ptr + n_atoms);
  const long e0 = __ldg(env_ptr + i), e1 = __ldg(env_ptr + i + 1);
  const int ne = (int)(e1 - e0);
  if (e1 - e0 > max_env || e1 < e0) {
    if (lane == 0) record_device_error(err, DEV_MOL_TOO_LARGE);
    if (e1 >= e0)
      for (long k = 3 * e0 + lane; k < 3 * e1; k += 32) contrib[k] = 0.0f;
    if (lane < 3) contrib[3 * (E + i) + lane] = 0.0f;
    return;
  }
  load_grad_row(s.g, grad_rep + (size_t)i * rep_ld, c, lane);
  for (int k = lane; k < 3 * (ne + 1); k += 32) s.facc[k] = 0.0f;
  const double xi = __ldg(coords + 3 * (size_t)i), yi = __ldg(coords + 3 * (size_t)i + 1),
               zi = __ldg(coords + 3 * (size_t)i + 2);
  int n = 0;
  for (long b0 = e0; b0 < e1; b0 += 32) {
    const long e = b0 + lane;
    bool ok = false;
    float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
    int el = 0;
    if (e < e1)
      ok = periodic_entry(coords, elem, n_atoms, cell, env_atom, env_shift, e, xi, yi, zi, c.n_el, c.rcut2, dx, dy,
                          dz, r2, el, err);
    const unsigned mask = __ballot_sync(0xffffffffu, ok);
    if (ok) {
      const int slot = n + __popc(mask & ((1u << lane) - 1u));
      const float r = sqrtf(r2);
      const float inv = 1.0f / r;
      s.nb_u[slot] = make_float4(dx * inv, dy * inv, dz * inv, r);
      s.nb_el[slot] = el;
      s.nb_idx[slot] = (int)(e - e0);          // accumulator: the entry
      const float fc = cutoff_f(r, c);
      const float s2 = log1pf(c.eta2 * inv * inv);
      s.nb_2b[slot] = make_float4(logf(r) - 0.5f * s2, 0.5f / s2,
                                  fc * expf(-c.N2 * logf(r)) * c.inv_sqrt_2pi / sqrtf(s2), fc);
    }
    n += __popc(mask);
  }
  __syncwarp();
  vjp_from_neighbours(n, ne, c, s, lane);       // the centre's accumulator after the entries'
  __syncwarp();
  for (int k = lane; k < 3 * ne; k += 32) contrib[3 * e0 + k] = s.facc[k];
  if (lane < 3) contrib[3 * (E + i) + lane] = s.facc[3 * ne + lane];
}

// grad[k] (+)= scale * (contrib[E + k] + sum over the entries naming atom k, in
// entry order); rev_ptr / rev_entry: the entries grouped by atom.
__global__ void periodic_reduce_kernel(int n_atoms, const int64_t* __restrict__ env_ptr,
                                       const int64_t* __restrict__ rev_ptr, const int64_t* __restrict__ rev_entry,
                                       const float* __restrict__ contrib, float scale, int accumulate,
                                       float* __restrict__ grad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * n_atoms) return;
  const int k = t / 3, x = t % 3;
  const long E = env_ptr[n_atoms];
  float sum = contrib[3 * (E + k) + x];
  for (long q = rev_ptr[k]; q < rev_ptr[k + 1]; ++q) sum += contrib[3 * rev_entry[q] + x];
  grad[t] = accumulate ? grad[t] + scale * sum : scale * sum;
}

static int rep_pad_of(int rep_dim) { return (rep_dim + 3) & ~3; }

static int check_geometry(const float* coords, const int32_t* elem, const int32_t* mol_ptr,
                          int n_mol, int n_atoms, int max_mol_atoms) {
  QMLR_REQUIRE(n_mol >= 0 && n_atoms >= 0, "n_mol and n_atoms must be >= 0");
  QMLR_REQUIRE(max_mol_atoms >= 1 && max_mol_atoms <= 256,
               "max_mol_atoms must be in 1..256 (got %d)", max_mol_atoms);
  QMLR_REQUIRE(n_atoms == 0 || (coords && elem), "coords/elem are NULL");
  QMLR_REQUIRE(n_mol == 0 || mol_ptr, "mol_ptr is NULL");
  return QMLR_OK;
}

}  // namespace qmlr

using namespace qmlr;

extern "C" int qmlr_fchl19_rep_dim(const qmlr_fchl19_params* p, int32_t* rep_dim) {
  int rc = validate_params(p);
  if (rc) return rc;
  QMLR_REQUIRE(rep_dim, "rep_dim is NULL");
  *rep_dim = rep_dim_of(*p);
  return QMLR_OK;
}

extern "C" int qmlr_fchl19(const float* coords, const int32_t* elem, const int32_t* mol_ptr,
                           int32_t n_mol, int32_t n_atoms, int32_t max_mol_atoms,
                           const qmlr_fchl19_params* p, float* rep, int32_t rep_ld, void* stream) {
  int rc = validate_params(p);
  if (rc) return rc;
  rc = check_geometry(coords, elem, mol_ptr, n_mol, n_atoms, max_mol_atoms);
  if (rc) return rc;
  const int rd = rep_dim_of(*p);
  QMLR_REQUIRE(rep_ld >= rd, "rep_ld (%d) < rep_dim (%d)", rep_ld, rd);
  QMLR_REQUIRE(n_atoms == 0 || rep, "rep is NULL");
  if (n_atoms == 0) return QMLR_OK;
  QMLR_REQUIRE(n_mol >= 1, "n_atoms > 0 but n_mol == 0");
  const Fchl19Consts c = make_consts(*p);
  const int rp = rep_pad_of(rd);
  const int mx = max_mol_atoms;
  const int mxp = (mx + 3) & ~3;
  const size_t smem = kWarpsFwd * fwd_warp_bytes(mxp, rp);
  QMLR_REQUIRE(smem <= 227 * 1024, "shared memory request too large");
  if (p->n_el <= 5 && p->n2 <= 32 && p->n3 <= 32) {
    // 32-atom ranges once they still give every SM several CTAs, one atom per warp below that
    const int range = n_atoms >= kFwdRange * 8 * sm_count() ? kFwdRange : kWarpsFwd;
    const size_t rsmem = (size_t)reg_stage_atoms(mx, range) * 16 + kWarpsFwd * reg_warp_bytes(mxp);
    QMLR_CUDA_TRY(smem_attr_once((const void*)fchl19_forward_reg_kernel,
                                 (int)((size_t)reg_stage_atoms(mx, kFwdRange) * 16 + kWarpsFwd * reg_warp_bytes(mxp))));
    const int rgrid = (n_atoms + range - 1) / range;
    fchl19_forward_reg_kernel<<<rgrid, 32 * kWarpsFwd, rsmem, as_stream(stream)>>>(
        coords, elem, mol_ptr, n_mol, n_atoms, mx, mxp, range, c, rep, rep_ld, device_error_ptr());
  } else {
    QMLR_CUDA_TRY(smem_attr_once((const void*)fchl19_forward_kernel, 227 * 1024));
    const int grid = (n_atoms + kWarpsFwd - 1) / kWarpsFwd;
    fchl19_forward_kernel<<<grid, 32 * kWarpsFwd, smem, as_stream(stream)>>>(
        coords, elem, mol_ptr, n_mol, n_atoms, mx, mxp, rp, c, rep, rep_ld, device_error_ptr());
  }
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

extern "C" int qmlr_fchl19_vjp(const float* coords, const int32_t* elem, const int32_t* mol_ptr,
                               int32_t n_mol, int32_t n_atoms, int32_t max_mol_atoms,
                               const qmlr_fchl19_params* p, const float* grad_rep, int32_t rep_ld,
                               float* grad_coords, int32_t accumulate, void* stream) {
  int rc = validate_params(p);
  if (rc) return rc;
  rc = check_geometry(coords, elem, mol_ptr, n_mol, n_atoms, max_mol_atoms);
  if (rc) return rc;
  const int rd = rep_dim_of(*p);
  QMLR_REQUIRE(rep_ld >= rd, "rep_ld (%d) < rep_dim (%d)", rep_ld, rd);
  QMLR_REQUIRE(n_atoms == 0 || (grad_rep && grad_coords), "grad_rep/grad_coords are NULL");
  if (n_atoms == 0 || n_mol == 0) return QMLR_OK;
  const Fchl19Consts c = make_consts(*p);
  const int rp = rep_pad_of(rd);
  const int mx = max_mol_atoms;
  const int mxp = (mx + 3) & ~3;
  const size_t smem = (size_t)mxp * 16 + kWarpsVjp * vjp_warp_bytes(mxp, rp);
  QMLR_REQUIRE(smem <= 200 * 1024, "shared memory request too large");
  QMLR_CUDA_TRY(smem_attr_once((const void*)fchl19_vjp_kernel, 200 * 1024));
  fchl19_vjp_kernel<<<n_mol, 32 * kWarpsVjp, smem, as_stream(stream)>>>(
      coords, elem, mol_ptr, n_mol, mx, mxp, rp, c, grad_rep, rep_ld, grad_coords, accumulate,
      device_error_ptr());
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

extern "C" int qmlr_jac_offsets(const int32_t* mol_ptr, int32_t n_mol, int64_t* jac_ptr, int64_t* host_total,
                                void* stream) {
  QMLR_REQUIRE(mol_ptr && jac_ptr && n_mol >= 0, "bad arguments");
  cudaStream_t st = as_stream(stream);
  jac_offsets_kernel<<<1, 1024, 0, st>>>(mol_ptr, n_mol, jac_ptr);
  QMLR_LAUNCH_CHECK();
  if (host_total) {
    int64_t t = 0;
    QMLR_CUDA_TRY(cudaMemcpyAsync(&t, jac_ptr + n_mol, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    QMLR_CUDA_TRY(cudaStreamSynchronize(st));
    *host_total = t;
  }
  return QMLR_OK;
}

extern "C" int qmlr_fchl19_jac(const float* coords, const int32_t* elem, const int32_t* mol_ptr,
                               int32_t n_mol, int32_t n_atoms, int32_t max_mol_atoms,
                               const qmlr_fchl19_params* p, const int64_t* jac_ptr, float* jac,
                               int32_t rep_ld, int32_t* row_elem, void* stream) {
  int rc = validate_params(p);
  if (rc) return rc;
  rc = check_geometry(coords, elem, mol_ptr, n_mol, n_atoms, max_mol_atoms);
  if (rc) return rc;
  const int rd = rep_dim_of(*p);
  QMLR_REQUIRE(rep_ld >= rd, "rep_ld (%d) < rep_dim (%d)", rep_ld, rd);
  QMLR_REQUIRE(n_atoms == 0 || (jac_ptr && jac && row_elem), "NULL pointer argument");
  if (n_atoms == 0) return QMLR_OK;
  const Fchl19Consts c = make_consts(*p);
  const int rp = rep_pad_of(rd);
  const int mx = max_mol_atoms;
  const int mxp = (mx + 3) & ~3;
  const size_t smem = kWarpsFwd * jac_warp_bytes(mxp, rp);
  QMLR_REQUIRE(smem <= 227 * 1024, "shared memory request too large");
  QMLR_CUDA_TRY(smem_attr_once((const void*)fchl19_jac_kernel, 227 * 1024));
  const int grid = (n_atoms + kWarpsFwd - 1) / kWarpsFwd;
  fchl19_jac_kernel<<<grid, 32 * kWarpsFwd, smem, as_stream(stream)>>>(
      coords, elem, mol_ptr, n_mol, n_atoms, mx, mxp, rp, c, jac_ptr, jac, rep_ld, row_elem,
      device_error_ptr());
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

extern "C" int qmlr_fchl19_vjp_atoms(const float* coords, const int32_t* elem, const int32_t* mol_ptr,
                                     int32_t n_mol, int32_t n_atoms, int32_t max_mol_atoms,
                                     const qmlr_fchl19_params* p, const float* grad_rep, int32_t rep_ld,
                                     const int64_t* pair_ptr, float* contrib, float scale,
                                     float* grad_coords, int32_t accumulate, void* stream) {
  int rc = validate_params(p);
  if (rc) return rc;
  rc = check_geometry(coords, elem, mol_ptr, n_mol, n_atoms, max_mol_atoms);
  if (rc) return rc;
  const int rd = rep_dim_of(*p);
  QMLR_REQUIRE(rep_ld >= rd, "rep_ld (%d) < rep_dim (%d)", rep_ld, rd);
  if (n_atoms == 0 || n_mol == 0) return QMLR_OK;
  QMLR_REQUIRE(grad_rep && pair_ptr && contrib && grad_coords, "NULL pointer argument");
  const Fchl19Consts c = make_consts(*p);
  const int rp = rep_pad_of(rd);
  const int mx = max_mol_atoms;
  const int mxp = (mx + 3) & ~3;
  const size_t smem = kWarpsFwd * ((size_t)mxp * 16 + vjp_warp_bytes(mxp, rp));
  QMLR_REQUIRE(smem <= 227 * 1024, "shared memory request too large");
  QMLR_CUDA_TRY(smem_attr_once((const void*)fchl19_vjp_centre_kernel, 227 * 1024));
  cudaStream_t st = as_stream(stream);
  fchl19_vjp_centre_kernel<<<(n_atoms + kWarpsFwd - 1) / kWarpsFwd, 32 * kWarpsFwd, smem, st>>>(
      coords, elem, mol_ptr, n_mol, n_atoms, mx, mxp, rp, c, grad_rep, rep_ld, pair_ptr, contrib,
      device_error_ptr());
  QMLR_LAUNCH_CHECK();
  vjp_reduce_kernel<<<(3 * n_atoms + 255) / 256, 256, 0, st>>>(mol_ptr, n_mol, n_atoms, pair_ptr, contrib, scale,
                                                              accumulate, grad_coords);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

static int periodic_setup(const qmlr_fchl19_params* p, const float* coords, const int32_t* elem, int32_t n_atoms,
                          const double* host_cell, const int64_t* env_ptr, const int32_t* env_atom,
                          const int32_t* env_shift, int32_t max_env, Cell9* cell) {
  int rc = validate_params(p);
  if (rc) return rc;
  QMLR_REQUIRE(n_atoms >= 0, "n_atoms must be >= 0");
  QMLR_REQUIRE(max_env >= 0 && max_env <= 2048, "max_env must be in 0..2048 (got %d)", max_env);
  QMLR_REQUIRE(host_cell, "host_cell is NULL");
  QMLR_REQUIRE(n_atoms == 0 || (coords && elem && env_ptr && (max_env == 0 || (env_atom && env_shift))),
               "NULL pointer argument");
  for (int k = 0; k < 9; ++k) {
    QMLR_REQUIRE(std::isfinite(host_cell[k]), "cell entries must be finite");
    cell->a[k] = host_cell[k];
  }
  return QMLR_OK;
}

extern "C" int qmlr_fchl19_periodic(const float* coords, const int32_t* elem, int32_t n_atoms, const double* host_cell,
                                    const int64_t* env_ptr, const int32_t* env_atom, const int32_t* env_shift,
                                    int32_t max_env, const qmlr_fchl19_params* p, float* rep, int32_t rep_ld,
                                    void* stream) {
  Cell9 cell;
  int rc = periodic_setup(p, coords, elem, n_atoms, host_cell, env_ptr, env_atom, env_shift, max_env, &cell);
  if (rc) return rc;
  const int rd = rep_dim_of(*p);
  QMLR_REQUIRE(rep_ld >= rd, "rep_ld (%d) < rep_dim (%d)", rep_ld, rd);
  QMLR_REQUIRE(p->n_el <= 5 && p->n2 <= 32 && p->n3 <= 32,
               "the periodic kernels support n_el <= 5 and radial grids of at most 32 points");
  if (n_atoms == 0) return QMLR_OK;
  QMLR_REQUIRE(rep, "rep is NULL");
  const Fchl19Consts c = make_consts(*p);
  const int envp = (std::max(max_env, 1) + 3) & ~3;
  const size_t smem = kWarpsFwd * reg_warp_bytes(envp);
  QMLR_REQUIRE(smem <= 227 * 1024, "max_env too large for shared memory");
  QMLR_CUDA_TRY(smem_attr_once((const void*)fchl19_periodic_kernel, (int)smem));
  fchl19_periodic_kernel<<<(n_atoms + kWarpsFwd - 1) / kWarpsFwd, 32 * kWarpsFwd, smem, as_stream(stream)>>>(
      coords, elem, n_atoms, cell, env_ptr, env_atom, env_shift, max_env, envp, c, rep, rep_ld, device_error_ptr());
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

extern "C" int qmlr_fchl19_periodic_vjp(const float* coords, const int32_t* elem, int32_t n_atoms,
                                        const double* host_cell, const int64_t* env_ptr, const int32_t* env_atom,
                                        const int32_t* env_shift, int32_t max_env, const qmlr_fchl19_params* p,
                                        const float* grad_rep, int32_t rep_ld, const int64_t* rev_ptr,
                                        const int64_t* rev_entry, float* contrib, float scale, float* grad_coords,
                                        int32_t accumulate, void* stream) {
  Cell9 cell;
  int rc = periodic_setup(p, coords, elem, n_atoms, host_cell, env_ptr, env_atom, env_shift, max_env, &cell);
  if (rc) return rc;
  const int rd = rep_dim_of(*p);
  QMLR_REQUIRE(rep_ld >= rd, "rep_ld (%d) < rep_dim (%d)", rep_ld, rd);
  if (n_atoms == 0) return QMLR_OK;
  QMLR_REQUIRE(grad_rep && rev_ptr && (max_env == 0 || rev_entry) && contrib && grad_coords,
               "NULL pointer argument");
  const Fchl19Consts c = make_consts(*p);
  const int rp = rep_pad_of(rd);
  const int envp = (std::max(max_env, 1) + 3) & ~3;
  const size_t smem = kWarpsVjp * vjp_warp_bytes(envp + 4, rp);
  QMLR_REQUIRE(smem <= 227 * 1024, "max_env too large for shared memory");
  QMLR_CUDA_TRY(smem_attr_once((const void*)fchl19_periodic_vjp_kernel, (int)smem));
  cudaStream_t st = as_stream(stream);
  fchl19_periodic_vjp_kernel<<<(n_atoms + kWarpsVjp - 1) / kWarpsVjp, 32 * kWarpsVjp, smem, st>>>(
      coords, elem, n_atoms, cell, env_ptr, env_atom, env_shift, max_env, envp, c, grad_rep, rep_ld, contrib,
      device_error_ptr());
  QMLR_LAUNCH_CHECK();
  periodic_reduce_kernel<<<(3 * n_atoms + 255) / 256, 256, 0, st>>>(n_atoms, env_ptr, rev_ptr, rev_entry, contrib,
                                                                    scale, accumulate, grad_coords);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}
