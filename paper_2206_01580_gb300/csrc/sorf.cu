// SORF feature map: forward, segment sum into Z, energies and the backward
// pass to the projected representations (sm_103a).
//
// SORF section of the paper: W x = (sqrt(d)/sigma) [H D_t]_{t=1..T} x for each
// of N_F/d independent stacks, z = sqrt(2/N_F) cos(W x + b). The fast
// Walsh-Hadamard transform replaces the dense product (O(d log d) per stack).
//
// Design (GB300): one thread owns one (atom, stack) pair and keeps the whole
// d-vector in registers (d <= 128): the d log2 d butterflies run with no
// shuffles and no shared memory, sign flips are XORs of the IEEE sign bit,
// and the Hadamard normalisation is folded into one scale at the end. A CTA
// holds up to 128 stacks of one molecule and walks the molecule's atoms in
// order, so the segment sum Z_m = sum_I z_I (and E_m = sum_I alpha^T z_I)
// is formed on chip in a fixed order: deterministic, no atomics, z never
// written to HBM. The backward pass applies the transposed chain
// (H symmetric, D diagonal) to -sqrt(2/N_F) alpha sin(u) and reduces over the
// CTA's stacks in shared memory.
#include "sorf_math.cuh"

namespace qmlr {

constexpr int kStacksPerCta = 128;

enum SorfMode { M_PER_ATOM = 0, M_PER_MOL = 1, M_ENERGY = 2, M_ENERGY_GRAD = 3, M_SIN_T = 4 };

// One warp checks the staged x of an atom against x2max; a non-finite or
// too-long x is recorded as DEV_RANGE.
template <int D>
__device__ __forceinline__ void check_range(const float* xs, float x2max, int lane, int* err) {
  float q = 0.f;
#pragma unroll
  for (int i = lane; i < D; i += 32) q = fmaf(xs[i], xs[i], q);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
  if (lane == 0 && !(q <= x2max)) record_device_error(err, DEV_RANGE);
}

struct SorfArgs {
  const float* x;
  const int32_t* mol_ptr;
  const uint32_t* sign_bits;
  const float* b;
  const float* alpha;
  void* out;
  float* gx;
  int n_atoms, n_stack, T, n_features, n_part;
  float scale;  // (sqrt(d)/sigma) / d^{T/2}
  float pref;   // sqrt(2/N_F)
  float x2max;  // largest |x|^2 of an atom whose phases the reduction handles exactly
  int* err;     // device error word
  // layout of b and alpha: element (stack s, index i) at s*sstr + i*istr
  // (natural order: sstr = d, istr = 1; stack-minor: sstr = 1, istr = n_stack)
  long sstr = 0, istr = 1;
};

template <int D, int MODE>
__global__ void __launch_bounds__(kStacksPerCta)
sorf_kernel(SorfArgs a) {
  constexpr int W = (D + 31) / 32;
  extern __shared__ __align__(16) float smem[];
  float* xs = smem;                                     // [D] current atom
  uint32_t* sg = reinterpret_cast<uint32_t*>(xs + D);    // [T*W][blockDim]
  float* work = reinterpret_cast<float*>(sg + a.T * W * blockDim.x);  // mode-specific
  const int tid = threadIdx.x, nt = blockDim.x;
  const int part = blockIdx.y;
  const int s = part * kStacksPerCta + tid;
  const bool active = s < a.n_stack;
  const int m = blockIdx.x;
  const int a0 = a.mol_ptr[m], a1 = a.mol_ptr[m + 1];

  for (int k = 0; k < a.T * W; ++k)
    sg[k * nt + tid] = active ? __ldg(a.sign_bits + ((long)s * a.T) * W + k) : 0u;
  if (MODE == M_PER_MOL)
    for (int i = 0; i < D; ++i) work[i * (nt + 1) + tid] = 0.f;

  const float* bs = a.b + (long)(active ? s : 0) * D;
  const float* as = (MODE == M_ENERGY || MODE == M_ENERGY_GRAD) ? a.alpha + (long)(active ? s : 0) * D : nullptr;
  // (this kernel reads b and alpha in natural order)
  double e_acc = 0.0;

  for (int atom = a0; atom < a1; ++atom) {
    __syncthreads();
    for (int i = tid; i < D; i += nt) xs[i] = __ldg(a.x + (long)atom * D + i);
    __syncthreads();
    if (tid < 32 && part == 0) check_range<D>(xs, a.x2max, tid, a.err);
    float v[D];
#pragma unroll
    for (int i = 0; i < D; ++i) v[i] = xs[i];
    for (int t = 0; t < a.T; ++t) {
      uint32_t w[W];
#pragma unroll
      for (int q = 0; q < W; ++q) w[q] = sg[(t * W + q) * nt + tid];
      flip<D>(v, w);
      fwht<D>(v);
    }
    if (MODE == M_SIN_T) {
      // out[atom][i][s] = sqrt(2/N_F) sin(u_i): stacks contiguous (coalesced across the warp)
      if (active) {
        float* o = static_cast<float*>(a.out) + (long)atom * a.n_features + s;
#pragma unroll
        for (int i = 0; i < D; ++i) o[(long)i * a.n_stack] = a.pref * fast_sin(fmaf(v[i], a.scale, __ldg(bs + i)));
      }
    } else if (MODE == M_PER_ATOM) {
      if (active) {
        float* o = static_cast<float*>(a.out) + (long)atom * a.n_features + (long)s * D;
#pragma unroll
        for (int i = 0; i < D; ++i) o[i] = a.pref * fast_cos(fmaf(v[i], a.scale, __ldg(bs + i)));
      }
    } else if (MODE == M_PER_MOL) {
      if (active) {
#pragma unroll
        for (int i = 0; i < D; ++i)
          work[i * (nt + 1) + tid] += a.pref * fast_cos(fmaf(v[i], a.scale, __ldg(bs + i)));
      }
    } else if (MODE == M_ENERGY) {
      if (active) {
        float e = 0.f;
#pragma unroll
        for (int i = 0; i < D; ++i) e = fmaf(__ldg(as + i), fast_cos(fmaf(v[i], a.scale, __ldg(bs + i))), e);
        e_acc += (double)e;
      }
    } else {  // M_ENERGY_GRAD
      float e = 0.f;
      if (active) {
#pragma unroll
        for (int i = 0; i < D; ++i) {
          float sn, cs;
          fast_sincos(fmaf(v[i], a.scale, __ldg(bs + i)), &sn, &cs);
          const float al = __ldg(as + i);
          e = fmaf(al, cs, e);
          v[i] = -a.pref * a.scale * al * sn;   // dE/d(chain output)
        }
      } else {
#pragma unroll
        for (int i = 0; i < D; ++i) v[i] = 0.f;
      }
      e_acc += (double)e;
      for (int t = a.T - 1; t >= 0; --t) {
        uint32_t w[W];
#pragma unroll
        for (int q = 0; q < W; ++q) w[q] = sg[(t * W + q) * nt + tid];
        fwht<D>(v);
        flip<D>(v, w);
      }
      // reduce over the CTA's stacks: work[tid][D+1]
#pragma unroll
      for (int i = 0; i < D; ++i) work[tid * (D + 1) + i] = v[i];
      __syncthreads();
      for (int i = tid; i < D; i += nt) {
        float sum = 0.f;
        for (int k = 0; k < nt; ++k) sum += work[k * (D + 1) + i];
        a.gx[((long)part * a.n_atoms + atom) * D + i] = sum;
      }
    }
  }

  if (MODE == M_PER_MOL) {
    __syncthreads();
    // Z[m][part*128*D + tid_stack*D + i]: consecutive threads write consecutive features
    float* o = static_cast<float*>(a.out) + (long)m * a.n_features + (long)part * kStacksPerCta * D;
    const int nf = min(nt, a.n_stack - part * kStacksPerCta) * D;
    for (int f = tid; f < nf; f += nt) o[f] = work[(f % D) * (nt + 1) + f / D];
  } else if (MODE == M_ENERGY || MODE == M_ENERGY_GRAD) {
    __syncthreads();
    double* red = reinterpret_cast<double*>(work);
    red[tid] = e_acc;
    __syncthreads();
    if (tid == 0) {
      double sum = 0.0;
      for (int k = 0; k < nt; ++k) sum += red[k];
      sum *= (double)a.pref;
      double* E = static_cast<double*>(a.out);
      if (a.n_part == 1) E[m] = sum;
      else atomicAdd(E + m, sum);
    }
  }
}

// Segment sum Z[m] = sqrt(2/N_F) sum_I cos(W x_I + b) with b stack-minor
// (b[i * n_stack + s]: a warp's loads of one index are contiguous). Thread =
// stack; its running sums live in shared memory as a padded row [D + 4] read
// and written as float4 (conflict-free), the atom's x is read as float4
// broadcasts, and sqrt(2/N_F) is applied once when Z is written.
template <int D>
__global__ void __launch_bounds__(kStacksPerCta, 3)
sorf_mol_kernel(SorfArgs a) {
  constexpr int W = (D + 31) / 32, LD = D + 4;
  extern __shared__ __align__(16) float smem[];
  float* xs = smem;                                      // [D]
  uint32_t* sg = reinterpret_cast<uint32_t*>(xs + D);    // [T*W][nt]
  const int tid = threadIdx.x, nt = blockDim.x;
  float* acc = reinterpret_cast<float*>(sg + a.T * W * nt);   // [nt][LD]
  const int part = blockIdx.y;
  const int s = part * kStacksPerCta + tid;
  const bool active = s < a.n_stack;
  const int m = blockIdx.x;
  const int a0 = a.mol_ptr[m], a1 = a.mol_ptr[m + 1];
  for (int k = 0; k < a.T * W; ++k)
    sg[k * nt + tid] = active ? __ldg(a.sign_bits + ((long)s * a.T) * W + k) : 0u;
  float4* row = reinterpret_cast<float4*>(acc + tid * LD);
#pragma unroll
  for (int q = 0; q < D / 4; ++q) row[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  const float* bs = a.b + (active ? s : 0);
  for (int atom = a0; atom < a1; ++atom) {
    __syncthreads();
    for (int i = tid; i < D / 4; i += nt)
      reinterpret_cast<float4*>(xs)[i] = __ldg(reinterpret_cast<const float4*>(a.x + (long)atom * D) + i);
    __syncthreads();
    if (tid < 32 && part == 0) check_range<D>(xs, a.x2max, tid, a.err);
    float v[D];
#pragma unroll
    for (int q = 0; q < D / 4; ++q) {
      const float4 x4 = reinterpret_cast<const float4*>(xs)[q];
      v[4 * q] = x4.x;
      v[4 * q + 1] = x4.y;
      v[4 * q + 2] = x4.z;
      v[4 * q + 3] = x4.w;
    }
    for (int t = 0; t < a.T; ++t) {
      uint32_t w[W];
#pragma unroll
      for (int q = 0; q < W; ++q) w[q] = sg[(t * W + q) * nt + tid];
      flip<D>(v, w);
      fwht<D>(v);
    }
    if (active) {
#pragma unroll
      for (int q = 0; q < D / 4; ++q) {
        float4 r = row[q];
        r.x += fast_cos(fmaf(v[4 * q], a.scale, __ldg(bs + (long)(4 * q) * a.n_stack)));
        r.y += fast_cos(fmaf(v[4 * q + 1], a.scale, __ldg(bs + (long)(4 * q + 1) * a.n_stack)));
        r.z += fast_cos(fmaf(v[4 * q + 2], a.scale, __ldg(bs + (long)(4 * q + 2) * a.n_stack)));
        r.w += fast_cos(fmaf(v[4 * q + 3], a.scale, __ldg(bs + (long)(4 * q + 3) * a.n_stack)));
        row[q] = r;
      }
    }
  }
  __syncthreads();
  // Z[m][part*128*D + stack*D + i]: consecutive threads write consecutive features
  float* o = static_cast<float*>(a.out) + (long)m * a.n_features + (long)part * kStacksPerCta * D;
  const int nf = min(nt, a.n_stack - part * kStacksPerCta) * D;
  for (int f = tid; f < nf; f += nt) o[f] = a.pref * acc[(f / D) * LD + f % D];
}

// bT[i * n_stack + s] = b[s * d + i]
__global__ void transpose_phases_kernel(const float* __restrict__ b, int d, int n_stack, float* __restrict__ bT) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= d * n_stack) return;
  const int s = f / d, i = f % d;
  bT[(long)i * n_stack + s] = b[f];
}

// ---------------------------------------------------------------------------
// Force rows of the energy+force normal equations (RFF section: derivative
// features dz/dr stacked under the energy rows). For molecule m, atom k, axis x:
//   row = -dZ_m/dr_{k,x} = sum_I sqrt(2/N_F) sin(u_I) (.) (W t_{I,k,x})
// with t_{I,k,x} = U_{e(I)}^T d rho_I / d r_{k,x} the projected Jacobian row and W
// the linear SORF map (sign flips, Hadamard chain, sqrt(d)/sigma scale). One
// thread per stack holds the tangent's d-vector in registers; the sum over
// centres I runs in order in a shared-memory accumulator.
template <int D>
__global__ void __launch_bounds__(kStacksPerCta)
force_rows_kernel(const float* __restrict__ tang, const int64_t* __restrict__ jac_ptr,
                  const int32_t* __restrict__ mol_ptr, const float* __restrict__ sin_t,
                  const uint32_t* __restrict__ sign_bits, int T, int n_stack, int n_features, float scale,
                  float* __restrict__ rows, long ld, long row0) {
  constexpr int W = (D + 31) / 32;
  constexpr int CH = 16;   // centres staged per round
  extern __shared__ __align__(16) float smem[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int part = blockIdx.y;
  const int sidx = part * kStacksPerCta + tid;
  const bool active = sidx < n_stack;
  const int m = blockIdx.x;
  const int a0 = mol_ptr[m], M = mol_ptr[m + 1] - a0;
  const long jb = jac_ptr[m];
  uint32_t* sg = reinterpret_cast<uint32_t*>(smem);                 // [T*W][nt]
  float* ts = reinterpret_cast<float*>(sg + T * W * nt);            // [CH][D] staged tangents
  float* acc = ts + CH * D;                                         // [D][nt+1]
  for (int k = 0; k < T * W; ++k) sg[k * nt + tid] = active ? __ldg(sign_bits + (long)sidx * T * W + k) : 0u;
  for (int kx = 0; kx < 3 * M; ++kx) {
    const int kl = kx / 3, x = kx % 3;
    __syncthreads();   // every thread has written out the previous row's columns of acc
    for (int i = 0; i < D; ++i) acc[i * (nt + 1) + tid] = 0.f;
    for (int c0 = 0; c0 < M; c0 += CH) {
      const int cn = min(CH, M - c0);
      __syncthreads();
      for (int q = tid; q < cn * D; q += nt) {
        const int ci = q / D, i = q % D;
        ts[q] = __ldg(tang + (jb + ((long)(c0 + ci) * M + kl) * 3 + x) * D + i);
      }
      __syncthreads();
      for (int ci = 0; ci < cn; ++ci) {
        float v[D];
#pragma unroll
        for (int i = 0; i < D; ++i) v[i] = ts[ci * D + i];
        for (int t = 0; t < T; ++t) {
          uint32_t w[W];
#pragma unroll
          for (int q = 0; q < W; ++q) w[q] = sg[(t * W + q) * nt + tid];
          flip<D>(v, w);
          fwht<D>(v);
        }
        if (active) {
          const float* sp = sin_t + (long)(a0 + c0 + ci) * n_features + sidx;
#pragma unroll
          for (int i = 0; i < D; ++i) acc[i * (nt + 1) + tid] += __ldg(sp + (long)i * n_stack) * v[i] * scale;
        }
      }
    }
    __syncthreads();
    float* o = rows + (row0 + (long)(a0 + kl) * 3 + x) * ld + (long)part * kStacksPerCta * D;
    const int nf = min(nt, n_stack - part * kStacksPerCta) * D;
    for (int f = tid; f < nf; f += nt) o[f] = acc[(f % D) * (nt + 1) + f / D];
  }
}

// ---------------------------------------------------------------------------
// Energy (and gradient) with one CTA per (atom, stack part): atoms of one
// molecule run in parallel. The atom's energy partial (FP64) is reduced over
// the CTA's stacks by warp shuffles and then over the warps in order, and goes
// to atom_e[part][atom]; molecule energies are then summed over atoms and
// parts in order by segment_energy_kernel. The gradient d-vectors of the
// stacks are reduce-scattered within each warp by shuffles (after the five
// halving steps lane l holds elements [l*D/32, (l+1)*D/32) summed over the
// warp) and the warps' partial vectors are added in order.

// One halving step of the warp reduce-scatter: lanes with the OFF bit set keep
// the upper half of v[0:N) and send the lower half, the others the reverse.
template <int D, int N, int OFF>
__device__ __forceinline__ void reduce_scatter_step(float (&v)[D], int lane) {
  const bool upper = (lane & OFF) != 0;
#pragma unroll
  for (int j = 0; j < N / 2; ++j) {
    const float send = upper ? v[j] : v[j + N / 2];
    const float keep = upper ? v[j + N / 2] : v[j];
    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
  }
}

template <int D, bool GRAD>
__global__ void __launch_bounds__(kStacksPerCta)
sorf_atom_kernel(SorfArgs a, double* __restrict__ atom_e) {
  constexpr int W = (D + 31) / 32;
  constexpr int NW = kStacksPerCta / 32;
  extern __shared__ __align__(16) float smem[];
  float* xs = smem;                                           // [D]
  double* red = reinterpret_cast<double*>(smem + D + 4);      // [NW]
  uint32_t* sg = reinterpret_cast<uint32_t*>(red + NW);       // [T*W][nt]
  float* work = reinterpret_cast<float*>(sg + 4 * W * kStacksPerCta);  // gradient partials
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int atom = blockIdx.x, part = blockIdx.y;
  const int s = part * kStacksPerCta + tid;
  const bool active = s < a.n_stack;
  for (int i = tid; i < D; i += nt) xs[i] = __ldg(a.x + (long)atom * D + i);
  for (int k = 0; k < a.T * W; ++k) sg[k * nt + tid] = active ? __ldg(a.sign_bits + (long)s * a.T * W + k) : 0u;
  __syncthreads();
  if (tid < 32 && part == 0) check_range<D>(xs, a.x2max, tid, a.err);
  float v[D];
#pragma unroll
  for (int i = 0; i < D; ++i) v[i] = xs[i];
  for (int t = 0; t < a.T; ++t) {
    uint32_t w[W];
#pragma unroll
    for (int q = 0; q < W; ++q) w[q] = sg[(t * W + q) * nt + tid];
    flip<D>(v, w);
    fwht<D>(v);
  }
  const float* bs = a.b + (long)(active ? s : 0) * a.sstr;
  const float* as = a.alpha + (long)(active ? s : 0) * a.sstr;
  float e = 0.f;
  if (active) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const float u = fmaf(v[i], a.scale, __ldg(bs + i * a.istr));
      const float al = __ldg(as + i * a.istr);
      if (GRAD) {
        float sn, cs;
        fast_sincos(u, &sn, &cs);
        e = fmaf(al, cs, e);
        v[i] = -a.pref * a.scale * al * sn;
      } else {
        e = fmaf(al, fast_cos(u), e);
      }
    }
  } else if (GRAD) {
#pragma unroll
    for (int i = 0; i < D; ++i) v[i] = 0.f;
  }
  double ed = (double)e;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ed += __shfl_xor_sync(0xffffffffu, ed, o);
  if (lane == 0) red[warp] = ed;
  if (GRAD) {
    for (int t = a.T - 1; t >= 0; --t) {
      uint32_t w[W];
#pragma unroll
      for (int q = 0; q < W; ++q) w[q] = sg[(t * W + q) * nt + tid];
      fwht<D>(v);
      flip<D>(v, w);
    }
    if constexpr (D >= 32) {
      reduce_scatter_step<D, D, 16>(v, lane);
      reduce_scatter_step<D, D / 2, 8>(v, lane);
      reduce_scatter_step<D, D / 4, 4>(v, lane);
      reduce_scatter_step<D, D / 8, 2>(v, lane);
      reduce_scatter_step<D, D / 16, 1>(v, lane);
      constexpr int PER = D / 32;
#pragma unroll
      for (int k = 0; k < PER; ++k) work[warp * D + lane * PER + k] = v[k];
    } else {
#pragma unroll
      for (int i = 0; i < D; ++i) work[tid * (D + 1) + i] = v[i];
    }
  }
  __syncthreads();
  if (tid == 0) {
    const int nw = (nt + 31) / 32;
    double sum = 0.0;
    for (int k = 0; k < nw; ++k) sum += red[k];
    atom_e[(long)part * a.n_atoms + atom] = sum * (double)a.pref;
  }
  if (GRAD) {
    const int nw = (nt + 31) / 32;
    for (int i = tid; i < D; i += nt) {
      float sum = 0.f;
      if constexpr (D >= 32) {
        for (int k = 0; k < nw; ++k) sum += work[k * D + i];
      } else {
        for (int k = 0; k < nt; ++k) sum += work[k * (D + 1) + i];
      }
      a.gx[((long)part * a.n_atoms + atom) * D + i] = sum;
    }
  }
}

// E[m] = sum over the molecule's atoms (in order) of sum over parts (in order).
__global__ void segment_energy_kernel(const double* __restrict__ atom_e, int n_part, int n_atoms,
                                      const int32_t* __restrict__ mol_ptr, int n_mol, double* __restrict__ E) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_mol) return;
  double sum = 0.0;
  for (int i = mol_ptr[m]; i < mol_ptr[m + 1]; ++i)
    for (int p = 0; p < n_part; ++p) sum += atom_e[(long)p * n_atoms + i];
  E[m] = sum;
}

int sorf_segment_energy(const double* atom_e, int n_part, int n_atoms, const int32_t* mol_ptr, int n_mol,
                        double* E, cudaStream_t s) {
  if (n_mol == 0) return QMLR_OK;
  segment_energy_kernel<<<(n_mol + 255) / 256, 256, 0, s>>>(atom_e, n_part, n_atoms, mol_ptr, n_mol, E);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

template <int D, bool GRAD>
static int launch_atoms(const SorfArgs& a, double* atom_e, int n_mol, double* E, cudaStream_t s) {
  const int nt = std::min(kStacksPerCta, ((a.n_stack + 31) / 32) * 32);
  constexpr int W = (D + 31) / 32;
  const size_t smem = (size_t)(D + 4) * 4 + (kStacksPerCta / 32) * 8 + (size_t)4 * W * kStacksPerCta * 4 +
                      (GRAD ? (D >= 32 ? (size_t)(kStacksPerCta / 32) * D * 4 : (size_t)nt * (D + 1) * 4) : 0);
  QMLR_CUDA_TRY(smem_attr_once((const void*)sorf_atom_kernel<D, GRAD>, 227 * 1024));
  if (a.n_atoms > 0) {
    dim3 grid(a.n_atoms, a.n_part);
    sorf_atom_kernel<D, GRAD><<<grid, nt, smem, s>>>(a, atom_e);
    QMLR_LAUNCH_CHECK();
  }
  segment_energy_kernel<<<(n_mol + 255) / 256, 256, 0, s>>>(atom_e, a.n_part, a.n_atoms, a.mol_ptr, n_mol, E);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

// Energies and (optionally) gradients, atoms in parallel. Internal entry used
// by qmlr_sorf_grad and the model's prediction (b/alpha layout from a.sstr/istr).
int sorf_energy_atoms(const SorfArgs& a, int d, double* atom_e, int n_mol, double* E, bool grad,
                      cudaStream_t s) {
  switch (d) {
    case 16: return grad ? launch_atoms<16, true>(a, atom_e, n_mol, E, s) : launch_atoms<16, false>(a, atom_e, n_mol, E, s);
    case 32: return grad ? launch_atoms<32, true>(a, atom_e, n_mol, E, s) : launch_atoms<32, false>(a, atom_e, n_mol, E, s);
    case 64: return grad ? launch_atoms<64, true>(a, atom_e, n_mol, E, s) : launch_atoms<64, false>(a, atom_e, n_mol, E, s);
    default: return grad ? launch_atoms<128, true>(a, atom_e, n_mol, E, s) : launch_atoms<128, false>(a, atom_e, n_mol, E, s);
  }
}

SorfArgs make_sorf_args(const float* x, int d, const int32_t* mol_ptr, int n_atoms, const uint32_t* sign_bits,
                        int T, const float* b, int n_features, double sigma, const float* alpha, float* gx,
                        bool stack_minor) {
  SorfArgs a;
  a.x = x;
  a.mol_ptr = mol_ptr;
  a.sign_bits = sign_bits;
  a.b = b;
  a.alpha = alpha;
  a.out = nullptr;
  a.gx = gx;
  a.n_atoms = n_atoms;
  a.n_stack = n_features / d;
  a.T = T;
  a.n_features = n_features;
  a.n_part = (a.n_stack + kStacksPerCta - 1) / kStacksPerCta;
  a.scale = (float)(sqrt((double)d) / sigma / pow((double)d, 0.5 * T));
  a.pref = (float)sqrt(2.0 / n_features);
  a.x2max = sorf_x2max(d, sigma);
  a.err = device_error_ptr();
  a.sstr = stack_minor ? 1 : d;
  a.istr = stack_minor ? a.n_stack : 1;
  return a;
}

// Energies and gradients for a model whose phases and weights are stored
// stack-minor (element (s, i) at i * n_stack + s: coalesced across the warp).
int sorf_energy_grad_model(const float* x, int d, const int32_t* mol_ptr, int n_mol, int n_atoms,
                           const uint32_t* sign_bits, int T, const float* bT, int n_features, double sigma,
                           const float* alphaT, double* atom_e, double* E, float* gx, cudaStream_t s) {
  SorfArgs a = make_sorf_args(x, d, mol_ptr, n_atoms, sign_bits, T, bT, n_features, sigma, alphaT, gx, true);
  return sorf_energy_atoms(a, d, atom_e, n_mol, E, gx != nullptr, s);
}

template <int D>
static size_t sorf_smem(int mode, int T, int nt) {
  constexpr int W = (D + 31) / 32;
  size_t base = (size_t)D * 4 + (size_t)T * W * nt * 4;
  size_t work = 0;
  if (mode == M_PER_MOL) work = (size_t)D * (nt + 1) * 4;
  if (mode == M_SIN_T) work = 0;
  if (mode == M_ENERGY) work = (size_t)nt * 8;
  if (mode == M_ENERGY_GRAD) work = std::max((size_t)nt * (D + 1) * 4, (size_t)nt * 8);
  return base + ((work + 15) & ~(size_t)15) + 16;
}

template <int D>
static int launch_mol(const SorfArgs& a0, int n_mol, cudaStream_t s) {
  constexpr int W = (D + 31) / 32;
  QMLR_REQUIRE((reinterpret_cast<uintptr_t>(a0.x) & 15) == 0, "x must be 16-byte aligned");
  const int nt = std::min(kStacksPerCta, ((a0.n_stack + 31) / 32) * 32);
  const size_t smem = (size_t)D * 4 + (size_t)a0.T * W * nt * 4 + (size_t)nt * (D + 4) * 4;
  QMLR_REQUIRE(smem <= 227 * 1024, "SORF shared memory request too large");
  QMLR_CUDA_TRY(smem_attr_once((const void*)sorf_mol_kernel<D>, 227 * 1024));
  // phases in stack-minor order for coalesced loads (stream-ordered scratch)
  const int nf = a0.n_stack * D;
  float* bT = nullptr;
  QMLR_CUDA_TRY(cudaMallocAsync(&bT, sizeof(float) * nf, s));
  transpose_phases_kernel<<<(nf + 255) / 256, 256, 0, s>>>(a0.b, D, a0.n_stack, bT);
  int rc = QMLR_OK;
  {
    cudaError_t e = cudaGetLastError();
    count_launch();
    if (e != cudaSuccess) {
      set_error("kernel launch failed: %s", cudaGetErrorString(e));
      rc = QMLR_ECUDA;
    }
  }
  if (rc == QMLR_OK) {
    SorfArgs a = a0;
    a.b = bT;
    dim3 grid(n_mol, a.n_part);
    sorf_mol_kernel<D><<<grid, nt, smem, s>>>(a);
    cudaError_t e = cudaGetLastError();
    count_launch();
    if (e != cudaSuccess) {
      set_error("kernel launch failed: %s", cudaGetErrorString(e));
      rc = QMLR_ECUDA;
    }
  }
  cudaFreeAsync(bT, s);
  return rc;
}

template <int D, int MODE>
static int launch_mode(const SorfArgs& a, int n_mol, cudaStream_t s) {
  if (MODE == M_PER_MOL) return launch_mol<D>(a, n_mol, s);
  const int nt = std::min(kStacksPerCta, ((a.n_stack + 31) / 32) * 32);
  const size_t smem = sorf_smem<D>(MODE, a.T, nt);
  QMLR_REQUIRE(smem <= 227 * 1024, "SORF shared memory request too large");
  QMLR_CUDA_TRY(smem_attr_once((const void*)sorf_kernel<D, MODE>, 227 * 1024));
  dim3 grid(n_mol, a.n_part);
  sorf_kernel<D, MODE><<<grid, nt, smem, s>>>(a);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

template <int D>
static int launch_d(const SorfArgs& a, int mode, int n_mol, cudaStream_t s) {
  switch (mode) {
    case M_PER_ATOM: return launch_mode<D, M_PER_ATOM>(a, n_mol, s);
    case M_PER_MOL: return launch_mode<D, M_PER_MOL>(a, n_mol, s);
    case M_ENERGY: return launch_mode<D, M_ENERGY>(a, n_mol, s);
    case M_SIN_T: return launch_mode<D, M_SIN_T>(a, n_mol, s);
    default: return launch_mode<D, M_ENERGY_GRAD>(a, n_mol, s);
  }
}

static int sorf_dispatch(const float* x, int d, const int32_t* mol_ptr, int n_mol, int n_atoms,
                         const uint32_t* sign_bits, int T, const float* b, int n_features,
                         double sigma, const float* alpha, int mode, void* out, float* gx,
                         void* stream) {
  QMLR_REQUIRE(d == 16 || d == 32 || d == 64 || d == 128, "d must be 16, 32, 64 or 128 (got %d)", d);
  QMLR_REQUIRE(T >= 1 && T <= 4, "T must be in 1..4 (got %d)", T);
  QMLR_REQUIRE(n_features >= d && n_features % d == 0, "n_features must be a positive multiple of d");
  QMLR_REQUIRE(sigma > 0, "sigma must be > 0");
  QMLR_REQUIRE(n_mol >= 0 && n_atoms >= 0, "negative sizes");
  if (n_mol == 0) return QMLR_OK;
  QMLR_REQUIRE(x && mol_ptr && sign_bits && b && out, "NULL pointer argument");
  QMLR_REQUIRE((mode != M_ENERGY && mode != M_ENERGY_GRAD) || alpha, "alpha is NULL");
  QMLR_REQUIRE(mode != M_ENERGY_GRAD || gx, "gx is NULL");
  SorfArgs a;
  a.x = x;
  a.mol_ptr = mol_ptr;
  a.sign_bits = sign_bits;
  a.b = b;
  a.alpha = alpha;
  a.out = out;
  a.gx = gx;
  a.n_atoms = n_atoms;
  a.n_stack = n_features / d;
  a.T = T;
  a.n_features = n_features;
  a.n_part = (a.n_stack + kStacksPerCta - 1) / kStacksPerCta;
  a.scale = (float)(sqrt((double)d) / sigma / pow((double)d, 0.5 * T));
  a.pref = (float)sqrt(2.0 / n_features);
  a.x2max = sorf_x2max(d, sigma);
  a.err = device_error_ptr();
  cudaStream_t s = as_stream(stream);
  if ((mode == M_ENERGY || mode == M_ENERGY_GRAD) && a.n_part > 1)
    QMLR_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double) * n_mol, s));
  switch (d) {
    case 16: return launch_d<16>(a, mode, n_mol, s);
    case 32: return launch_d<32>(a, mode, n_mol, s);
    case 64: return launch_d<64>(a, mode, n_mol, s);
    default: return launch_d<128>(a, mode, n_mol, s);
  }
}

}  // namespace qmlr

using namespace qmlr;

extern "C" int32_t qmlr_sorf_parts(int32_t n_features, int32_t d) {
  if (d <= 0 || n_features <= 0) return 0;
  return (n_features / d + kStacksPerCta - 1) / kStacksPerCta;
}

extern "C" int qmlr_sorf(const float* x, int32_t d, const int32_t* mol_ptr, int32_t n_mol,
                         int32_t n_atoms, const uint32_t* sign_bits, int32_t T, const float* b,
                         int32_t n_features, double sigma, const float* alpha, int32_t mode,
                         void* out, void* stream) {
  QMLR_REQUIRE(mode == QMLR_SORF_PER_ATOM || mode == QMLR_SORF_PER_MOL || mode == QMLR_SORF_ENERGY ||
                   mode == QMLR_SORF_SIN_T,
               "unknown SORF mode %d", mode);
  return sorf_dispatch(x, d, mol_ptr, n_mol, n_atoms, sign_bits, T, b, n_features, sigma, alpha,
                       mode, out, nullptr, stream);
}

template <int D>
static int launch_force_rows(const float* tang, const int64_t* jac_ptr, const int32_t* mol_ptr, int n_mol,
                             const float* sin_t, const uint32_t* sign_bits, int T, int n_features,
                             float scale, float* rows, long ld, long row0, cudaStream_t s) {
  constexpr int W = (D + 31) / 32;
  const int n_stack = n_features / D;
  const int nt = std::min(kStacksPerCta, ((n_stack + 31) / 32) * 32);
  const size_t smem = (size_t)T * W * nt * 4 + 16 * D * 4 + (size_t)D * (nt + 1) * 4;
  QMLR_REQUIRE(smem <= 227 * 1024, "force-row shared memory request too large");
  QMLR_CUDA_TRY(smem_attr_once((const void*)force_rows_kernel<D>, 227 * 1024));
  dim3 grid(n_mol, (n_stack + kStacksPerCta - 1) / kStacksPerCta);
  force_rows_kernel<D><<<grid, nt, smem, s>>>(tang, jac_ptr, mol_ptr, sin_t, sign_bits, T, n_stack,
                                              n_features, scale, rows, ld, row0);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

extern "C" int qmlr_force_rows(const float* tangents, int32_t d, const int64_t* jac_ptr,
                               const int32_t* mol_ptr, int32_t n_mol, const float* sin_t,
                               const uint32_t* sign_bits, int32_t T, int32_t n_features, double sigma,
                               float* rows, int64_t ld, int64_t row0, void* stream) {
  QMLR_REQUIRE(d == 16 || d == 32 || d == 64 || d == 128, "d must be 16, 32, 64 or 128 (got %d)", d);
  QMLR_REQUIRE(T >= 1 && T <= 4, "T must be in 1..4");
  QMLR_REQUIRE(n_features >= d && n_features % d == 0, "n_features must be a positive multiple of d");
  QMLR_REQUIRE(ld >= n_features && row0 >= 0 && sigma > 0, "bad row layout or sigma");
  if (n_mol == 0) return QMLR_OK;
  QMLR_REQUIRE(tangents && jac_ptr && mol_ptr && sin_t && sign_bits && rows, "NULL pointer argument");
  const float scale = (float)(sqrt((double)d) / sigma / pow((double)d, 0.5 * T));
  cudaStream_t s = as_stream(stream);
  switch (d) {
    case 16: return launch_force_rows<16>(tangents, jac_ptr, mol_ptr, n_mol, sin_t, sign_bits, T, n_features, scale, rows, ld, row0, s);
    case 32: return launch_force_rows<32>(tangents, jac_ptr, mol_ptr, n_mol, sin_t, sign_bits, T, n_features, scale, rows, ld, row0, s);
    case 64: return launch_force_rows<64>(tangents, jac_ptr, mol_ptr, n_mol, sin_t, sign_bits, T, n_features, scale, rows, ld, row0, s);
    default: return launch_force_rows<128>(tangents, jac_ptr, mol_ptr, n_mol, sin_t, sign_bits, T, n_features, scale, rows, ld, row0, s);
  }
}

extern "C" int qmlr_sorf_grad(const float* x, int32_t d, const int32_t* mol_ptr, int32_t n_mol,
                              int32_t n_atoms, const uint32_t* sign_bits, int32_t T, const float* b,
                              int32_t n_features, double sigma, const float* alpha, double* atom_energy,
                              double* energies, float* gx, void* stream) {
  QMLR_REQUIRE(d == 16 || d == 32 || d == 64 || d == 128, "d must be 16, 32, 64 or 128 (got %d)", d);
  QMLR_REQUIRE(T >= 1 && T <= 4, "T must be in 1..4 (got %d)", T);
  QMLR_REQUIRE(n_features >= d && n_features % d == 0, "n_features must be a positive multiple of d");
  QMLR_REQUIRE(sigma > 0, "sigma must be > 0");
  QMLR_REQUIRE(n_mol >= 0 && n_atoms >= 0, "negative sizes");
  if (n_mol == 0) return QMLR_OK;
  QMLR_REQUIRE(mol_ptr && energies && atom_energy, "NULL pointer argument");
  QMLR_REQUIRE(n_atoms == 0 || (x && sign_bits && b && alpha), "NULL pointer argument");
  SorfArgs a = make_sorf_args(x, d, mol_ptr, n_atoms, sign_bits, T, b, n_features, sigma, alpha, gx, false);
  return sorf_energy_atoms(a, d, atom_energy, n_mol, energies, gx != nullptr, as_stream(stream));
}
