// Trained-model handle and energy + force prediction (sm_103a).
//
// Atomic energy partition of the paper (RFF section): E = sum_I alpha^T
// z(rho_I); forces F = -dE/dr by the backward passes of SORF and FCHL19
// (Computational Details: forces summed on chip; on-device component split in
// the timings section). The handle owns device copies of U_e, the SORF signs
// and phases and alpha, plus a workspace sized by qmlr_model_reserve, so that
// qmlr_predict_ef itself allocates nothing (it can be captured in a CUDA
// graph). Pipeline per call, all on the caller's stream:
//   FCHL19 -> group by element -> projection -> SORF energy + dE/dx (one CTA
//   per atom) -> transposed projection -> FCHL19 VJP (one warp per centre,
//   ordered reduction with scale -1, so F = -grad directly).
#include "common.cuh"

#include "model_internal.cuh"

#include <vector>

namespace qmlr {

// smallest batch (atoms) whose SORF energies + gradients run on the tensor cores
constexpr int kSorfTcMinAtoms = 8192;

void PredictWorkspace::release() {
  cudaFree(atom_e);
  cudaFree(pair_ptr);
  cudaFree(contrib);
  atom_e = nullptr;
  pair_ptr = nullptr;
  contrib = nullptr;
  cap_mols = 0;
  cudaFree(rep);
  cudaFree(x);
  cudaFree(gx);
  cudaFree(grep);
  cudaFree(perm);
  cudaFree(offs);
  cudaFree(gwork);
  cudaFree(sorf_work);
  sorf_work = nullptr;
  sorf_work_bytes = 0;
  rep = x = gx = grep = nullptr;
  perm = offs = nullptr;
  gwork = nullptr;
  cap_atoms = 0;
}

int PredictWorkspace::reserve(const qmlr_model* m, int max_atoms) {
  if (max_atoms <= cap_atoms && offs) return QMLR_OK;
  release();
  const size_t n = (size_t)std::max(max_atoms, 1);
  gwork_bytes = qmlr_group_workspace_bytes(max_atoms);
  cudaError_t e = cudaMalloc(&rep, n * m->rep_ld * 4);
  if (e == cudaSuccess) e = cudaMalloc(&x, n * m->d * 4);
  if (e == cudaSuccess) e = cudaMalloc(&gx, (size_t)m->n_part * n * m->d * 4);
  if (e == cudaSuccess) e = cudaMalloc(&grep, n * m->rep_ld * 4);
  if (e == cudaSuccess) e = cudaMalloc(&perm, n * 4);
  if (e == cudaSuccess) e = cudaMalloc(&offs, 16 * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&gwork, gwork_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&atom_e, (size_t)m->n_part * n * 8);
  if (e == cudaSuccess) e = cudaMalloc(&pair_ptr, (n + 4096 + 1) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&contrib, n * (size_t)m->max_mol_atoms * 3 * 4);
  if (e == cudaSuccess && m->sorf_tables) {
    sorf_work_bytes = sorf_tc_work_bytes((int)n, m->n_features);
    e = cudaMalloc(&sorf_work, sorf_work_bytes);
  }
  if (e != cudaSuccess) {
    release();
    set_error("workspace allocation failed: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? QMLR_ENOMEM : QMLR_ECUDA;
  }
  cap_atoms = max_atoms;
  cap_mols = max_atoms + 4096;
  return QMLR_OK;
}

size_t PredictWorkspace::bytes_per_atom(const qmlr_model* m) {
  return (size_t)m->rep_ld * 8 + (size_t)m->d * 4 * (1 + m->n_part) + 4 + 64 + 8 * m->n_part + 8 +
         (size_t)m->max_mol_atoms * 12 + (m->sorf_tables ? (size_t)m->d * 4 + 4 : 0);
}

int predict_ef_ws(const qmlr_model* m, PredictWorkspace& w, const float* coords, const int32_t* elem,
                  const int32_t* mol_ptr, int n_mol, int n_atoms, double* energies, float* forces,
                  cudaStream_t s) {
  QMLR_REQUIRE(n_atoms >= 0 && n_mol >= 0, "negative sizes");
  QMLR_REQUIRE(n_atoms <= w.cap_atoms,
               "batch of %d atoms exceeds the reserved capacity %d (call qmlr_model_reserve)", n_atoms,
               w.cap_atoms);
  QMLR_REQUIRE(energies || n_mol == 0, "energies is NULL");
  if (n_mol == 0) return QMLR_OK;
  int rc;
  if (n_atoms == 0) {
    QMLR_CUDA_TRY(cudaMemsetAsync(energies, 0, sizeof(double) * n_mol, s));
    return QMLR_OK;
  }
  if ((rc = predict_features_ws(m, w, coords, elem, mol_ptr, n_mol, n_atoms, s))) return rc;
  return predict_from_features_ws(m, w, coords, elem, mol_ptr, n_mol, n_atoms, energies, forces, s);
}

int predict_features_ws(const qmlr_model* m, PredictWorkspace& w, const float* coords, const int32_t* elem,
                        const int32_t* mol_ptr, int n_mol, int n_atoms, cudaStream_t s) {
  void* stream = s;
  int rc;
  const int n_el = m->p.n_el;
  if (m->timing) QMLR_CUDA_TRY(cudaEventRecord(m->tev[0], s));
  if ((rc = qmlr_fchl19(coords, elem, mol_ptr, n_mol, n_atoms, m->max_mol_atoms, &m->p, w.rep, m->rep_ld, stream)))
    return rc;
  if (m->timing) QMLR_CUDA_TRY(cudaEventRecord(m->tev[1], s));
  if ((rc = qmlr_group_by_element(elem, n_atoms, n_el, w.perm, w.offs, w.gwork, w.gwork_bytes, stream)))
    return rc;
  rc = proj_tc_launch(w.rep, m->rep_ld, m->rep_dim, 1, 0, m->Ufwd, m->d, w.perm, w.offs, n_atoms, n_el, w.x,
                      m->d, m->d, s);
  if (m->timing) QMLR_CUDA_TRY(cudaEventRecord(m->tev[2], s));
  return rc;
}

int predict_from_features_ws(const qmlr_model* m, PredictWorkspace& w, const float* coords, const int32_t* elem,
                             const int32_t* mol_ptr, int n_mol, int n_atoms, double* energies, float* forces,
                             cudaStream_t s) {
  void* stream = s;
  int rc;
  const int n_el = m->p.n_el;
  QMLR_REQUIRE(n_mol <= w.cap_mols, "batch of %d molecules exceeds the reserved capacity %d", n_mol, w.cap_mols);
  if (m->timing) QMLR_CUDA_TRY(cudaEventRecord(m->tev[3], s));
  // gradient partials: one per 128-stack part of the FWHT kernel, one of the tensor-core kernel
  int g_parts = m->n_part;
  // the tensor-core form walks a 128-atom tile's 2 N_F/128 half stacks in one CTA
  // (~0.4 ms at N_F = 16384): small batches are faster on the FWHT kernel
  if (forces && m->sorf_tc && n_atoms >= kSorfTcMinAtoms) {
    if ((rc = sorf_tc_energy_grad(w.x, n_atoms, m->sorf_tables, m->T, m->b, m->alpha, m->n_features, m->sigma,
                                  w.atom_e, w.gx, w.sorf_work, w.sorf_work_bytes, s)))
      return rc;
    if ((rc = sorf_segment_energy(w.atom_e, 1, n_atoms, mol_ptr, n_mol, energies, s))) return rc;
    g_parts = 1;
  } else if ((rc = sorf_energy_grad_model(w.x, m->d, mol_ptr, n_mol, n_atoms, m->signs, m->T, m->bT,
                                          m->n_features, m->sigma, m->alphaT, w.atom_e, energies,
                                          forces ? w.gx : nullptr, s))) {
    return rc;
  }
  if (m->timing) QMLR_CUDA_TRY(cudaEventRecord(m->tev[4], s));
  if (!forces) return QMLR_OK;
  if ((rc = proj_tc_launch(w.gx, m->d, m->d, g_parts, (long)n_atoms * m->d, m->Utrn, m->rep_dim, w.perm, w.offs,
                           n_atoms, n_el, w.grep, m->rep_ld, m->rep_ld, s)))
    return rc;
  if (m->timing) QMLR_CUDA_TRY(cudaEventRecord(m->tev[5], s));
  if ((rc = qmlr_jac_offsets(mol_ptr, n_mol, w.pair_ptr, nullptr, stream))) return rc;
  // forces F = -dE/dr: scale -1 in the ordered reduction
  rc = qmlr_fchl19_vjp_atoms(coords, elem, mol_ptr, n_mol, n_atoms, m->max_mol_atoms, &m->p, w.grep,
                             m->rep_ld, w.pair_ptr, w.contrib, -1.0f, forces, 0, stream);
  if (m->timing) QMLR_CUDA_TRY(cudaEventRecord(m->tev[6], s));
  return rc;
}

}  // namespace qmlr

using namespace qmlr;

extern "C" int qmlr_model_create(const qmlr_fchl19_params* p, int32_t max_mol_atoms, const float* host_U,
                                 int32_t d, const uint32_t* host_sign_bits, int32_t T, const float* host_b,
                                 int32_t n_features, double sigma, const float* host_alpha,
                                 qmlr_model** out) {
  int rc = validate_params(p);
  if (rc) return rc;
  QMLR_REQUIRE(out && host_U && host_sign_bits && host_b && host_alpha, "NULL pointer argument");
  QMLR_REQUIRE(d == 16 || d == 32 || d == 64 || d == 128, "d must be 16, 32, 64 or 128");
  QMLR_REQUIRE(T >= 1 && T <= 4, "T must be in 1..4");
  QMLR_REQUIRE(n_features >= d && n_features % d == 0, "n_features must be a multiple of d");
  QMLR_REQUIRE(max_mol_atoms >= 1 && max_mol_atoms <= 256, "max_mol_atoms must be in 1..256");
  QMLR_REQUIRE(sigma > 0, "sigma must be > 0");
  qmlr_model* m = new qmlr_model();
  m->p = *p;
  m->max_mol_atoms = max_mol_atoms;
  m->rep_dim = rep_dim_of(*p);
  m->rep_ld = (m->rep_dim + 3) & ~3;
  m->d = d;
  m->T = T;
  m->n_features = n_features;
  m->sigma = sigma;
  m->n_part = qmlr_sorf_parts(n_features, d);
  const int W = (d + 31) / 32;
  const size_t nU = (size_t)p->n_el * m->rep_dim * d;
  const size_t nS = (size_t)(n_features / d) * T * W;
  cudaError_t e = cudaSuccess;
  e = cudaMalloc(&m->U, nU * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->signs, nS * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->b, (size_t)n_features * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->alpha, (size_t)n_features * 4);
  if (e == cudaSuccess) e = cudaMemcpy(m->U, host_U, nU * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->signs, host_sign_bits, nS * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->b, host_b, (size_t)n_features * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->alpha, host_alpha, (size_t)n_features * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&m->bT, (size_t)n_features * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->alphaT, (size_t)n_features * 4);
  if (e == cudaSuccess) {
    const int ns = n_features / d;
    std::vector<float> t1((size_t)n_features), t2((size_t)n_features);
    for (int st = 0; st < ns; ++st)
      for (int i = 0; i < d; ++i) {
        t1[(size_t)i * ns + st] = host_b[(size_t)st * d + i];
        t2[(size_t)i * ns + st] = host_alpha[(size_t)st * d + i];
      }
    e = cudaMemcpy(m->bT, t1.data(), (size_t)n_features * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->alphaT, t2.data(), (size_t)n_features * 4, cudaMemcpyHostToDevice);
  }
  const size_t bf = proj_tc_basis_bytes(p->n_el, m->rep_dim, d), bt = proj_tc_basis_bytes(p->n_el, d, m->rep_dim);
  if (e == cudaSuccess) e = cudaMalloc(&m->Ufwd, bf);
  if (e == cudaSuccess) e = cudaMalloc(&m->Utrn, bt);
  if (e != cudaSuccess) {
    set_error("model allocation/copy failed: %s", cudaGetErrorString(e));
    qmlr_model_destroy(m);
    return e == cudaErrorMemoryAllocation ? QMLR_ENOMEM : QMLR_ECUDA;
  }
  if (e == cudaSuccess && sorf_tc_supported(d, T, n_features)) {
    e = cudaMalloc(&m->sorf_tables, sorf_tc_table_bytes(n_features));
    m->sorf_tc = e == cudaSuccess;
  }
  if (e != cudaSuccess) {
    set_error("model allocation failed: %s", cudaGetErrorString(e));
    qmlr_model_destroy(m);
    return e == cudaErrorMemoryAllocation ? QMLR_ENOMEM : QMLR_ECUDA;
  }
  rc = m->sorf_tables ? sorf_tc_tables(m->signs, T, n_features, m->sorf_tables, 0) : QMLR_OK;
  if (rc == QMLR_OK) rc = proj_tc_split_basis(m->U, p->n_el, m->rep_dim, d, (long)m->rep_dim * d, d, false, m->Ufwd, 0);
  if (rc == QMLR_OK) rc = proj_tc_split_basis(m->U, p->n_el, d, m->rep_dim, (long)m->rep_dim * d, d, true, m->Utrn, 0);
  if (rc == QMLR_OK && cudaStreamSynchronize(0) != cudaSuccess) {
    set_error("splitting the model basis failed");
    rc = QMLR_ECUDA;
  }
  if (rc) {
    qmlr_model_destroy(m);
    return rc;
  }
  *out = m;
  return QMLR_OK;
}

extern "C" int qmlr_model_destroy(qmlr_model* m) {
  if (!m) return QMLR_OK;
  m->ws.release();
  cudaFree(m->U);
  cudaFree(m->signs);
  cudaFree(m->b);
  cudaFree(m->alpha);
  cudaFree(m->bT);
  cudaFree(m->alphaT);
  cudaFree(m->Ufwd);
  cudaFree(m->Utrn);
  cudaFree(m->sorf_tables);
  for (int k = 0; k < 8; ++k)
    if (m->tev[k]) cudaEventDestroy(m->tev[k]);
  delete m;
  return QMLR_OK;
}

extern "C" int qmlr_model_set_alpha(qmlr_model* m, const float* host_alpha) {
  QMLR_REQUIRE(m && host_alpha, "NULL pointer argument");
  QMLR_CUDA_TRY(cudaMemcpy(m->alpha, host_alpha, (size_t)m->n_features * 4, cudaMemcpyHostToDevice));
  const int ns = m->n_features / m->d;
  std::vector<float> t((size_t)m->n_features);
  for (int st = 0; st < ns; ++st)
    for (int i = 0; i < m->d; ++i) t[(size_t)i * ns + st] = host_alpha[(size_t)st * m->d + i];
  QMLR_CUDA_TRY(cudaMemcpy(m->alphaT, t.data(), (size_t)m->n_features * 4, cudaMemcpyHostToDevice));
  return QMLR_OK;
}

namespace qmlr {
// b[i] = float(a[i]); bT[(i % d) * n_stack + i / d] = float(a[i])  (natural and stack-minor copies)
__global__ void f64_to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, float* __restrict__ bT,
                                  int n, int d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float v = (float)a[i];
    b[i] = v;
    bT[(long)(i % d) * (n / d) + i / d] = v;
  }
}
}  // namespace qmlr

extern "C" int qmlr_model_set_alpha_device(qmlr_model* m, const double* alpha, void* stream) {
  QMLR_REQUIRE(m && alpha, "NULL pointer argument");
  f64_to_f32_kernel<<<(m->n_features + 255) / 256, 256, 0, as_stream(stream)>>>(alpha, m->alpha, m->alphaT,
                                                                                m->n_features, m->d);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

extern "C" int qmlr_model_reserve(qmlr_model* m, int32_t max_atoms) {
  QMLR_REQUIRE(m && max_atoms >= 0, "bad arguments");
  return m->ws.reserve(m, max_atoms);
}

extern "C" int qmlr_predict_ef(qmlr_model* m, const float* coords, const int32_t* elem,
                               const int32_t* mol_ptr, int32_t n_mol, int32_t n_atoms,
                               double* energies, float* forces, void* stream) {
  QMLR_REQUIRE(m, "model is NULL");
  return predict_ef_ws(m, m->ws, coords, elem, mol_ptr, n_mol, n_atoms, energies, forces, as_stream(stream));
}

static int check_batch(const qmlr_model* m, int n_mol, int n_atoms) {
  QMLR_REQUIRE(n_atoms >= 1 && n_mol >= 1, "the split prediction needs a non-empty batch");
  QMLR_REQUIRE(n_atoms <= m->ws.cap_atoms,
               "batch of %d atoms exceeds the reserved capacity %d (call qmlr_model_reserve)", n_atoms,
               m->ws.cap_atoms);
  return QMLR_OK;
}

extern "C" int qmlr_predict_features(qmlr_model* m, const float* coords, const int32_t* elem,
                                     const int32_t* mol_ptr, int32_t n_mol, int32_t n_atoms, void* stream) {
  QMLR_REQUIRE(m, "model is NULL");
  int rc = check_batch(m, n_mol, n_atoms);
  if (rc) return rc;
  return predict_features_ws(m, m->ws, coords, elem, mol_ptr, n_mol, n_atoms, as_stream(stream));
}

extern "C" int qmlr_predict_ef_from_features(qmlr_model* m, const float* coords, const int32_t* elem,
                                             const int32_t* mol_ptr, int32_t n_mol, int32_t n_atoms,
                                             double* energies, float* forces, void* stream) {
  QMLR_REQUIRE(m, "model is NULL");
  QMLR_REQUIRE(energies, "energies is NULL");
  int rc = check_batch(m, n_mol, n_atoms);
  if (rc) return rc;
  return predict_from_features_ws(m, m->ws, coords, elem, mol_ptr, n_mol, n_atoms, energies, forces,
                                  as_stream(stream));
}

// d(sum_m g[m] E_m) / d r_k = -g[mol(k)] F_k (each atom is in one molecule).
__global__ void energy_vjp_kernel(const float* __restrict__ F, const int32_t* __restrict__ mol_ptr, int n_mol,
                                  int n_atoms, const double* __restrict__ g, float* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * n_atoms) return;
  const int atom = t / 3;
  int lo = 0, hi = n_mol;   // mol_ptr[lo] <= atom < mol_ptr[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (mol_ptr[mid] <= atom) lo = mid; else hi = mid;
  }
  out[t] = (float)(-g[lo] * (double)F[t]);
}

extern "C" int qmlr_energy_vjp(const float* forces, const int32_t* mol_ptr, int32_t n_mol, int32_t n_atoms,
                               const double* grad_E, float* grad_coords, void* stream) {
  QMLR_REQUIRE(n_mol >= 0 && n_atoms >= 0, "negative sizes");
  if (n_atoms == 0) return QMLR_OK;
  QMLR_REQUIRE(n_mol >= 1, "n_atoms > 0 but n_mol == 0");
  QMLR_REQUIRE(forces && mol_ptr && grad_E && grad_coords, "NULL pointer argument");
  energy_vjp_kernel<<<(3 * n_atoms + 255) / 256, 256, 0, as_stream(stream)>>>(forces, mol_ptr, n_mol, n_atoms,
                                                                              grad_E, grad_coords);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

extern "C" int qmlr_model_set_sorf_tc(qmlr_model* m, int32_t enable) {
  QMLR_REQUIRE(m, "model is NULL");
  QMLR_REQUIRE(!enable || m->sorf_tables,
               "the tensor-core SORF kernel needs d = 128 and T <= 3 (this model: d = %d, T = %d)", m->d, m->T);
  m->sorf_tc = enable != 0;
  return QMLR_OK;
}

extern "C" int32_t qmlr_model_sorf_tc(const qmlr_model* m) { return m && m->sorf_tc ? 1 : 0; }

extern "C" int qmlr_model_set_timing(qmlr_model* m, int32_t enable) {
  QMLR_REQUIRE(m, "model is NULL");
  if (enable && !m->tev[0])
    for (int k = 0; k < 8; ++k) QMLR_CUDA_TRY(cudaEventCreate(&m->tev[k]));
  m->timing = enable != 0;
  return QMLR_OK;
}

extern "C" int qmlr_model_timings(qmlr_model* m, float* host_ms, int32_t n) {
  QMLR_REQUIRE(m && host_ms && n >= 0, "bad arguments");
  QMLR_REQUIRE(m->tev[0], "timing was never enabled on this model");
  const int pairs[5][2] = {{0, 1}, {1, 2}, {3, 4}, {4, 5}, {5, 6}};
  for (int k = 0; k < std::min(n, 5); ++k) {
    QMLR_CUDA_TRY(cudaEventSynchronize(m->tev[pairs[k][1]]));
    QMLR_CUDA_TRY(cudaEventElapsedTime(&host_ms[k], m->tev[pairs[k][0]], m->tev[pairs[k][1]]));
  }
  return QMLR_OK;
}
