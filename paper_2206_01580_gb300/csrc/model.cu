// Trained-model handle and energy + force prediction (sm_103a).
//
// Atomic energy partition of the paper (RFF section): E = sum_I alpha^T
// z(rho_I); forces F = -dE/dr by the backward passes of SORF and FCHL19
// (Computational Details: forces summed on chip; on-device component split in
// the timings section). The handle owns device copies of U_e, the SORF signs
// and phases and alpha, plus a workspace sized by qmlr_model_reserve, so that
// qmlr_predict_ef itself allocates nothing (it can be captured in a CUDA
// graph). Pipeline per call, all on the caller's stream:
//   FCHL19 -> group by element -> projection -> SORF energy + dE/dx
//   -> transposed projection -> FCHL19 VJP -> F = -grad.
#include "common.cuh"

struct qmlr_model {
  qmlr_fchl19_params p;
  int max_mol_atoms;
  int rep_dim, rep_ld, d, T, n_features, n_part;
  double sigma;
  float* U;          // [n_el][rep_dim][d]
  uint32_t* signs;   // [n_stack][T][W]
  float* b;          // [N_F]
  float* alpha;      // [N_F]
  // workspace
  int cap_atoms = 0;
  float* rep = nullptr;     // [cap][rep_ld]
  float* x = nullptr;       // [cap][d]
  float* gx = nullptr;      // [n_part][cap][d]
  float* grep = nullptr;    // [cap][rep_ld]
  int32_t* perm = nullptr;  // [cap]
  int32_t* offs = nullptr;  // [n_el+1]
  void* gwork = nullptr;
  int64_t gwork_bytes = 0;
};

namespace qmlr {

__global__ void negate_kernel(float* v, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = -v[i];
}

static void free_ws(qmlr_model* m) {
  cudaFree(m->rep);
  cudaFree(m->x);
  cudaFree(m->gx);
  cudaFree(m->grep);
  cudaFree(m->perm);
  cudaFree(m->gwork);
  m->rep = m->x = m->gx = m->grep = nullptr;
  m->perm = nullptr;
  m->gwork = nullptr;
  m->cap_atoms = 0;
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
  if (e == cudaSuccess) e = cudaMalloc(&m->offs, 16 * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemcpy(m->U, host_U, nU * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->signs, host_sign_bits, nS * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->b, host_b, (size_t)n_features * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->alpha, host_alpha, (size_t)n_features * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_error("model allocation/copy failed: %s", cudaGetErrorString(e));
    qmlr_model_destroy(m);
    return e == cudaErrorMemoryAllocation ? QMLR_ENOMEM : QMLR_ECUDA;
  }
  *out = m;
  return QMLR_OK;
}

extern "C" int qmlr_model_destroy(qmlr_model* m) {
  if (!m) return QMLR_OK;
  free_ws(m);
  cudaFree(m->U);
  cudaFree(m->signs);
  cudaFree(m->b);
  cudaFree(m->alpha);
  cudaFree(m->offs);
  delete m;
  return QMLR_OK;
}

extern "C" int qmlr_model_set_alpha(qmlr_model* m, const float* host_alpha) {
  QMLR_REQUIRE(m && host_alpha, "NULL pointer argument");
  QMLR_CUDA_TRY(cudaMemcpy(m->alpha, host_alpha, (size_t)m->n_features * 4, cudaMemcpyHostToDevice));
  return QMLR_OK;
}

namespace qmlr {
__global__ void f64_to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
}  // namespace qmlr

extern "C" int qmlr_model_set_alpha_device(qmlr_model* m, const double* alpha, void* stream) {
  QMLR_REQUIRE(m && alpha, "NULL pointer argument");
  f64_to_f32_kernel<<<(m->n_features + 255) / 256, 256, 0, as_stream(stream)>>>(alpha, m->alpha,
                                                                                m->n_features);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}

extern "C" int qmlr_model_reserve(qmlr_model* m, int32_t max_atoms) {
  QMLR_REQUIRE(m && max_atoms >= 0, "bad arguments");
  if (max_atoms <= m->cap_atoms) return QMLR_OK;
  free_ws(m);
  const size_t n = (size_t)max_atoms;
  m->gwork_bytes = qmlr_group_workspace_bytes(max_atoms);
  cudaError_t e = cudaMalloc(&m->rep, n * m->rep_ld * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->x, n * m->d * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->gx, (size_t)m->n_part * n * m->d * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->grep, n * m->rep_ld * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->perm, std::max<size_t>(n, 1) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->gwork, m->gwork_bytes);
  if (e != cudaSuccess) {
    free_ws(m);
    set_error("workspace allocation failed: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? QMLR_ENOMEM : QMLR_ECUDA;
  }
  m->cap_atoms = max_atoms;
  return QMLR_OK;
}

extern "C" int qmlr_predict_ef(qmlr_model* m, const float* coords, const int32_t* elem,
                               const int32_t* mol_ptr, int32_t n_mol, int32_t n_atoms,
                               double* energies, float* forces, void* stream) {
  QMLR_REQUIRE(m, "model is NULL");
  QMLR_REQUIRE(n_atoms >= 0 && n_mol >= 0, "negative sizes");
  QMLR_REQUIRE(n_atoms <= m->cap_atoms,
               "batch of %d atoms exceeds the reserved capacity %d (call qmlr_model_reserve)", n_atoms,
               m->cap_atoms);
  QMLR_REQUIRE(energies || n_mol == 0, "energies is NULL");
  if (n_mol == 0) return QMLR_OK;
  cudaStream_t s = as_stream(stream);
  int rc;
  const int n_el = m->p.n_el;
  if (n_atoms == 0) {
    QMLR_CUDA_TRY(cudaMemsetAsync(energies, 0, sizeof(double) * n_mol, s));
    return QMLR_OK;
  }
  if ((rc = qmlr_fchl19(coords, elem, mol_ptr, n_mol, n_atoms, m->max_mol_atoms, &m->p, m->rep, m->rep_ld, stream)))
    return rc;
  if ((rc = qmlr_group_by_element(elem, n_atoms, n_el, m->perm, m->offs, m->gwork, m->gwork_bytes, stream)))
    return rc;
  if ((rc = qmlr_project(m->rep, m->rep_ld, m->rep_dim, m->perm, m->offs, n_atoms, n_el, m->U, m->d, m->x,
                         stream)))
    return rc;
  if (!forces) {
    return qmlr_sorf(m->x, m->d, mol_ptr, n_mol, n_atoms, m->signs, m->T, m->b, m->n_features, m->sigma,
                     m->alpha, QMLR_SORF_ENERGY, energies, stream);
  }
  if ((rc = qmlr_sorf_grad(m->x, m->d, mol_ptr, n_mol, n_atoms, m->signs, m->T, m->b, m->n_features, m->sigma,
                           m->alpha, energies, m->gx, stream)))
    return rc;
  if ((rc = qmlr_project_t(m->gx, m->n_part, m->perm, m->offs, n_atoms, n_el, m->U, m->d, m->rep_dim, m->grep,
                           m->rep_ld, stream)))
    return rc;
  if ((rc = qmlr_fchl19_vjp(coords, elem, mol_ptr, n_mol, n_atoms, m->max_mol_atoms, &m->p, m->grep, m->rep_ld,
                            forces, 0, stream)))
    return rc;
  negate_kernel<<<(unsigned)((3L * n_atoms + 255) / 256), 256, 0, s>>>(forces, 3L * n_atoms);
  QMLR_LAUNCH_CHECK();
  return QMLR_OK;
}
