// Internal layout of the model handle (shared by model.cu and serve.cu).
#pragma once

#include "common.cuh"

struct qmlr_model;

namespace qmlr {

// Device buffers of one prediction pass for batches of up to cap_atoms atoms.
struct PredictWorkspace {
  int cap_atoms = 0;
  float* rep = nullptr;     // [cap][rep_ld]
  float* x = nullptr;       // [cap][d]
  float* gx = nullptr;      // [n_part][cap][d]
  float* grep = nullptr;    // [cap][rep_ld]
  int32_t* perm = nullptr;  // [cap]
  int32_t* offs = nullptr;  // [n_el+1]
  void* gwork = nullptr;
  int64_t gwork_bytes = 0;
  double* atom_e = nullptr;   // [n_part][cap] per-atom energy partials
  int64_t* pair_ptr = nullptr;// [cap_mols + 1] offsets of the per-centre force contributions
  float* contrib = nullptr;   // [cap * max_mol_atoms * 3]
  int cap_mols = 0;
  void* sorf_work = nullptr;  // tensor-core SORF: FP16 parts of x and row scales
  size_t sorf_work_bytes = 0;

  int reserve(const qmlr_model* m, int max_atoms);
  void release();
  static size_t bytes_per_atom(const qmlr_model* m);
};

// SORF energies (and gradients when gx != NULL) with stack-minor phases/weights.
int sorf_energy_grad_model(const float* x, int d, const int32_t* mol_ptr, int n_mol, int n_atoms,
                           const uint32_t* sign_bits, int T, const float* bT, int n_features, double sigma,
                           const float* alphaT, double* atom_e, double* E, float* gx, cudaStream_t s);

// Tensor-core SORF energies and gradients (sorf_tc.cu): chain tables
// [2][N_F][128] FP16, per-call workspace of FP16 parts of x and row scales.
size_t sorf_tc_table_bytes(int n_features);
size_t sorf_tc_work_bytes(int n_atoms, int n_features);
bool sorf_tc_supported(int d, int T, int n_features);
int sorf_tc_tables(const uint32_t* sign_bits, int T, int n_features, void* tables, cudaStream_t s);
int sorf_tc_energy_grad(const float* x, int n_atoms, const void* tables, int T, const float* b,
                        const float* alpha, int n_features, double sigma, double* atom_e, float* gx, void* work,
                        size_t work_bytes, cudaStream_t s);
// E[m] = sum over the molecule's atoms and the n_part partials (sorf.cu).
int sorf_segment_energy(const double* atom_e, int n_part, int n_atoms, const int32_t* mol_ptr, int n_mol,
                        double* E, cudaStream_t s);

// Tensor-core grouped projection (project_tc.cu).
size_t proj_tc_basis_bytes(int n_el, int K, int N);
int proj_tc_split_basis(const float* U, int n_el, int K, int N, long es, int ldu, bool trans, uint16_t* out,
                        cudaStream_t s, float scale = 1.0f);
int proj_tc_launch(const float* A, int lda, int K, int n_part, long a_part_stride, const uint16_t* basis, int N,
                   const int32_t* perm, const int32_t* elem_offsets, int n_atoms, int n_el, float* C, int ldc,
                   int zero_pad_to, cudaStream_t s);

// The two halves of predict_ef_ws: the representation, element grouping and
// projection (independent of the weights), then the SORF energies/gradients,
// the transposed projection and the VJP from those features.
int predict_features_ws(const qmlr_model* m, PredictWorkspace& w, const float* coords, const int32_t* elem,
                        const int32_t* mol_ptr, int n_mol, int n_atoms, cudaStream_t s);
int predict_from_features_ws(const qmlr_model* m, PredictWorkspace& w, const float* coords, const int32_t* elem,
                             const int32_t* mol_ptr, int n_mol, int n_atoms, double* energies, float* forces,
                             cudaStream_t s);

// Energies and forces of a CSR batch with the given workspace (no allocation).
int predict_ef_ws(const qmlr_model* m, PredictWorkspace& w, const float* coords, const int32_t* elem,
                  const int32_t* mol_ptr, int n_mol, int n_atoms, double* energies, float* forces,
                  cudaStream_t s);

}  // namespace qmlr

struct qmlr_model {
  qmlr_fchl19_params p;
  int max_mol_atoms;
  int rep_dim, rep_ld, d, T, n_features, n_part;
  double sigma;
  float* U = nullptr;          // [n_el][rep_dim][d]
  uint32_t* signs = nullptr;   // [n_stack][T][W]
  float* b = nullptr;          // [N_F]
  float* alpha = nullptr;      // [N_F]
  float* bT = nullptr;         // [d][n_stack] stack-minor copy of b
  float* alphaT = nullptr;     // [d][n_stack] stack-minor copy of alpha
  uint16_t* Ufwd = nullptr;    // U split for the tensor-core projection (bf16 [n_el][3][N_pad][K_pad])
  uint16_t* Utrn = nullptr;    // U split for the transposed projection
  qmlr::PredictWorkspace ws;   // workspace of qmlr_predict_ef
  void* sorf_tables = nullptr;  // chain tables of the tensor-core SORF (d = 128, T <= 3)
  bool sorf_tc = false;        // energies + gradients on the tensor cores (else the FWHT kernel)
  bool timing = false;         // record events around the prediction's kernels (diagnostics)
  cudaEvent_t tev[8] = {};     // FCHL19 | grouping + projection | SORF | projection^T | adjoint
};
