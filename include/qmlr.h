/*
 * qmlr.h - C ABI of the GB300 (sm_103a) implementation of the SORF + FCHL19
 * approximate kernel method (Browning, Faber, von Lilienfeld, "GPU-Accelerated
 * Approximate Kernel Method for Quantum Machine Learning").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an int status (QMLR_OK = 0 on success). On failure
 *   qmlr_last_error() returns a message for the calling thread.
 * - Array arguments are device pointers owned by the caller unless the name
 *   starts with host_. Nothing is freed or retained by the library unless a
 *   handle says so.
 * - Work is enqueued on the caller's CUDA stream (passed as void*, a
 *   cudaStream_t; NULL = legacy default stream) and is asynchronous unless
 *   stated otherwise.
 * - Arguments are validated on the host before any launch (QMLR_EINVAL).
 *   Conditions only the device can see (a molecule with more atoms than the
 *   launch was sized for, an element index out of range) make the kernel skip
 *   that molecule and record a code that qmlr_device_status() returns.
 * - Layouts are row-major. Atoms of one molecule are contiguous; molecule m
 *   owns atoms [mol_ptr[m], mol_ptr[m+1]) (CSR offsets, mol_ptr[0] = 0).
 * - Element indices are 0..n_el-1 (the synthetic workloads use H,C,N,O,F).
 */
#ifndef QMLR_H
#define QMLR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  QMLR_OK = 0,
  QMLR_EINVAL = 1,    /* invalid argument (shape, size, pointer, parameter) */
  QMLR_ENOMEM = 2,    /* an allocation made by the library failed */
  QMLR_ECUDA = 3,     /* a CUDA runtime call or launch failed */
  QMLR_EBUSY = 4,     /* serving: request not admitted (slots or memory) */
  QMLR_ETIMEOUT = 5,  /* a bounded wait ran out */
  QMLR_ENOTCONV = 6,  /* solve: refinement did not reach its tolerance (alpha written) */
  QMLR_EDEVICE = 7    /* a kernel recorded a device-side input error */
};

/* Library version string; never NULL. */
const char* qmlr_version(void);

/* Message describing the last failure on the calling thread ("" if none). */
const char* qmlr_last_error(void);

/* Number of CUDA kernels this library has launched since it was loaded (all threads). */
int64_t qmlr_launch_count(void);

/*
 * Synchronises `stream`, then reads and clears the device-side error word of
 * the current device. *host_code = 0 if no kernel recorded an error since the
 * last call; 1 = molecule larger than the launch's max_mol_atoms, 2 = element
 * index out of range, 3 = index out of range, 4 = bounded wait ran out,
 * 5 = matrix not positive definite, 6 = a SORF input whose phases would leave
 * the range the feature kernels reduce exactly (see qmlr_sorf). Returns
 * QMLR_EDEVICE when *host_code != 0.
 */
int qmlr_device_status(void* stream, int32_t* host_code);

/* ------------------------------------------------------------------------
 * FCHL19 representation (Representation section: two-body, cutoff,
 * three-body, ATM and Fourier-angular equations; parameter table of the
 * Computational Details section).
 * ------------------------------------------------------------------------ */
typedef struct qmlr_fchl19_params {
  int32_t n_el;      /* element types, 1..8 */
  int32_t n2;        /* two-body radial grid points, R_s = rcut*k/n2, k=1..n2 (1..64) */
  int32_t n3;        /* three-body radial grid points, R_s = rcut*k/n3 (1..64) */
  int32_t nfourier;  /* Fourier order of the angular term; must be 1 */
  double eta2;       /* two-body log-normal width parameter */
  double eta3;       /* three-body Gaussian width */
  double N2;         /* two-body decay exponent: r^-N2 */
  double N3;         /* three-body ATM decay exponent: (r_ij r_jk r_ik)^-N3 */
  double c3;         /* three-body weight */
  double zeta;       /* angular Gaussian width */
  double rcut;       /* cutoff radius in Angstrom */
} qmlr_fchl19_params;

/*
 * Periodic environments (for the paper's periodic MOF and water systems): for
 * every atom i, the lattice images R_j + n . cell (n an integer triple; all
 * atoms j, i's own images included, i itself excluded) with |R_j + n . cell -
 * R_i| < rcut. Host code (cell list in fractional coordinates, any triclinic
 * cell, rcut larger than the cell allowed). Synchronous.
 *   host_coords  double [n_atoms][3] (need not lie inside the cell)
 *   host_cell    double [3][3] lattice vectors as rows (non-singular)
 *   host_env_ptr int64 [n_atoms+1] CSR offsets, written by ..._count
 *   host_env_atom  int32 [env_ptr[n_atoms]]     j of each entry
 *   host_env_shift int32 [env_ptr[n_atoms]][3]  n of each entry
 * Entries of one atom are sorted by (j, n). qmlr_periodic_environment checks
 * that host_env_ptr matches the coordinates it is given.
 */
int qmlr_periodic_environment_count(const double* host_coords, int32_t n_atoms, const double* host_cell,
                                    double rcut, int64_t* host_env_ptr);
int qmlr_periodic_environment(const double* host_coords, int32_t n_atoms, const double* host_cell, double rcut,
                              const int64_t* host_env_ptr, int32_t* host_env_atom, int32_t* host_env_shift);

/*
 * The environment entries grouped by the atom they name (host, synchronous):
 * host_rev_ptr int64 [n_atoms+1], host_rev_entry int64 [env_ptr[n_atoms]]:
 * the entries e with env_atom[e] == k are host_rev_entry[rev_ptr[k] .. rev_ptr[k+1]),
 * ascending. Used by qmlr_fchl19_periodic_vjp to sum each atom's gradient in a
 * fixed order.
 */
int qmlr_periodic_reverse(const int64_t* host_env_ptr, const int32_t* host_env_atom, int32_t n_atoms,
                          int64_t* host_rev_ptr, int64_t* host_rev_entry);

/*
 * FCHL19 of a periodic system (the paper's periodic MOF and water systems): the
 * row of atom i sums over its environment entries (j, n) (device copies of the
 * qmlr_periodic_environment arrays) at R_j + n . cell, the displacement formed
 * in FP64 and rounded to FP32. Entries at or beyond the cutoff in FP32 are
 * skipped.
 *   coords     float [n_atoms][3]    elem int32 [n_atoms]
 *   host_cell  double [3][3] lattice vectors as rows (read on the call)
 *   env_ptr    int64 [n_atoms+1], env_atom int32 [E], env_shift int32 [E][3]  (device)
 *   max_env    upper bound on entries per atom (sizes shared memory; 0..2048,
 *              the adjoint needs max_env of a few hundred at most); an atom with
 *              more entries is recorded as device error 1 and its row set to zero
 *   rep        float [n_atoms][rep_ld]
 * Deterministic; asynchronous. n_el <= 5, n2, n3 <= 32.
 */
int qmlr_fchl19_periodic(const float* coords, const int32_t* elem, int32_t n_atoms, const double* host_cell,
                         const int64_t* env_ptr, const int32_t* env_atom, const int32_t* env_shift,
                         int32_t max_env, const qmlr_fchl19_params* p, float* rep, int32_t rep_ld, void* stream);

/*
 * Vector-Jacobian product of the periodic FCHL19 (forces of a periodic system):
 *   grad_coords[k] (+)= scale * sum_i (d rho_i / d R_k)^T grad_rep[i]
 * where an image R_j + n . cell moves with R_j. Same geometry arguments as
 * qmlr_fchl19_periodic; rev_ptr, rev_entry (device) from qmlr_periodic_reverse;
 * contrib: device scratch float [(E + n_atoms)][3]. Every atom's sum runs in a
 * fixed order (deterministic); asynchronous.
 */
int qmlr_fchl19_periodic_vjp(const float* coords, const int32_t* elem, int32_t n_atoms, const double* host_cell,
                             const int64_t* env_ptr, const int32_t* env_atom, const int32_t* env_shift,
                             int32_t max_env, const qmlr_fchl19_params* p, const float* grad_rep, int32_t rep_ld,
                             const int64_t* rev_ptr, const int64_t* rev_entry, float* contrib, float scale,
                             float* grad_coords, int32_t accumulate, void* stream);

/* rep_dim = n_el*n2 + n_el(n_el+1)/2 * n3 * 2 (780 for 5 elements, n2=24, n3=22). */
int qmlr_fchl19_rep_dim(const qmlr_fchl19_params* p, int32_t* rep_dim);

/*
 * FCHL19 forward: rho_i for every atom.
 *   coords   float [n_atoms][3]  positions (Angstrom)
 *   elem     int32 [n_atoms]     element index
 *   mol_ptr  int32 [n_mol+1]     CSR molecule offsets; neighbours are taken
 *                                within the same molecule only
 *   max_mol_atoms                upper bound on atoms per molecule (1..256);
 *                                sizes the shared-memory staging
 *   rep      float [n_atoms][rep_ld], rep_ld >= rep_dim; columns rep_dim..rep_ld-1
 *            are written as zeros.
 * Layout of a row: two-body block [element of j][n2], then three-body block
 * [unordered element pair (a<=b), row-major upper triangle][n3][cos, sin].
 * Deterministic: each atom's row is summed by one warp in a fixed order.
 */
int qmlr_fchl19(const float* coords, const int32_t* elem, const int32_t* mol_ptr,
                int32_t n_mol, int32_t n_atoms, int32_t max_mol_atoms,
                const qmlr_fchl19_params* p, float* rep, int32_t rep_ld, void* stream);

/*
 * FCHL19 vector-Jacobian product (forces through the representation; the
 * backward pass the Computational Details section describes, with three-body
 * terms recomputed rather than stored):
 *   grad_coords[k] (+)= sum_i (d rho_i / d r_k)^T grad_rep[i]
 *   grad_rep    float [n_atoms][rep_ld]
 *   grad_coords float [n_atoms][3]; overwritten when accumulate == 0, added to otherwise.
 * Same geometry arguments as qmlr_fchl19. Deterministic (fixed-order sums per molecule).
 */
int qmlr_fchl19_vjp(const float* coords, const int32_t* elem, const int32_t* mol_ptr,
                    int32_t n_mol, int32_t n_atoms, int32_t max_mol_atoms,
                    const qmlr_fchl19_params* p, const float* grad_rep, int32_t rep_ld,
                    float* grad_coords, int32_t accumulate, void* stream);

/*
 * Jacobian rows of FCHL19 (forward mode, for the force rows of energy+force
 * training): jac_ptr int64 [n_mol+1] row offsets, jac_ptr[m] = sum_{m'<m} 3 M_{m'}^2,
 * written by qmlr_jac_offsets (which also returns the total on the host,
 * synchronously, when host_total is not NULL).
 */
int qmlr_jac_offsets(const int32_t* mol_ptr, int32_t n_mol, int64_t* jac_ptr, int64_t* host_total,
                     void* stream);

/*
 * jac float [jac_ptr[n_mol]][rep_ld]: row jac_ptr[m] + (I*M + k)*3 + x holds
 * d rho_{I} / d r_{k,x} for centre I and atom k of molecule m (local indices, M atoms):
 * zero when k is beyond the cutoff of I; for k = I minus the sum over the
 * neighbours (translation invariance). Three-body terms are recomputed.
 * row_elem int32 [jac_ptr[n_mol]]: element of each row's centre (for the projection).
 */
int qmlr_fchl19_jac(const float* coords, const int32_t* elem, const int32_t* mol_ptr, int32_t n_mol,
                    int32_t n_atoms, int32_t max_mol_atoms, const qmlr_fchl19_params* p,
                    const int64_t* jac_ptr, float* jac, int32_t rep_ld, int32_t* row_elem,
                    void* stream);

/*
 * The same vector-Jacobian product with one warp per centre atom (the atoms
 * of a molecule run in parallel; for small batches and large molecules):
 *   pair_ptr   int64 [n_mol+1] from qmlr_jac_offsets (sum of 3 M^2)
 *   contrib    float [pair_ptr[n_mol]] scratch: per-centre contributions
 *   grad_coords[k] = scale * sum_i (d rho_i / d r_k)^T grad_rep[i]  (+ previous value if accumulate)
 * The sum over centres runs in order (deterministic); scale = -1 gives forces.
 */
int qmlr_fchl19_vjp_atoms(const float* coords, const int32_t* elem, const int32_t* mol_ptr,
                          int32_t n_mol, int32_t n_atoms, int32_t max_mol_atoms,
                          const qmlr_fchl19_params* p, const float* grad_rep, int32_t rep_ld,
                          const int64_t* pair_ptr, float* contrib, float scale, float* grad_coords,
                          int32_t accumulate, void* stream);

/* ------------------------------------------------------------------------
 * Per-element projection (SORF section: SVD of the representations of each
 * element, rho_proj = rho^T U_e^{N_PCA}; GPU implementation paragraph: each
 * element has its own projection matrix).
 * ------------------------------------------------------------------------ */

/* Bytes of device workspace qmlr_group_by_element needs for n_atoms atoms. */
int64_t qmlr_group_workspace_bytes(int32_t n_atoms);

/*
 * Stable grouping of atoms by element (a counting sort on the device):
 *   perm         int32 [n_atoms]  atom indices, element 0 first, ascending atom
 *                                 index within an element
 *   elem_offsets int32 [n_el+1]   atoms of element e are perm[elem_offsets[e] .. elem_offsets[e+1])
 *   work         device workspace of qmlr_group_workspace_bytes(n_atoms) bytes
 * Element indices outside [0, n_el) are recorded as a device error and
 * grouped with element 0.
 */
int qmlr_group_by_element(const int32_t* elem, int32_t n_atoms, int32_t n_el, int32_t* perm,
                          int32_t* elem_offsets, void* work, int64_t work_bytes, void* stream);

/*
 * Element grouping that allocates nothing (the paper has no counterpart: this
 * is an integration convenience). Same result as qmlr_group_by_element, for
 * callers that cannot allocate device memory when they need it: a host
 * framework that owns every device buffer through its own pool and hands out
 * no raw allocations, or a latency-bound service that must not wait on the
 * allocator in its request path. The counting sort's scratch is a fixed 256 KiB array inside the
 * library (one per device that loads it, kept until the process exits), so
 * n_atoms is limited to QMLR_GROUP_NOALLOC_MAX_ATOMS; larger inputs are
 * rejected with QMLR_EINVAL before any launch.
 *   - The first call on a device looks up that device's copy of the array
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - All calls share the one array: calls whose work overlaps on the GPU
 *     (different streams, or different host threads on one device) race and
 *     must be serialised by the caller. The array keeps the last call's
 *     contents; every value a call reads is written by that call first.
 *   - No cudaMalloc, cudaFree or allocating library routine is called.
 */
#define QMLR_GROUP_NOALLOC_MAX_ATOMS 4194304
int qmlr_group_by_element_noalloc(const int32_t* elem, int32_t n_atoms, int32_t n_el,
                                  int32_t* perm, int32_t* elem_offsets, void* stream);

/* Bytes of device workspace qmlr_project and qmlr_project_t need (the split basis). */
int64_t qmlr_project_workspace_bytes(int32_t n_el, int32_t rep_dim, int32_t d);

/*
 * x[i][:] = rep[i][:rep_dim] * U[elem(i)]   (SORF section: projection onto the element's
 * principal directions). Runs on the tensor cores with 3-way BF16 splits of
 * both operands and FP32 accumulation (products to ~2^-24 relative, the
 * accuracy of an FP32 GEMM); the split basis is made on every call in the
 * caller's workspace (no allocation).
 *   rep  float [n_atoms][rep_ld]
 *   perm, elem_offsets  from qmlr_group_by_element
 *   U    float [n_el][rep_dim][d]   (U_e with the d basis vectors as columns)
 *   x    float [n_atoms][d]
 *   work device workspace of qmlr_project_workspace_bytes(n_el, rep_dim, d) bytes
 *        (used until the call's work on `stream` has finished)
 * d is a power of two, 16..512.
 */
int qmlr_project(const float* rep, int32_t rep_ld, int32_t rep_dim, const int32_t* perm,
                 const int32_t* elem_offsets, int32_t n_atoms, int32_t n_el, const float* U,
                 int32_t d, float* x, void* work, int64_t work_bytes, void* stream);

/*
 * Transposed projection (chain rule through the projection):
 *   grad_rep[i][:rep_dim] = U[elem(i)] * sum_p gx[p][i][:]
 * gx holds n_part partial gradients [n_part][n_atoms][d] (summed in a fixed
 * order). Columns rep_dim..rep_ld-1 of grad_rep are written as zeros. Same
 * tensor-core arithmetic and workspace as qmlr_project.
 */
int qmlr_project_t(const float* gx, int32_t n_part, const int32_t* perm,
                   const int32_t* elem_offsets, int32_t n_atoms, int32_t n_el, const float* U,
                   int32_t d, int32_t rep_dim, float* grad_rep, int32_t rep_ld, void* work,
                   int64_t work_bytes, void* stream);

/* ------------------------------------------------------------------------
 * SORF feature map (SORF section; RFF feature-map equation; GPU
 * implementation paragraph on structured orthogonal features).
 *   u = (sqrt(d)/sigma) [H D_{s,T}] ... [H D_{s,1}] x / sqrt(d)^T + b,  z = sqrt(2/N_F) cos(u)
 * for every stack s = 0..N_F/d-1, with H the unnormalised Walsh-Hadamard
 * matrix and D_{s,t} the Rademacher diagonal of stack s, transform t (applied
 * before H). sign_bits[(s*T + t)*(d/32 rounded up) + w] bit j set means
 * D_{s,t}[32w + j] = -1.
 * ------------------------------------------------------------------------ */
enum {
  QMLR_SORF_PER_ATOM = 0, /* out: float [n_atoms][N_F]  z for every atom */
  QMLR_SORF_PER_MOL = 1,  /* out: float [n_mol][N_F]    Z_m = sum_{I in m} z_I (fixed order) */
  QMLR_SORF_ENERGY = 2,   /* out: double [n_mol]        E_m = sum_{I in m} alpha^T z_I */
  QMLR_SORF_SIN_T = 4     /* out: float [n_atoms][d][N_F/d]  sqrt(2/N_F) sin(u) with the stack index
                             fastest (feature f = s*d + i stored at [atom][i][s]); used by qmlr_force_rows */
};

/*
 * x          float [n_atoms][d] projected representations
 * sign_bits  uint32 [n_stack][T][ceil(d/32)]
 * b          float [N_F] phases
 * alpha      float [N_F] regression weights (ENERGY mode; otherwise may be NULL)
 * out        see mode
 * T is 1..4; d is a power of two, 16..128; N_F = n_features is a multiple of d.
 * In ENERGY mode with more than 128 stacks the per-part molecule sums are
 * added to out with FP64 atomics (out is zeroed first).
 * Range: the cosines and sines reduce u = W x + b by 2 pi exactly while
 * |u| < 2^17 pi (about 4.1e5). Since each stack of W is sqrt(d)/sigma times an
 * orthogonal matrix, |u_i| <= (sqrt(d)/sigma) |x|_2 + |b_i|; an atom whose
 * (sqrt(d)/sigma) |x|_2 exceeds 2^17 pi - 4 pi (or is not finite) is recorded
 * as device error 6 (qmlr_device_status) and its features are not meaningful.
 * The same check runs in qmlr_sorf_grad and the model's prediction.
 * In PER_MOL mode the phases are copied once per call into stream-ordered
 * scratch (N_F floats, stack index fastest) for coalesced loads.
 */
int qmlr_sorf(const float* x, int32_t d, const int32_t* mol_ptr, int32_t n_mol, int32_t n_atoms,
              const uint32_t* sign_bits, int32_t T, const float* b, int32_t n_features,
              double sigma, const float* alpha, int32_t mode, void* out, void* stream);

/*
 * Dense random Fourier features (RFF section: z(x) = sqrt(2/N_F) cos(W x + b)
 * with W = G / sigma, G standard normal), the feature map SORF replaces; the
 * reference side of the paper's SORF-versus-RFF comparison.
 *   x     float [n_atoms][d], d = 1..256
 *   G     float [N_F][d]  the standard-normal draw (1/sigma is applied inside)
 *   b     float [N_F]     phases
 *   mode  QMLR_SORF_PER_ATOM: out float [n_atoms][N_F];
 *         QMLR_SORF_PER_MOL:  out float [n_mol][N_F], Z_m = sum_{I in m} z_I
 *         (atoms in order; an empty molecule gives a zero row)
 * FP32 arithmetic (dot products with a fixed summation order, cosf);
 * deterministic. Asynchronous.
 */
int qmlr_rff(const float* x, int32_t d, const int32_t* mol_ptr, int32_t n_mol, int32_t n_atoms,
             const float* G, const float* b, int32_t n_features, double sigma, int32_t mode,
             float* out, void* stream);

/*
 * The same dense random Fourier features on the tensor cores: u = x (G/sigma)^T
 * as a tcgen05 GEMM on 3-way BF16 splits of both operands (FP32 accumulation:
 * products to ~2^-24, the accuracy of an FP32 GEMM), in chunks of up to 65 536
 * atoms, then cos(u + b) (cosf) and, in PER_MOL mode, the per-molecule sums of
 * each chunk's atoms in order (a molecule split across chunks adds its parts
 * in chunk order). Arguments as qmlr_rff; d = 1..512; work: device scratch of
 * qmlr_rff_tc_workspace_bytes(n_atoms, d, n_features, mode) bytes (the split
 * (G/sigma), the row order and, in PER_MOL mode, one chunk of u). Deterministic;
 * asynchronous.
 */
int64_t qmlr_rff_tc_workspace_bytes(int32_t n_atoms, int32_t d, int32_t n_features, int32_t mode);
int qmlr_rff_tc(const float* x, int32_t d, const int32_t* mol_ptr, int32_t n_mol, int32_t n_atoms,
                const float* G, const float* b, int32_t n_features, double sigma, int32_t mode, float* out,
                void* work, int64_t work_bytes, void* stream);

/*
 * Force rows of the energy+force normal equations (RFF section: the
 * derivative features dz/dr stacked under Z): for molecule m, atom k, axis x
 *   rows[row0 + 3*(mol_ptr[m] + k) + x][f] = -dZ_m/dr_{k,x}[f]
 *       = sum_{I in m} sqrt(2/N_F) sin(u_I[f]) (W t_{I,k,x})[f]
 *   tangents float [n_jac_rows][d]: t_{I,k,x} = U_{e(I)}^T d rho_I/d r_{k,x} (qmlr_fchl19_jac
 *            rows projected with qmlr_project), row jac_ptr[m] + (I*M + k)*3 + x
 *   sin_t    float [n_atoms][d][N_F/d] from qmlr_sorf(..., QMLR_SORF_SIN_T)
 *   rows     float, row stride ld >= N_F
 * The sum over centres I runs in order (deterministic).
 */
int qmlr_force_rows(const float* tangents, int32_t d, const int64_t* jac_ptr, const int32_t* mol_ptr,
                    int32_t n_mol, const float* sin_t, const uint32_t* sign_bits, int32_t T,
                    int32_t n_features, double sigma, float* rows, int64_t ld, int64_t row0,
                    void* stream);

/* Number of stack parts qmlr_sorf_grad splits N_F/d stacks into: ceil(N_F/d / 128). */
int32_t qmlr_sorf_parts(int32_t n_features, int32_t d);

/*
 * Energy and its gradient with respect to the projected representations
 * (the SORF backward pass: transposed Hadamard chain applied to
 * -sqrt(2/N_F) alpha * sin(u)); one CTA per (atom, stack part), so the atoms
 * of a molecule run in parallel:
 *   atom_energy double [n_part][n_atoms]  per-atom partial energies (written; scratch)
 *   energies    double [n_mol]            E_m = sum over atoms, then parts, in order
 *   gx          float [n_part][n_atoms][d]  dE/dx_I from the stacks of part p, or NULL
 *                                          (energies only)
 * n_part = qmlr_sorf_parts(n_features, d); qmlr_project_t sums the parts.
 */
int qmlr_sorf_grad(const float* x, int32_t d, const int32_t* mol_ptr, int32_t n_mol,
                   int32_t n_atoms, const uint32_t* sign_bits, int32_t T, const float* b,
                   int32_t n_features, double sigma, const float* alpha, double* atom_energy,
                   double* energies, float* gx, void* stream);

/*
 * The same energies and gradients with both Hadamard chains on the tensor
 * cores (SORF section: u_s = c M_s x + b_s with M_s = H D_T ... H D_1 and
 * c = (sqrt(d)/sigma) / d^{T/2}; gradient -sqrt(2/N_F) c sum_s M_s^T
 * (alpha_s * sin u_s)). For d = 128 and T <= 3 the entries of M_s are integers
 * of magnitude <= d^{T/2} (<= 1448), exact in FP16, so M_s is stored as FP16
 * tables and both directions are tcgen05 products (kind::f16, FP32
 * accumulation): x is split per atom into two FP16 parts after a power-of-two
 * row scale (2^-22 relative per element), the backward operand
 * alpha * sin(u) likewise with one power-of-two scale for all features; the
 * backward accumulator is promoted into FP32 sums every 8 half stacks.
 * Phases use the same reduction and range check as qmlr_sorf (device error 6).
 *
 *   qmlr_sorf_tc_table_bytes(N_F)   bytes of the chain tables (4 N_F d bytes)
 *   qmlr_sorf_tc_tables             fills them from the packed signs (device
 *                                   tables, 16-byte aligned; caller-owned;
 *                                   build once per set of signs)
 *   qmlr_sorf_tc_workspace_bytes(n, N_F) bytes of the per-call workspace
 *                                   (~516 B per atom + 4 N_F; 256-byte aligned)
 *   qmlr_sorf_grad_tc               atom_energy double [n_atoms] (one part),
 *                                   energies double [n_mol], gx float
 *                                   [n_atoms][128] (one part: pass n_part = 1
 *                                   to qmlr_project_t); x, b, alpha, gx 16-byte
 *                                   aligned; gx is required.
 * Errors: QMLR_EINVAL for d != 128, T > 3, N_F not a multiple of 128, NULL or
 * misaligned pointers, a workspace below the required size. Asynchronous on
 * `stream`; deterministic; allocates nothing; a persistent kernel of one CTA
 * per SM whose waits are bounded (device error 4, a timeout, on expiry).
 */
int64_t qmlr_sorf_tc_table_bytes(int32_t n_features);
int64_t qmlr_sorf_tc_workspace_bytes(int32_t n_atoms, int32_t n_features);
int qmlr_sorf_tc_tables(const uint32_t* sign_bits, int32_t d, int32_t T, int32_t n_features,
                        void* tables, void* stream);
int qmlr_sorf_grad_tc(const float* x, int32_t d, const int32_t* mol_ptr, int32_t n_mol,
                      int32_t n_atoms, const void* tables, int32_t T, const float* b,
                      int32_t n_features, double sigma, const float* alpha, double* atom_energy,
                      double* energies, float* gx, void* work, int64_t work_bytes, void* stream);

/*
 * Energy rows Z_m = sqrt(2/N_F) sum_{I in m} cos(u(x_I)) (SORF section; the
 * rows of the normal equations) with the forward chains on the tensor cores:
 * the same FP16 tables, operand split, phases and range check as
 * qmlr_sorf_grad_tc, cos of the phases, and each molecule's atoms added in
 * atom order in FP32 (the order of qmlr_sorf's PER_MOL mode), so Z_m does not
 * depend on the batch the molecule is in. Each CTA of the persistent kernel
 * owns a contiguous range of whole molecules; a molecule of any size is
 * carried across 128-atom tiles.
 *   Z     float [n_mol] rows of stride ldz >= N_F (16-byte aligned), every
 *         row written (an empty molecule gives a zero row)
 *   work  qmlr_sorf_tc_segment_workspace_bytes(n_atoms, N_F) bytes, 256-byte
 *         aligned (FP16 parts of x, row scales, carried rows)
 * Same argument rules and errors as qmlr_sorf_grad_tc. Asynchronous on
 * `stream`; allocates nothing.
 */
int64_t qmlr_sorf_tc_segment_workspace_bytes(int32_t n_atoms, int32_t n_features);
int qmlr_sorf_segment_sum_tc(const float* x, int32_t d, const int32_t* mol_ptr, int32_t n_mol,
                             int32_t n_atoms, const void* tables, int32_t T, const float* b,
                             int32_t n_features, double sigma, float* Z, int64_t ldz, void* work,
                             int64_t work_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Regularised normal equations (RFF section: (Z^T Z + lambda I) alpha = Z^T E,
 * energy and force rows stacked for energy+force training; the paper solves
 * by LU in FP64 and builds Z^T Z in FP64 or FP32 with Kahan summation).
 * ------------------------------------------------------------------------ */
enum {
  QMLR_GRAM_FP32 = 0,   /* plain FP32 SIMT product (comparison form, no compensation) */
  QMLR_GRAM_BF16X3 = 1, /* tensor cores, 2-way BF16 split S0+S1: S0'S0 + S0'S1 + S1'S0 (~2^-16 rel.) */
  QMLR_GRAM_BF16X6 = 2, /* tensor cores, 3-way BF16 split: the six products of order <= 2 (~2^-24 rel.) */
  QMLR_GRAM_BF16X1 = 3, /* tensor cores, one BF16 part: S0'S0 (Z rounded to 8 significant bits) */
  QMLR_GRAM_FP8X1 = 4   /* tensor cores (kind::f8f6f4), one e4m3 part with per-feature power-of-two
                           scales: Q'Q / (s_i s_j), Q = e4m3(Z s) (4 significant bits) */
};

/*
 * Split-precision Gram operand, transposed (feature-major, rows contiguous):
 *   S0 = bf16(Z), S1 = bf16(Z - S0), S2 = bf16(Z - S0 - S1)   (round to nearest even)
 *   zt[q][f][r] = S_q[r][f] for q < n_split (1, 2 or 3); bf16 bit patterns,
 *   [n_split][n_features][k_pad]; k_pad >= n_rows, k_pad % 64 == 0; rows
 *   n_rows..k_pad-1 are written as zeros.
 *   Z float [n_rows][ldz]
 */
int qmlr_gram_operand(const float* Z, int64_t n_rows, int32_t n_features, int64_t ldz,
                      int32_t n_split, uint16_t* zt, int64_t k_pad, void* stream);

/*
 * The e4m3 Gram operand (QMLR_GRAM_FP8X1), transposed like the split operand:
 *   inv_scale float [n_features]: 1/s_f with s_f = 2^floor(log2(448 / max_r |Z[r][f]|))
 *                                 (s_f = 1 for an all-zero feature)
 *   zt uint8 [n_features][k_pad]: e4m3 bit patterns of s_f Z[r][f], rounded to
 *                                 nearest even, saturated at 448; rows n_rows..k_pad-1 zero
 *   k_pad >= n_rows, k_pad % 128 == 0. Deterministic. Asynchronous.
 */
int qmlr_gram_operand_fp8(const float* Z, int64_t n_rows, int32_t n_features, int64_t ldz, uint8_t* zt,
                          int64_t k_pad, float* inv_scale, void* stream);

/*
 * G = Z^T Z as a full symmetric float [n_features][n_features] matrix.
 *   QMLR_GRAM_FP32:   reads Z [n_rows][ldz] (zt may be NULL)
 *   QMLR_GRAM_BF16X3: reads zt with n_split = 2; QMLR_GRAM_BF16X6: n_split = 3
 *                     (Z may be NULL); n_features % 128 == 0.
 *   QMLR_GRAM_BF16X1: reads zt with n_split = 1; the qmlr_gram_tc defaults
 *                     (256-wide tiles, the whole K range in the accumulator);
 *                     n_features % 256 == 0.
 * Deterministic: every element is summed in a fixed order. Split forms with
 * at least 4 x (SM count) tiles of 128 x 128 run as one cooperative launch of
 * one CTA per SM (same per-tile arithmetic, bitwise the same G); that launch
 * takes a 4-byte counter from the stream-ordered allocator and frees it
 * stream-ordered.
 */
int qmlr_gram(int32_t precision, const float* Z, int64_t n_rows, int32_t n_features, int64_t ldz,
              const uint16_t* zt, int64_t k_pad, float* G, void* stream);

/*
 * The tensor-core Gram with its tiling and accumulation chosen by the caller
 * (the forms that only build a preconditioner can trade accuracy for time).
 *   precision  QMLR_GRAM_BF16X1 / BF16X3 / BF16X6 (zt from qmlr_gram_operand with
 *              n_split 1 / 2 / 3, k_pad % 64 == 0) or QMLR_GRAM_FP8X1 (zt and
 *              inv_scale from qmlr_gram_operand_fp8, k_pad % 128 == 0)
 *   promote    K blocks (128-byte lines of K: 64 bf16 or 128 e4m3 values) summed
 *              in the tensor cores' FP32 accumulator before that sum is added
 *              into FP32 register sums; 1 = every block (the accumulator's
 *              truncating adds then span one block), 0 = the whole K range
 *   tile_n     columns per 128-row tile: 128 or 256 (0: 256 for BF16X1 and FP8X1,
 *              128 otherwise); n_features must be a multiple of it
 * Register sums are Kahan sums for BF16X3/BF16X6 with 128-wide tiles, plain
 * FP32 sums otherwise; BF16X6 supports 128-wide tiles only. One cooperative
 * launch of one CTA per SM (fewer for small matrices); a 4-byte counter comes
 * from the stream-ordered allocator. Deterministic. Asynchronous.
 */
typedef struct qmlr_gram_opts {
  int32_t precision;
  int32_t promote;
  int32_t tile_n;
} qmlr_gram_opts;
int qmlr_gram_tc(const qmlr_gram_opts* opts, const void* zt, int64_t k_pad, int32_t n_features,
                 const float* inv_scale, float* G, void* stream);

/* c = Z^T y in FP64 (y double [n_rows], c double [n_features]); fixed-order sums. */
int64_t qmlr_zty_workspace_bytes(int64_t n_rows, int32_t n_features);
int qmlr_zty(const float* Z, int64_t n_rows, int32_t n_features, int64_t ldz, const double* y,
             double* c, void* work, int64_t work_bytes, void* stream);

/*
 * In-place FP64 Cholesky factorisation A = L L^T of the lower triangle of
 * L (double [n][ldl], row-major); the strict upper triangle is not referenced.
 * Synchronous. *host_info = 0 on success, else the 1-based column whose pivot
 * was not positive (the factor is then not usable).
 */
int qmlr_cholesky(double* L, int64_t ldl, int32_t n, int32_t* host_info, void* stream);

/*
 * Mixed-precision factor A ~= L L^T (same layout and info as qmlr_cholesky),
 * meant as the preconditioner of an iteration on the exact operator (the
 * ridge solve below). Right-looking in 256-column panels: each panel is
 * factorised in double-float FP32 arithmetic (pair products and two-sums,
 * ~2^-44 relative; the entries are stored in FP64); the update of the
 * remaining lower triangle by a panel
 * runs on the tensor cores from the panel's 3-way BF16 split (products to
 * ~2^-24 relative, FP32 sums over each 64-deep K block, subtracted in FP32
 * arithmetic from the not yet factorised matrix, which is held as float pairs
 * hi + lo in the same storage), so L L^T matches A to ~1e-7 of max|A| rather
 * than to FP64 round-off. work: device scratch of qmlr_cholesky_mixed_workspace_bytes(n)
 * bytes, 256-byte aligned. Synchronous. The factor's side stream, events and
 * diagonal-block buffer are one set per device, so calls on one device (from
 * any host thread or stream, including qmlr_gram_solve with QMLR_FACTOR_MIXED)
 * run one at a time: a call waits until the previous one has finished on the GPU.
 */
int64_t qmlr_cholesky_mixed_workspace_bytes(int32_t n);
int qmlr_cholesky_mixed(double* L, int64_t ldl, int32_t n, void* work, int64_t work_bytes,
                        int32_t* host_info, void* stream);

/* v <- (L L^T)^{-1} v with a factor from qmlr_cholesky or qmlr_cholesky_mixed
   (forward, then backward substitution, in FP64). Non-finite entries whose bit
   pattern is all ones make the dataflow sweeps time out (device error 4). */
int qmlr_cholesky_solve(const double* L, int64_t ldl, int32_t n, double* v, void* stream);

enum {
  QMLR_SOLVE_PCG = 0,    /* conjugate gradients on the exact operator, Cholesky-preconditioned */
  QMLR_SOLVE_REFINE = 1  /* classical iterative refinement with the Cholesky factor */
};

enum {
  QMLR_FACTOR_FP64 = 0,  /* preconditioner factor: qmlr_cholesky (FP64 throughout) */
  QMLR_FACTOR_MIXED = 1  /* preconditioner factor: qmlr_cholesky_mixed (tensor-core updates) */
};

typedef struct qmlr_solve_opts {
  int32_t method;      /* QMLR_SOLVE_PCG or QMLR_SOLVE_REFINE */
  int32_t max_iter;    /* refinement iterations after the first solve (>= 0) */
  double tol;          /* target ||c - A alpha|| / ||c|| */
  double shift;        /* added to the diagonal of the factorised matrix only: >= 0 absolute,
                          < 0 relative (|shift| * max_i G_ii); raised tenfold (up to 8 times)
                          when a pivot is not positive */
  int32_t iters_done;  /* out: refinement iterations run */
  double rel_resid;    /* out: final ||c - A alpha|| / ||c|| with the exact operator */
  double shift_used;   /* out: the shift of the factor that was used */
  float factor_ms;     /* out: device time of assembly + Cholesky factorisation (CUDA events) */
  float refine_ms;     /* out: device time of the first solve and the refinement */
  int32_t factor;      /* QMLR_FACTOR_FP64 or QMLR_FACTOR_MIXED */
} qmlr_solve_opts;

/*
 * q = Z^T (Z p) + lambda p: the exact operator of the ridge solve below (the
 * RFF section's normal-equation matrix applied to a vector without forming
 * it). Z float [n_rows][ldz] (row-major), p and q double [n_features] (device).
 * Arithmetic: FP32 products split exactly by FMA and summed in float pairs
 * (two-sum) folded into FP64 every 128 terms, i.e. about twice FP32's
 * precision (relative error ~1e-12 of the sum of |terms| on feature data);
 * fixed summation order, so repeated calls agree bitwise. work: device scratch
 * of qmlr_normal_apply_workspace_bytes bytes, 256-byte aligned. Asynchronous.
 */
int64_t qmlr_normal_apply_workspace_bytes(int64_t n_rows, int32_t n_features);
int qmlr_normal_apply(const float* Z, int64_t n_rows, int32_t n_features, int64_t ldz, double lambda,
                      const double* p, double* q, void* work, int64_t work_bytes, void* stream);

/* Device workspace bytes of qmlr_gram_solve. */
int64_t qmlr_solve_workspace_bytes(int64_t n_rows, int32_t n_features);

/*
 * Solve (Z^T Z + lambda I) alpha = Z^T y (synchronous; returns once alpha is final).
 *   G      float [n_features]^2 symmetric Gram (any precision form of qmlr_gram)
 *   Z      float [n_rows][ldz] the stored feature rows (the exact operator is
 *          A v = Z^T (Z v) + lambda v, evaluated as in qmlr_normal_apply)
 *   y      double [n_rows] targets
 *   alpha  double [n_features] out
 * Steps: c = Z^T y; Cholesky factor of G + (lambda + shift) I (FP64 or mixed
 * precision, opts->factor); alpha = factor solve of c; then up to max_iter
 * refinement steps against the exact operator, which alone sets the residual.
 * QMLR_ENOTCONV: tolerance not reached (alpha and opts->rel_resid still written).
 * QMLR_EINVAL with a message when the factorisation still meets a non-positive
 * pivot after the shift escalation.
 */
int qmlr_gram_solve(const float* G, const float* Z, int64_t n_rows, int32_t n_features,
                    int64_t ldz, const double* y, double lambda, qmlr_solve_opts* opts,
                    double* alpha, void* work, int64_t work_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Per-element PCA basis (SORF section: U_e from the SVD of the element's
 * representations; setup step, run once per model).
 * ------------------------------------------------------------------------ */

/* Device workspace bytes of qmlr_pca_fit. */
int64_t qmlr_pca_workspace_bytes(int32_t rep_ld, int32_t d);

/*
 * U[e] (float [n_el][rep_dim][d]) = leading d eigenvectors of
 * C_e = sum_i rho_i rho_i^T over the first max_per_element atoms of element e
 * in perm order (perm, elem_offsets from qmlr_group_by_element), computed in
 * FP64 by randomized subspace iteration + Rayleigh-Ritz + Jacobi. Columns are
 * ordered by descending eigenvalue; each column's largest-magnitude entry is
 * positive; columns with eigenvalue <= 1e-12 of the largest (and all columns
 * of an element without atoms) are zero. Synchronous (reads elem_offsets).
 * d <= 128.
 */
int qmlr_pca_fit(const float* rep, int32_t rep_ld, int32_t rep_dim, const int32_t* perm,
                 const int32_t* elem_offsets, int32_t n_el, int32_t max_per_element, int32_t d,
                 float* U, void* work, int64_t work_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Trained model and energy + force prediction (atomic energy partition
 * E = sum_I alpha^T z(rho_I), RFF section; forces by the SORF and FCHL19
 * backward passes, Computational Details).
 * ------------------------------------------------------------------------ */
typedef struct qmlr_model qmlr_model;

/*
 * Model file: the checkpoint of a trained model, in host memory only (no GPU
 * needed). Holds the FCHL19 parameters, rep_dim, d, T, N_F, sigma, the lambda
 * the weights were trained with, and the arrays
 *   host_U         float  [n_el][rep_dim][d]
 *   host_sign_bits uint32 [N_F/d][T][ceil(d/32)]  (bit set: D entry -1)
 *   host_b         float  [N_F]
 *   host_alpha     double [N_F]
 * Little-endian, a fixed field-by-field header after the magic "QMLRMDL1" and a
 * version word, then the arrays in that order, then the 64-bit FNV-1a of all
 * preceding bytes. qmlr_model_file_info reads the scalars (so the caller can
 * size the arrays); qmlr_model_file_read copies the arrays out. Both reject a
 * file with a bad magic, an unknown version, sizes that disagree with its
 * length, or a failed checksum (QMLR_EINVAL with a message). Synchronous.
 */
int qmlr_model_file_write(const char* path, const qmlr_fchl19_params* p, int32_t rep_dim, int32_t d,
                          int32_t n_transform, int32_t n_features, double sigma, double lambda,
                          const float* host_U, const uint32_t* host_sign_bits, const float* host_b,
                          const double* host_alpha);
int qmlr_model_file_info(const char* path, qmlr_fchl19_params* p, int32_t* rep_dim, int32_t* d,
                         int32_t* n_transform, int32_t* n_features, double* sigma, double* lambda);
int qmlr_model_file_read(const char* path, float* host_U, uint32_t* host_sign_bits, float* host_b,
                         double* host_alpha);

/*
 * Copies the model to the current device. Host arrays (read once):
 *   host_U         float [n_el][rep_dim][d]
 *   host_sign_bits uint32 [N_F/d][T][ceil(d/32)]
 *   host_b         float [N_F]
 *   host_alpha     float [N_F]
 * max_mol_atoms bounds the atoms per molecule of every later batch.
 */
int qmlr_model_create(const qmlr_fchl19_params* p, int32_t max_mol_atoms, const float* host_U,
                      int32_t d, const uint32_t* host_sign_bits, int32_t T, const float* host_b,
                      int32_t n_features, double sigma, const float* host_alpha, qmlr_model** out);
int qmlr_model_destroy(qmlr_model* m);
int qmlr_model_set_alpha(qmlr_model* m, const float* host_alpha);
/* Replace alpha from a device FP64 vector [N_F] (e.g. the output of qmlr_gram_solve); asynchronous. */
int qmlr_model_set_alpha_device(qmlr_model* m, const double* alpha, void* stream);

/*
 * Diagnostics: with timing enabled the model records CUDA events around the
 * kernels of each prediction on the caller's stream; qmlr_model_timings waits
 * for the last prediction and writes up to five times in ms: [0] FCHL19
 * forward, [1] element grouping + projection, [2] SORF energies and gradient,
 * [3] transposed projection, [4] FCHL19 adjoint with its ordered reduction
 * (entries 3 and 4 only when forces were requested). Not for use while a
 * prediction is being captured into a CUDA graph.
 */
/*
 * Which kernel computes the SORF energies and gradients of qmlr_predict_ef
 * with forces: the tensor-core chains (qmlr_sorf_grad_tc; the default when
 * the model has d = 128 and T <= 3, tables built at model creation) or the
 * FWHT kernel of qmlr_sorf_grad (enable = 0). Batches below 8192 atoms and
 * energy-only predictions always use the FWHT kernel (the tensor-core form
 * takes a fixed ~0.4 ms per 128-atom tile at N_F = 16384). Results are
 * bitwise independent of the batch a molecule is in within each form; the
 * two forms agree to the parity bounds. Enabling it on a model without tables
 * returns QMLR_EINVAL.
 */
int qmlr_model_set_sorf_tc(qmlr_model* m, int32_t enable);
int32_t qmlr_model_sorf_tc(const qmlr_model* m);

int qmlr_model_set_timing(qmlr_model* m, int32_t enable);
int qmlr_model_timings(qmlr_model* m, float* host_ms, int32_t n);

/* Allocates (or grows) the model's prediction workspace for batches of up to max_atoms atoms. */
int qmlr_model_reserve(qmlr_model* m, int32_t max_atoms);

/*
 * Energies (double [n_mol]) and forces F = -dE/dr (float [n_atoms][3];
 * NULL = energies only) for a CSR batch of molecules; device inputs/outputs,
 * asynchronous on `stream`, no allocation (n_atoms <= reserved capacity).
 */
int qmlr_predict_ef(qmlr_model* m, const float* coords, const int32_t* elem,
                    const int32_t* mol_ptr, int32_t n_mol, int32_t n_atoms, double* energies,
                    float* forces, void* stream);

/*
 * qmlr_predict_ef in two calls, for overlapping the part that does not depend
 * on the weights with other work (e.g. the solve that produces them):
 * qmlr_predict_features computes the representations, element grouping and
 * projections of the batch into the model's workspace;
 * qmlr_predict_ef_from_features then forms energies (and forces) from them with
 * the model's current weights. The second call must get the same batch, on a
 * stream ordered after the first, with no other prediction through the same
 * model in between. Same results as qmlr_predict_ef (bitwise).
 */
int qmlr_predict_features(qmlr_model* m, const float* coords, const int32_t* elem,
                          const int32_t* mol_ptr, int32_t n_mol, int32_t n_atoms, void* stream);
int qmlr_predict_ef_from_features(qmlr_model* m, const float* coords, const int32_t* elem,
                                  const int32_t* mol_ptr, int32_t n_mol, int32_t n_atoms,
                                  double* energies, float* forces, void* stream);

/*
 * Chain rule of molecule energies through their forces, for automatic-
 * differentiation wrappers: given F = -dE/dr from qmlr_predict_ef and an
 * upstream gradient grad_E (double [n_mol]) of a loss L with respect to the
 * energies, grad_coords[k][x] = dL/dr_{k,x} = -grad_E[mol(k)] F[k][x] (every
 * atom belongs to exactly one molecule, so this is the whole product).
 * forces and grad_coords float [n_atoms][3] (may be the same buffer).
 * Asynchronous.
 */
int qmlr_energy_vjp(const float* forces, const int32_t* mol_ptr, int32_t n_mol, int32_t n_atoms,
                    const double* grad_E, float* grad_coords, void* stream);

/* ------------------------------------------------------------------------
 * Diagnostics: throughput of single functional units on the current device
 * (the denominators of the ALU-bound kernels' rooflines). Each rate is
 * operations per second of one kind, issued independently by 8 CTAs of 256
 * threads per SM (CUDA events, 5 launches after a warm-up); synchronous.
 * ------------------------------------------------------------------------ */
enum {
  QMLR_RATE_DFMA = 0,    /* FP64 fused multiply-adds */
  QMLR_RATE_FFMA = 1,    /* FP32 fused multiply-adds */
  QMLR_RATE_FADD = 2,    /* FP32 adds */
  QMLR_RATE_FADD_X2 = 3, /* FP32 element adds issued as packed add.rn.f32x2 */
  QMLR_RATE_EXP = 4,     /* __expf */
  QMLR_RATE_SIN = 5,     /* __sinf */
  QMLR_RATE_SHFL = 6,    /* 32-bit warp shuffles (per lane) */
  QMLR_RATE_COUNT = 7
};
int qmlr_unit_rates(double* host_rates, int32_t n_rates, void* stream);

/* ------------------------------------------------------------------------
 * Continuous-batching server for energy + force prediction (the timings
 * section's observation that single configurations leave the GPU idle and
 * batching cuts the cost per configuration). Host-side runtime in the library.
 * ------------------------------------------------------------------------ */
typedef struct qmlr_server qmlr_server;

typedef struct qmlr_serve_config {
  int32_t n_lanes;            /* batches in flight on the device (1..8), one CUDA stream each */
  int32_t max_batch_atoms;    /* atoms per batch (>= the model's max_mol_atoms) */
  int32_t max_batch_mols;     /* molecules per batch (real + padding) */
  int32_t max_slots;          /* requests held (queued, running or not yet collected) */
  int64_t max_inflight_atoms; /* atoms held */
  int64_t mem_budget_bytes;   /* device memory the lanes may take (<= 0: no limit) */
  int32_t use_graphs;         /* capture each (lane, batch-size bucket) prediction as a CUDA graph */
} qmlr_serve_config;

typedef struct qmlr_serve_report {
  int64_t completed, rejected, batches;
  double p50_us, p99_us, mean_us, max_us;  /* submit -> result ready latency */
  double throughput_rps;                   /* completed requests per second (first submit -> last result) */
  double us_per_atom;                      /* same span per predicted atom */
  double mean_batch_atoms;
} qmlr_serve_report;

/*
 * Starts a server for a model on the current device: allocates n_lanes
 * workspaces and pinned staging buffers and a batcher thread. QMLR_EINVAL
 * when the lanes do not fit mem_budget_bytes. The model must outlive the server.
 */
int qmlr_serve_create(qmlr_model* m, const qmlr_serve_config* cfg, qmlr_server** out);

/*
 * Admits one molecule (host coordinates float [n_atoms][3], elements int32
 * [n_atoms]; copied before return). QMLR_EBUSY when the request or atom limit
 * of held work would be exceeded (nothing is queued). Thread-safe.
 */
int qmlr_serve_submit(qmlr_server* s, const float* host_coords, const int32_t* host_elem,
                      int32_t n_atoms, uint64_t* ticket);

/*
 * Waits up to timeout_us (bounded at 600 s) for a ticket's result and
 * collects it: *host_E (double) and host_F float [n_atoms][3] (F = -dE/dr;
 * either may be NULL). QMLR_ETIMEOUT if not ready (the ticket stays valid).
 * A collected ticket is released. Thread-safe.
 */
int qmlr_serve_poll(qmlr_server* s, uint64_t ticket, double* host_E, float* host_F,
                    int64_t timeout_us);

int qmlr_serve_stats(qmlr_server* s, qmlr_serve_report* out);
int qmlr_serve_reset_stats(qmlr_server* s);

/*
 * The latencies behind the statistics (submit -> result ready, microseconds,
 * in completion order since the last reset) with the atom count of each
 * request: copies min(count, capacity) pairs into host_latency_us (float) and
 * host_atoms (int32), and sets *count to the number recorded. Thread-safe.
 */
int qmlr_serve_latencies(qmlr_server* s, float* host_latency_us, int32_t* host_atoms, int64_t capacity,
                         int64_t* count);

/*
 * Load driver: replays a request trace against the server from two host
 * threads (one submits molecule pick[i] of the pool at arrival_us[i]
 * microseconds after the start, spinning until then; one collects results in
 * submission order), then returns the server's statistics for the run.
 * Pool: host_coords float [pool atoms][3], host_elem int32, host_mol_ptr
 * int32 [n_pool+1]. *rejected = requests refused by admission. Synchronous.
 */
int qmlr_serve_replay(qmlr_server* s, const float* host_coords, const int32_t* host_elem,
                      const int32_t* host_mol_ptr, int32_t n_pool, const double* arrival_us,
                      const int32_t* pick, int32_t n_req, int64_t* rejected, qmlr_serve_report* out);

/* Finishes the batches in flight, stops the batcher and frees the server. */
int qmlr_serve_destroy(qmlr_server* s);

#ifdef __cplusplus
}
#endif

#endif /* QMLR_H */
