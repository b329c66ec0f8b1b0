"""Training and prediction pipelines over the qmlr C ABI.

Each function only sequences library calls (FCHL19 -> projection -> SORF ->
Gram -> solve); every arithmetic step runs in the library's CUDA kernels.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import qmlr
from .params import FCHL19Params


@dataclass
class Batch:
    """A CSR batch of molecules resident on the device."""

    coords: torch.Tensor   # float32 [n_atoms, 3]
    elem: torch.Tensor     # int32 [n_atoms]
    mol_ptr: torch.Tensor  # int32 [n_mol + 1]
    max_atoms: int

    @property
    def n_atoms(self) -> int:
        return self.coords.shape[0]

    @property
    def n_mol(self) -> int:
        return self.mol_ptr.shape[0] - 1

    @staticmethod
    def from_host(coords, elem, mol_ptr) -> "Batch":
        mol_ptr = np.asarray(mol_ptr)
        return Batch(torch.as_tensor(np.asarray(coords, dtype=np.float32)).cuda(),
                     torch.as_tensor(np.asarray(elem, dtype=np.int32)).cuda(),
                     torch.as_tensor(mol_ptr.astype(np.int32)).cuda(),
                     int(np.diff(mol_ptr).max()) if len(mol_ptr) > 1 else 1)


# SORF energy rows Z on the tensor cores (qmlr_sorf_segment_sum_tc; d = 128,
# T <= 3) instead of the in-register fast Walsh-Hadamard kernel (qmlr_sorf,
# PER_MOL). Off by default: on the QM9-shaped workload both take 38 ms, the
# tensor-core form bound by its epilogue (cos and the ordered molecule sums),
# not by the products.
SORF_TC = False


@dataclass
class FeatureSpec:
    p: FCHL19Params
    d: int
    T: int
    sign_bits: torch.Tensor   # packed Rademacher signs
    b: torch.Tensor           # float32 [N_F]
    sigma: float
    tc_tables: torch.Tensor = None   # FP16 chain tables of the tensor-core SORF (built on first use)

    @property
    def n_features(self) -> int:
        return self.b.shape[0]

    @property
    def sorf_tc(self) -> bool:
        return SORF_TC and self.d == 128 and self.T <= 3 and self.n_features % 128 == 0


def segment_features(x, mol_ptr, spec: FeatureSpec, out=None):
    """Z [n_mol, N_F]: sqrt(2/N_F) sum over each molecule's atoms of cos(W x + b)."""
    if spec.sorf_tc:
        if spec.tc_tables is None:
            spec.tc_tables = qmlr.sorf_tc_tables(spec.sign_bits, spec.T, spec.n_features)
        return qmlr.sorf_segment_sum_tc(x, mol_ptr, spec.tc_tables, spec.T, spec.b, spec.sigma, out=out)
    Z = qmlr.sorf(x, mol_ptr, spec.sign_bits, spec.T, spec.b, spec.sigma, qmlr.SORF_PER_MOL)
    if out is not None:
        out.copy_(Z)
        return out
    return Z


def spec_from(p: FCHL19Params, d: int, signs, b, sigma: float) -> FeatureSpec:
    return FeatureSpec(p, d, signs.shape[1], qmlr.pack_signs(signs),
                       torch.as_tensor(np.asarray(b, dtype=np.float32)).cuda(), float(sigma))


def representations(batch: Batch, spec: FeatureSpec):
    rep = qmlr.fchl19(batch.coords, batch.elem, batch.mol_ptr, batch.max_atoms, spec.p)
    perm, offs = qmlr.group_by_element(batch.elem, spec.p.n_el)
    return rep, perm, offs


def fit_pca(rep, perm, offs, spec: FeatureSpec, max_per_element: int = 4096):
    return qmlr.pca_fit(rep, spec.p.rep_dim, perm, offs, spec.p.n_el, spec.d, max_per_element)


def feature_matrix(batch: Batch, spec: FeatureSpec, U, rep=None, perm=None, offs=None):
    """Energy rows Z [n_mol, N_F] (float32) of the batch."""
    if rep is None:
        rep, perm, offs = representations(batch, spec)
    x = qmlr.project(rep, spec.p.rep_dim, perm, offs, spec.p.n_el, U)
    return segment_features(x, batch.mol_ptr, spec)


# Relative diagonal shift of the preconditioner factor for each Gram form: the
# smallest power of two at which the mixed-precision factor of the QM9-shaped
# Gram (100 000 x 16384) stays positive definite (a smaller one fails a pivot
# and the solve refactorises with a tenfold shift).
# Measured on that Gram (PCG to 1e-8, 150 iterations at most): the 2-way split
# at 2^-15 converges in 10 iterations; the one-part BF16 form needs 2^-12 (33
# iterations), the e4m3 form 2^-8 (117 iterations); the plain FP32 SIMT form
# fails its pivots below 2^-11 (36 iterations there, 53 at 2^-10).
DEFAULT_SHIFT = {qmlr.GRAM_BF16X3: -2.0 ** -15, qmlr.GRAM_BF16X6: -2.0 ** -16, qmlr.GRAM_FP32: -2.0 ** -11,
                 qmlr.GRAM_BF16X1: -2.0 ** -12, qmlr.GRAM_FP8X1: -2.0 ** -8}

# Accumulation and tile width of each tensor-core form by default: every K
# block's accumulator is promoted into FP32 register sums (the tensor cores'
# accumulator adds truncate each product to the accumulator's exponent, so a
# long accumulation in TMEM is strongly biased: keeping the whole K range of
# the QM9-shaped Gram in TMEM made the factor indefinite until the shift was
# near 10 % of max G_ii); 256-wide tiles with plain FP32 register sums, which
# keep the drain off the critical path (the 2-way split: 51 ms instead of 95 ms
# with Kahan sums on 128-wide tiles, same iteration count); the 3-way split
# keeps Kahan sums on 128-wide tiles (its accuracy is the point of it).
DEFAULT_TC = {qmlr.GRAM_BF16X3: (1, 256), qmlr.GRAM_BF16X6: (1, 128), qmlr.GRAM_BF16X1: (1, 256),
              qmlr.GRAM_FP8X1: (1, 256)}


def gram_operand(Z, precision: int):
    """The tensor-core operand of a Gram form (None for the plain FP32 form)."""
    if precision == qmlr.GRAM_FP32:
        return None
    if precision == qmlr.GRAM_FP8X1:
        return qmlr.gram_operand_fp8(Z)
    return qmlr.gram_operand(Z, qmlr.GRAM_SPLITS[precision])


def gram(Z, precision: int, promote: int | None = None, tile: int | None = None, operand=None):
    """G = Z^T Z in the given form (tensor-core forms: promote / tile default to DEFAULT_TC)."""
    if precision == qmlr.GRAM_FP32:
        return qmlr.gram(Z, precision)
    p0, t0 = DEFAULT_TC[precision]
    if operand is None:
        operand = gram_operand(Z, precision)
    return qmlr.gram_tc(Z, precision, promote=p0 if promote is None else promote,
                        tile_n=t0 if tile is None else tile, operand=operand)


def solve(Z, y, lam: float, precision: int = qmlr.GRAM_BF16X3, method: int = qmlr.SOLVE_PCG,
          max_iter: int = 50, tol: float = 1e-10, shift: float | None = None,
          factor: int = qmlr.FACTOR_MIXED, promote: int | None = None, tile: int | None = None):
    """alpha (float64) of (Z^T Z + lam I) alpha = Z^T y; returns (alpha, iterations, rel. residual).
    The Gram (2-way BF16 split by default) only builds the preconditioner; the
    converged alpha is fixed by the exact operator."""
    if shift is None:
        shift = DEFAULT_SHIFT[precision]
    G = gram(Z, precision, promote, tile)
    return qmlr.gram_solve(G, Z, y, lam, method=method, max_iter=max_iter, tol=tol, shift=shift,
                           factor=factor)


def train_energy(batch: Batch, energies, spec: FeatureSpec, lam: float, U=None,
                 precision: int = qmlr.GRAM_BF16X3, **solve_kw):
    """Energy-only training: returns (alpha, U, iterations, relative residual)."""
    rep, perm, offs = representations(batch, spec)
    if U is None:
        U = fit_pca(rep, perm, offs, spec)
    Z = feature_matrix(batch, spec, U, rep, perm, offs)
    y = torch.as_tensor(np.asarray(energies, dtype=np.float64)).cuda()
    alpha, it, rel = solve(Z, y, lam, precision, **solve_kw)
    return alpha, U, it, rel


def energy_force_rows(batch: Batch, spec: FeatureSpec, U):
    """Rows of the energy+force normal equations: [Z; -dZ/dr] with Z [n_mol, N_F]
    stacked over the force rows [3 n_atoms, N_F] (row 3k+x pairs with F[k, x])."""
    rep, perm, offs = representations(batch, spec)
    x = qmlr.project(rep, spec.p.rep_dim, perm, offs, spec.p.n_el, U)
    n_mol, n_atoms = batch.n_mol, batch.n_atoms
    rows = torch.empty((n_mol + 3 * n_atoms, spec.n_features), device="cuda", dtype=torch.float32)
    segment_features(x, batch.mol_ptr, spec, out=rows[:n_mol])
    sin_t = qmlr.sorf(x, batch.mol_ptr, spec.sign_bits, spec.T, spec.b, spec.sigma, qmlr.SORF_SIN_T)
    del rep, x
    jac_ptr, jac, row_elem = qmlr.fchl19_jacobian(batch.coords, batch.elem, batch.mol_ptr, batch.max_atoms, spec.p)
    jperm, joffs = qmlr.group_by_element(row_elem, spec.p.n_el)
    tangents = qmlr.project(jac, spec.p.rep_dim, jperm, joffs, spec.p.n_el, U)
    del jac
    qmlr.force_rows(tangents, jac_ptr, batch.mol_ptr, sin_t, spec.sign_bits, spec.T, spec.n_features,
                    spec.sigma, out=rows, row0=n_mol)
    return rows


def train_energy_force(batch: Batch, energies, forces, spec: FeatureSpec, lam: float, U=None,
                       precision: int = qmlr.GRAM_BF16X3, **solve_kw):
    """Energy + force training: returns (alpha, U, iterations, relative residual)."""
    if U is None:
        rep, perm, offs = representations(batch, spec)
        U = fit_pca(rep, perm, offs, spec)
        del rep
    rows = energy_force_rows(batch, spec, U)
    y = torch.cat([torch.as_tensor(np.asarray(energies, dtype=np.float64)),
                   torch.as_tensor(np.asarray(forces, dtype=np.float64)).reshape(-1)]).cuda()
    alpha, it, rel = solve(rows, y, lam, precision, **solve_kw)
    return alpha, U, it, rel


def predict_periodic(system: "qmlr.PeriodicSystem", spec: FeatureSpec, U, alpha, forces: bool = True):
    """Energy (float64 [1]) and forces F = -dE/dR [N, 3] of a periodic system with
    the atomic energy partition over the cell's atoms: periodic FCHL19 ->
    grouping -> projection -> SORF energies and gradient -> transposed
    projection -> periodic FCHL19 adjoint (scale -1)."""
    p = spec.p
    rep = qmlr.fchl19_periodic(system, p)
    perm, offs = qmlr.group_by_element(system.elem, p.n_el)
    x = qmlr.project(rep, p.rep_dim, perm, offs, p.n_el, U)
    del rep
    mol_ptr = torch.tensor([0, system.n_atoms], dtype=torch.int32, device="cuda")
    if not forces:
        E = qmlr.sorf(x, mol_ptr, spec.sign_bits, spec.T, spec.b, spec.sigma, qmlr.SORF_ENERGY, alpha=alpha)
        return E, None
    E, gx = qmlr.sorf_grad(x, mol_ptr, spec.sign_bits, spec.T, spec.b, spec.sigma, alpha)
    grep = qmlr.project_t(gx, perm, offs, p.n_el, U, p.rep_dim)
    del gx
    F = qmlr.fchl19_periodic_vjp(system, p, grep, scale=-1.0)
    return E, F