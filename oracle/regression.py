"""PCA projection, feature matrix and regularised normal equations (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* PCA (SORF section, projection equations): for each element e the
  representations of that element are the columns of Z~_e = U_e S_e V_e^T;
  rho_proj = rho^T U_e^{N_PCA}, the first N_PCA columns of U_e. U_e is taken
  here as the eigenvectors of Z~_e Z~_e^T (uncentred), eigenvalues in
  descending order; each column is signed so that its entry of largest
  magnitude is positive; columns beyond the numerical rank are zero.
* Feature matrix (atomic energy partition, RFF section): the row of molecule
  m is Z_m = sum over the atoms I of m of z(rho_I).
* Reduced-precision Gram operands (the preconditioner inputs of the solve):
  ``round_to_format`` rounds to a binary floating-point format given by its
  fraction bits, smallest normal exponent and largest finite value (round to
  nearest, ties to even, saturating): bfloat16 is (7, -126, (2 - 2^-7) 2^127),
  e4m3 is (3, -6, 448). ``quantized_gram`` is the exact product Q^T Q of the
  rounded operand, for one bfloat16 part or for e4m3 with a power-of-two
  scale per feature (s_f = 2^floor(log2(448 / max |Z[:, f]|))).
* Normal equations (RFF section): (Z^T Z + lambda I) alpha = Z^T y, with
  energy and force rows stacked vertically for energy+force training. Solved
  here by a dense float64 Cholesky factorisation (the matrix is symmetric
  positive definite; the paper names LU) and one step of iterative
  refinement against the assembled matrix.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def pca_basis(reps_e: np.ndarray, d: int, rank_tol: float = 1e-12) -> np.ndarray:
    """U_e^{N_PCA} [rep_dim, d] from the representations of one element [n, rep_dim]."""
    X = np.asarray(reps_e, dtype=np.float64)
    C = X.T @ X
    w, V = np.linalg.eigh(C)
    order = np.argsort(w)[::-1]
    w, V = w[order], V[:, order]
    U = V[:, :d].copy()
    for c in range(U.shape[1]):
        k = int(np.argmax(np.abs(U[:, c])))
        if U[k, c] < 0:
            U[:, c] = -U[:, c]
    wmax = max(float(w[0]), 0.0) if len(w) else 0.0
    rank = int(np.sum(w > rank_tol * wmax)) if wmax > 0 else 0
    U[:, rank:] = 0.0
    if U.shape[1] < d:
        U = np.concatenate([U, np.zeros((U.shape[0], d - U.shape[1]))], axis=1)
    return U


def pca_bases(reps: np.ndarray, elem: np.ndarray, n_el: int, d: int,
              max_per_element: int | None = None, rng=None) -> np.ndarray:
    """U [n_el, rep_dim, d]; optionally a random subset of each element's atoms."""
    out = np.zeros((n_el, reps.shape[1], d))
    for e in range(n_el):
        idx = np.nonzero(np.asarray(elem) == e)[0]
        if max_per_element is not None and len(idx) > max_per_element:
            idx = np.sort(rng.choice(idx, size=max_per_element, replace=False))
        if len(idx):
            out[e] = pca_basis(reps[idx], d)
    return out


def project(reps: np.ndarray, elem: np.ndarray, U: np.ndarray) -> np.ndarray:
    """rho_proj_I = rho_I^T U_{e(I)} for every atom."""
    reps = np.asarray(reps, dtype=np.float64)
    out = np.zeros((reps.shape[0], U.shape[2]))
    for e in range(U.shape[0]):
        idx = np.nonzero(np.asarray(elem) == e)[0]
        out[idx] = reps[idx] @ U[e]
    return out


def segment_sum(z: np.ndarray, mol_ptr: np.ndarray) -> np.ndarray:
    """Z_m = sum_{I in m} z_I for a CSR batch."""
    n_mol = len(mol_ptr) - 1
    Z = np.zeros((n_mol, z.shape[1]))
    for m in range(n_mol):
        Z[m] = np.sum(z[mol_ptr[m]:mol_ptr[m + 1]], axis=0)
    return Z


def normal_equations(Z: np.ndarray, y: np.ndarray, lam: float):
    """A = Z^T Z + lambda I and c = Z^T y."""
    Z = np.asarray(Z, dtype=np.float64)
    A = Z.T @ Z + lam * np.eye(Z.shape[1])
    return A, Z.T @ np.asarray(y, dtype=np.float64)


def cholesky_solve(A: np.ndarray, c: np.ndarray, refine: int = 1):
    """alpha with A alpha = c via A = L L^T, then `refine` refinement steps
    r = c - A alpha, alpha += A^{-1} r. Returns (alpha, relative residual)."""
    L = np.linalg.cholesky(A)

    def solve(v):
        t = scipy.linalg.solve_triangular(L, v, lower=True)
        return scipy.linalg.solve_triangular(L.T, t, lower=False)

    alpha = solve(c)
    for _ in range(refine):
        alpha = alpha + solve(c - A @ alpha)
    res = np.linalg.norm(c - A @ alpha) / max(np.linalg.norm(c), 1e-300)
    return alpha, res


def ridge_solve(Z: np.ndarray, y: np.ndarray, lam: float, refine: int = 1):
    """Solve the regularised normal equations for rows Z [n_rows, N_F] and targets y."""
    A, c = normal_equations(Z, y, lam)
    return cholesky_solve(A, c, refine)


BF16_FORMAT = (7, -126, (2.0 - 2.0 ** -7) * 2.0 ** 127)
E4M3_FORMAT = (3, -6, 448.0)


def round_to_format(x, fmt) -> np.ndarray:
    """Nearest value (ties to even) of the format (fraction bits, smallest normal
    exponent, largest finite value); magnitudes above the largest finite value
    become it (saturation). Below the smallest normal the spacing stays
    2^(emin - fraction bits) (subnormals)."""
    mant, emin, vmax = fmt
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, ex = np.frexp(np.where(a > 0, a, 1.0))      # a = m 2^ex, m in [0.5, 1)
    e = np.maximum(ex - 1, emin)                   # exponent of the binade (or of the subnormals)
    quantum = np.ldexp(1.0, e - mant)
    q = np.minimum(np.round(a / quantum) * quantum, vmax)   # np.round: ties to even
    return np.copysign(q, x)


def fp8_feature_scales(Z) -> np.ndarray:
    """s_f = 2^floor(log2(448 / max_r |Z[r, f]|)), 1 for an all-zero feature."""
    amax = np.max(np.abs(np.asarray(Z, dtype=np.float64)), axis=0)
    s = np.ones_like(amax)
    nz = amax > 0
    _, ex = np.frexp(448.0 / amax[nz])
    s[nz] = np.ldexp(1.0, ex - 1)
    return s


def quantized_gram(Z, form: str) -> np.ndarray:
    """Q^T Q in float64 for the operand rounded to 'bf16' or to 'e4m3' with
    per-feature scales (then divided by s_i s_j)."""
    Z = np.asarray(Z, dtype=np.float64)
    if form == "bf16":
        Q = round_to_format(Z, BF16_FORMAT)
        return Q.T @ Q
    if form == "e4m3":
        s = fp8_feature_scales(Z)
        Q = round_to_format(Z * s[None, :], E4M3_FORMAT)
        return (Q.T @ Q) / np.outer(s, s)
    raise ValueError(form)
