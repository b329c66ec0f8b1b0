"""Energies, forces and derivative-feature rows of a trained model (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Atomic energy partition (RFF section): E_m = sum_{I in m} alpha^T z(rho_I),
with z the SORF (or RFF) map of the projected representation
rho_I^T U_{e(I)}. Forces are F = -dE/dr (the force rows of the energy+force
normal equations pair with F = -grad E). The derivative features of the RFF
section, dz/dr, enter the energy+force normal equations as rows -dZ_m/dr_{k,a},
stacked under the energy rows, with targets F_{k,a}.

Derivatives here are exact derivatives of the FP64 definition, taken by torch
automatic differentiation (reverse mode for forces, forward mode for the
derivative rows).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch
from torch.func import jacfwd

from . import fchl19, regression, sorf


@dataclass
class Model:
    p: fchl19.Params
    U: np.ndarray        # [n_el, rep_dim, d]
    W: np.ndarray        # [N_F, d]
    b: np.ndarray        # [N_F]
    alpha: np.ndarray | None = None   # [N_F]

    @property
    def n_features(self) -> int:
        return self.W.shape[0]


def _molecule_features(R: torch.Tensor, elem: np.ndarray, m: Model, x_lists=None) -> torch.Tensor:
    """z(rho_I) for the atoms of one molecule: [M, N_F] (differentiable in R)."""
    rho = fchl19.representation(R, elem, m.p, x_lists)
    U = torch.as_tensor(m.U)
    x = torch.stack([rho[i] @ U[int(elem[i])] for i in range(R.shape[0])]) if R.shape[0] else \
        torch.zeros((0, m.U.shape[2]), dtype=R.dtype)
    return sorf.features(x, m.W, m.b)


def molecule_row(R: torch.Tensor, elem: np.ndarray, m: Model, x_lists=None) -> torch.Tensor:
    """Z_m = sum_I z(rho_I)  [N_F]."""
    return _molecule_features(R, elem, m, x_lists).sum(dim=0)


def feature_matrix(coords: np.ndarray, elem: np.ndarray, mol_ptr: np.ndarray, m: Model) -> np.ndarray:
    """Energy rows Z [n_mol, N_F]."""
    Z = np.zeros((len(mol_ptr) - 1, m.n_features))
    with torch.no_grad():
        for k in range(len(mol_ptr) - 1):
            a, b = int(mol_ptr[k]), int(mol_ptr[k + 1])
            Z[k] = molecule_row(torch.as_tensor(coords[a:b], dtype=torch.float64),
                                elem[a:b], m).numpy()
    return Z


def force_rows(coords: np.ndarray, elem: np.ndarray, mol_ptr: np.ndarray, m: Model) -> np.ndarray:
    """Derivative rows [3 n_atoms, N_F]; row 3k+a is -dZ_{mol(k)} / dr_{k,a}."""
    out = np.zeros((3 * int(mol_ptr[-1]), m.n_features))
    for k in range(len(mol_ptr) - 1):
        a, b = int(mol_ptr[k]), int(mol_ptr[k + 1])
        R = torch.as_tensor(coords[a:b], dtype=torch.float64)
        J = jacfwd(lambda r: molecule_row(r, elem[a:b], m, coords[a:b]))(R)   # [N_F, M, 3]
        out[3 * a:3 * b] = -J.reshape(m.n_features, -1).T.numpy()
    return out


def energies_forces(coords: np.ndarray, elem: np.ndarray, mol_ptr: np.ndarray, m: Model,
                    forces: bool = True):
    """E [n_mol] and F [n_atoms, 3] = -dE/dr for a trained model."""
    alpha = torch.as_tensor(m.alpha, dtype=torch.float64)
    E = np.zeros(len(mol_ptr) - 1)
    F = np.zeros((int(mol_ptr[-1]), 3))
    for k in range(len(mol_ptr) - 1):
        a, b = int(mol_ptr[k]), int(mol_ptr[k + 1])
        R = torch.tensor(coords[a:b], dtype=torch.float64, requires_grad=forces)
        e = molecule_row(R, elem[a:b], m) @ alpha
        E[k] = float(e.detach())
        if forces and b > a:
            (g,) = torch.autograd.grad(e, R)
            F[a:b] = -g.numpy()
    return (E, F) if forces else E


def atom_energies(coords, elem, mol_ptr, m: Model) -> np.ndarray:
    """epsilon_I = alpha^T z(rho_I) for every atom."""
    out = np.zeros(int(mol_ptr[-1]))
    alpha = torch.as_tensor(m.alpha, dtype=torch.float64)
    with torch.no_grad():
        for k in range(len(mol_ptr) - 1):
            a, b = int(mol_ptr[k]), int(mol_ptr[k + 1])
            z = _molecule_features(torch.as_tensor(coords[a:b], dtype=torch.float64), elem[a:b], m)
            out[a:b] = (z @ alpha).numpy()
    return out


def train(coords, elem, mol_ptr, energies, m: Model, lam: float, forces=None, refine: int = 1):
    """alpha from the regularised normal equations; energy rows, plus force
    rows when reference forces [n_atoms, 3] are given. Returns (alpha, rel. residual)."""
    Z = feature_matrix(coords, elem, mol_ptr, m)
    y = np.asarray(energies, dtype=np.float64)
    if forces is not None:
        Z = np.concatenate([Z, force_rows(coords, elem, mol_ptr, m)], axis=0)
        y = np.concatenate([y, np.asarray(forces, dtype=np.float64).reshape(-1)])
    return regression.ridge_solve(Z, y, lam, refine)


def sorf_model(p: fchl19.Params, U: np.ndarray, signs: np.ndarray, b: np.ndarray,
               sigma: float, alpha=None) -> Model:
    return Model(p, U, sorf.sorf_matrix(signs, sigma), np.asarray(b, dtype=np.float64), alpha)


def prefactor(n_features: int) -> float:
    return math.sqrt(2.0 / n_features)


def periodic_energy_forces(coords: np.ndarray, elem: np.ndarray, cell: np.ndarray, m: Model):
    """E = sum over the cell's atoms of alpha^T z(rho_I U_e(I)), rho from the
    periodic FCHL19 (lattice images within r_cut), and F = -dE/dR [N, 3] by
    reverse-mode differentiation of that definition."""
    elem = np.asarray(elem)
    R = torch.tensor(np.asarray(coords, dtype=np.float64), requires_grad=True)
    rho = fchl19.representation_periodic(R, elem, cell, m.p)
    U = torch.as_tensor(m.U)
    x = torch.stack([rho[i] @ U[int(elem[i])] for i in range(R.shape[0])])
    e = sorf.features(x, m.W, m.b).sum(dim=0) @ torch.as_tensor(m.alpha, dtype=torch.float64)
    (g,) = torch.autograd.grad(e, R)
    return float(e.detach()), -g.numpy()
