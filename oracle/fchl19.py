"""FCHL19 atom-centred representation, plain FP64 definition (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows the Representation section of the paper:

* cutoff       f_cut(r) = (cos(pi r / r_cut) + 1) / 2, zero for r >= r_cut
                (the cutoff equation; "decays to zero at r_cut").
* two-body     f_cut(r) r^{-N2} / (R_s sigma(r) sqrt(2 pi))
                * exp(-(ln R_s - mu(r))^2 / (2 sigma(r)^2)),
                mu(r) = ln(r / sqrt(1 + eta2/r^2)), sigma(r)^2 = ln(1 + eta2/r^2)
                (two-body, mu and sigma equations).
* three-body   xi_3 * G_radial * G_angular * f_cut(r_ij) f_cut(r_jk) f_cut(r_ik)
                G_radial = sqrt(eta3/pi) exp(-eta3 ((r_ij + r_ik)/2 - R_s)^2)
                xi_3 = c3 (1 + 3 cos th_i cos th_j cos th_k) / (r_ij r_jk r_ik)^{N3}
                G_angular = [G^cos_n, G^sin_n] with
                G^cos_n = exp(-(zeta n)^2/2) (cos(n th) - cos(n(th + pi)))
                G^sin_n = exp(-(zeta n)^2/2) (sin(n th) - sin(n(th + pi)))
                th = angle k-i-j at the centre atom i, n = 1
                (three-body, radial, ATM and Fourier equations).

Periodic systems (the paper's MOF and water rows): ``representation_periodic``
takes the environment of an atom over all lattice images within r_cut (its own
images included), not the minimum image, so cells shorter than 2 r_cut are
described correctly; ``environment_row`` is the per-centre form of the sums.

Readings where the printed text is garbled or silent:
* radial grids R_s = r_cut * k / n for k = 1..n (0 excluded: ln 0 undefined);
* the ATM denominator is the product of the three triangle sides;
* the sine term subtracts sin(n(th + pi)) (the print repeats "cos");
* triplets are unordered pairs {j, k} of neighbours of i;
* f_cut(r_jk) is included as printed, and is zero when r_jk >= r_cut;
* layout: two-body block [element of j][R_s] then three-body block
  [unordered element pair (a <= b), row-major upper triangle][R_s][cos, sin].

All arithmetic is torch float64 so that forces and Jacobians are the exact
derivatives of this definition (torch autograd).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np
import torch

# Optimised parameters, table of the Computational Details section
# (columns "E" and "E + F").
PAPER_TABLE = {
    "E": dict(n2=23, n3=22, eta2=0.27, eta3=5.6, N2=2.78, N3=2.1, c3=60.1,
              zeta=math.pi, rcut=6.0),
    "EF": dict(n2=24, n3=20, eta2=0.32, eta3=2.7, N2=1.8, N3=0.57, c3=13.4,
               zeta=math.pi, rcut=6.0),
}


@dataclass(frozen=True)
class Params:
    n_el: int = 5
    n2: int = 24
    n3: int = 22
    nfourier: int = 1
    eta2: float = 0.27
    eta3: float = 5.6
    N2: float = 2.78
    N3: float = 2.1
    c3: float = 60.1
    zeta: float = math.pi
    rcut: float = 6.0

    @property
    def n_pairs(self) -> int:
        return self.n_el * (self.n_el + 1) // 2

    @property
    def rep_dim(self) -> int:
        return self.n_el * self.n2 + self.n_pairs * self.n3 * 2 * self.nfourier


def params(column: str, n2: int | None = None, n3: int | None = None, n_el: int = 5) -> Params:
    """Parameters from one column of the paper's table; n2/n3 may be overridden."""
    t = dict(PAPER_TABLE[column])
    if n2 is not None:
        t["n2"] = n2
    if n3 is not None:
        t["n3"] = n3
    return Params(n_el=n_el, **t)


def radial_grid(n: int, rcut: float) -> np.ndarray:
    """R_s = r_cut k / n, k = 1..n."""
    return rcut * np.arange(1, n + 1, dtype=np.float64) / n


def pair_index(a: int, b: int, n_el: int) -> int:
    """Index of the unordered element pair {a, b} in row-major upper-triangular order."""
    a, b = min(a, b), max(a, b)
    return a * n_el - a * (a - 1) // 2 + (b - a)


def cutoff(r: torch.Tensor, rcut: float) -> torch.Tensor:
    inside = r < rcut
    return torch.where(inside, 0.5 * (torch.cos(math.pi * r / rcut) + 1.0), torch.zeros_like(r))


def two_body_terms(r: torch.Tensor, p: Params) -> torch.Tensor:
    """[P, n2] two-body values for pair distances r [P] (all r < r_cut)."""
    Rs = torch.as_tensor(radial_grid(p.n2, p.rcut), dtype=r.dtype)
    s2 = torch.log(1.0 + p.eta2 / (r * r))
    mu = torch.log(r / torch.sqrt(1.0 + p.eta2 / (r * r)))
    s = torch.sqrt(s2)
    pref = cutoff(r, p.rcut) * r ** (-p.N2)
    lognormal = (1.0 / (Rs[None, :] * s[:, None] * math.sqrt(2.0 * math.pi))
                 * torch.exp(-(torch.log(Rs)[None, :] - mu[:, None]) ** 2 / (2.0 * s2[:, None])))
    return pref[:, None] * lognormal


def three_body_terms(rij, rik, rjk, cos_i, cos_j, cos_k, p: Params) -> torch.Tensor:
    """[T, n3, 2] three-body values (radial x angular x ATM x cutoffs)."""
    Rs = torch.as_tensor(radial_grid(p.n3, p.rcut), dtype=rij.dtype)
    xi3 = p.c3 * (1.0 + 3.0 * cos_i * cos_j * cos_k) / (rij * rjk * rik) ** p.N3
    radial = math.sqrt(p.eta3 / math.pi) * torch.exp(
        -p.eta3 * (0.5 * (rij + rik)[:, None] - Rs[None, :]) ** 2)
    theta = torch.arccos(torch.clamp(cos_i, -1.0, 1.0))
    n = 1
    damp = math.exp(-((p.zeta * n) ** 2) / 2.0)
    g_cos = damp * (torch.cos(n * theta) - torch.cos(n * (theta + math.pi)))
    g_sin = damp * (torch.sin(n * theta) - torch.sin(n * (theta + math.pi)))
    fc = cutoff(rij, p.rcut) * cutoff(rjk, p.rcut) * cutoff(rik, p.rcut)
    w = (xi3 * fc)[:, None] * radial
    return torch.stack([w * g_cos[:, None], w * g_sin[:, None]], dim=-1)


def neighbour_pairs(x: np.ndarray, rcut: float):
    """Ordered pairs (i, j), i != j, with |r_j - r_i| < r_cut (brute force)."""
    M = len(x)
    d = np.sqrt(np.sum((x[:, None, :] - x[None, :, :]) ** 2, axis=-1))
    mask = (d < rcut) & ~np.eye(M, dtype=bool)
    return np.nonzero(mask)


def triplets(x: np.ndarray, rcut: float):
    """(i, j, k) with j < k, both neighbours of i (brute force)."""
    M = len(x)
    d = np.sqrt(np.sum((x[:, None, :] - x[None, :, :]) ** 2, axis=-1))
    nb = (d < rcut) & ~np.eye(M, dtype=bool)
    ti, tj, tk = [], [], []
    for i in range(M):
        nbrs = np.nonzero(nb[i])[0]
        for a in range(len(nbrs)):
            for b in range(a + 1, len(nbrs)):
                ti.append(i)
                tj.append(nbrs[a])
                tk.append(nbrs[b])
    return np.asarray(ti, dtype=np.int64), np.asarray(tj, dtype=np.int64), np.asarray(tk, dtype=np.int64)


def representation(R: torch.Tensor, elem: np.ndarray, p: Params,
                   x_lists: np.ndarray | None = None) -> torch.Tensor:
    """FCHL19 of one molecule: R [M, 3] float64 tensor (may require grad),
    elem [M] element indices. Returns rho [M, rep_dim] float64.

    The neighbour pairs and triplets are selected from the plain values of the
    coordinates (``x_lists``, default R's values); under forward-mode
    differentiation pass them explicitly."""
    assert p.nfourier == 1
    M = R.shape[0]
    elem = np.asarray(elem, dtype=np.int64)
    xn = R.detach().cpu().numpy() if x_lists is None else np.asarray(x_lists)
    out = torch.zeros(M * p.rep_dim, dtype=R.dtype)

    ii, jj = neighbour_pairs(xn, p.rcut)
    if len(ii):
        rv = R[jj] - R[ii]
        r = torch.sqrt(torch.sum(rv * rv, dim=1))
        g2 = two_body_terms(r, p)                                   # [P, n2]
        col = elem[jj][:, None] * p.n2 + np.arange(p.n2)[None, :]
        idx = torch.as_tensor(ii[:, None] * p.rep_dim + col)
        out = out.index_add(0, idx.reshape(-1), g2.reshape(-1))

    ti, tj, tk = triplets(xn, p.rcut)
    if len(ti):
        vij = R[tj] - R[ti]
        vik = R[tk] - R[ti]
        vjk = R[tk] - R[tj]
        rij = torch.sqrt(torch.sum(vij * vij, dim=1))
        rik = torch.sqrt(torch.sum(vik * vik, dim=1))
        rjk = torch.sqrt(torch.sum(vjk * vjk, dim=1))
        cos_i = torch.sum(vij * vik, dim=1) / (rij * rik)           # angle at i
        cos_j = torch.sum(-vij * vjk, dim=1) / (rij * rjk)          # angle at j
        cos_k = torch.sum(vik * vjk, dim=1) / (rik * rjk)           # angle at k
        g3 = three_body_terms(rij, rik, rjk, cos_i, cos_j, cos_k, p)  # [T, n3, 2]
        pidx = np.array([pair_index(a, b, p.n_el) for a, b in zip(elem[tj], elem[tk])],
                        dtype=np.int64)
        base = p.n_el * p.n2 + pidx * (p.n3 * 2)
        col = base[:, None, None] + (np.arange(p.n3)[None, :, None] * 2
                                     + np.arange(2)[None, None, :])
        idx = torch.as_tensor(ti[:, None, None] * p.rep_dim + col)
        out = out.index_add(0, idx.reshape(-1), g3.reshape(-1))
    return out.reshape(M, p.rep_dim)


def representation_batch(coords: np.ndarray, elem: np.ndarray, mol_ptr: np.ndarray,
                         p: Params) -> np.ndarray:
    """FCHL19 of every atom of a CSR batch of molecules. Returns float64 [n_atoms, rep_dim]."""
    out = np.zeros((int(mol_ptr[-1]), p.rep_dim))
    for m in range(len(mol_ptr) - 1):
        a, b = int(mol_ptr[m]), int(mol_ptr[m + 1])
        if b > a:
            R = torch.as_tensor(np.asarray(coords[a:b], dtype=np.float64))
            out[a:b] = representation(R, elem[a:b], p).numpy()
    return out


def lattice_translations(cell: np.ndarray, rcut: float) -> np.ndarray:
    """Integer triples n (as float64 [K, 3]) with |n_a| <= ceil(rcut / h_a) + 1, h_a the
    spacing of the lattice planes normal to the other two vectors: every image
    within rcut of a point of the cell is among n . cell."""
    A = np.asarray(cell, dtype=np.float64)
    vol = abs(np.linalg.det(A))
    nmax = []
    for a in range(3):
        b, c = A[(a + 1) % 3], A[(a + 2) % 3]
        h = vol / np.linalg.norm(np.cross(b, c))
        nmax.append(int(np.ceil(rcut / h)) + 1)
    g = np.stack(np.meshgrid(*[np.arange(-m, m + 1) for m in nmax], indexing="ij"), axis=-1)
    return g.reshape(-1, 3).astype(np.float64)


def environment_row(v: torch.Tensor, el: np.ndarray, p: Params) -> torch.Tensor:
    """rho of one centre atom from its environment: v [K, 3] the vectors from the
    centre to the K neighbours (all within r_cut), el [K] their elements. The
    same two-body and three-body sums as ``representation``, written for a
    centre with given relative vectors. Returns [rep_dim] float64."""
    assert p.nfourier == 1
    el = np.asarray(el, dtype=np.int64)
    out = torch.zeros(p.rep_dim, dtype=v.dtype)
    K = v.shape[0]
    if K == 0:
        return out
    r = torch.sqrt(torch.sum(v * v, dim=1))
    g2 = two_body_terms(r, p)                                           # [K, n2]
    col = el[:, None] * p.n2 + np.arange(p.n2)[None, :]
    out = out.index_add(0, torch.as_tensor(col.reshape(-1)), g2.reshape(-1))
    a, b = np.triu_indices(K, k=1)
    if len(a):
        vij, vik = v[a], v[b]
        vjk = vik - vij
        rij, rik = r[a], r[b]
        rjk = torch.sqrt(torch.sum(vjk * vjk, dim=1))
        cos_i = torch.sum(vij * vik, dim=1) / (rij * rik)
        cos_j = torch.sum(-vij * vjk, dim=1) / (rij * rjk)
        cos_k = torch.sum(vik * vjk, dim=1) / (rik * rjk)
        g3 = three_body_terms(rij, rik, rjk, cos_i, cos_j, cos_k, p)     # [T, n3, 2]
        pidx = np.array([pair_index(x, y, p.n_el) for x, y in zip(el[a], el[b])], dtype=np.int64)
        base = p.n_el * p.n2 + pidx * (p.n3 * 2)
        col3 = base[:, None, None] + (np.arange(p.n3)[None, :, None] * 2 + np.arange(2)[None, None, :])
        out = out.index_add(0, torch.as_tensor(col3.reshape(-1)), g3.reshape(-1))
    return out


def representation_periodic(R: torch.Tensor, elem: np.ndarray, cell, p: Params) -> torch.Tensor:
    """FCHL19 under periodic boundary conditions (the paper's periodic MOF and
    water systems): the environment of atom i is every periodic image
    R_j + n . cell (n integer, all atoms j including i's own images, not i
    itself) within r_cut of R_i, and rho_i is the environment sum of
    ``environment_row`` (two-body over the images, three-body over unordered
    pairs of images, f_cut(r_jk) from the image positions). The vector to one
    of i's own images is the lattice translation n . cell itself (a constant):
    such an image moves with i, and two of them at opposite translations make
    a collinear triplet whose terms are constant. R [N, 3] float64 tensor (may
    require grad), cell [3, 3] lattice vectors as rows. Returns [N, rep_dim]."""
    elem = np.asarray(elem, dtype=np.int64)
    A = torch.as_tensor(np.asarray(cell, dtype=np.float64))
    shifts = torch.as_tensor(lattice_translations(A.numpy(), p.rcut)) @ A   # [K, 3]
    xn = R.detach().cpu().numpy()
    sn = shifts.numpy()
    n_at = R.shape[0]
    rows = []
    for i in range(n_at):
        rel = xn[None, :, :] + sn[:, None, :] - xn[i][None, None, :]      # [K, N, 3]
        keep = np.sqrt(np.sum(rel * rel, axis=-1)) < p.rcut
        zero = np.abs(sn).sum(axis=1) == 0
        keep[zero, i] = False
        kk, jj = np.nonzero(keep)
        own = jj == i
        v_other = R[jj[~own]] + shifts[kk[~own]] - R[i]
        v_own = shifts[kk[own]]
        v = torch.cat([v_other, v_own], dim=0)
        el = np.concatenate([elem[jj[~own]], elem[jj[own]]])
        rows.append(environment_row(v, el, p))
    return torch.stack(rows, dim=0)


def with_sizes(p: Params, n2: int, n3: int) -> Params:
    return replace(p, n2=n2, n3=n3)
