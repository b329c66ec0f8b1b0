"""Seeded synthetic workloads shaped like the paper's benchmarks.

This module draws inputs only: molecule geometries, element labels, the random
parameters the SORF feature map consumes (Rademacher signs and phases) and
synthetic regression targets from simple analytic potentials. It holds none of
the method's arithmetic (no representation, projection, feature map or solve),
so the CUDA path and the FP64 oracle can both be fed from it.

The paper's data sets (QM9, MD17, 3BPA) are not available; the generators
stand in for their shapes, sizes and composition:

* ``random_box``    - small molecules with atoms uniform in a cube (the
  parity-sized workload: 64 molecules x 9 atoms, 4 A box).
* ``grow_molecule`` - random bonded growth: each new atom bonds to a heavy atom
  with free valence at a random bond length in a random direction; contacts
  closer than 0.9 A are rejected.
* ``qm9_like``      - QM9-shaped set (3-29 atoms, mean 18, ~51 % H).
* ``conformations`` - MD17/3BPA-shaped sets: one grown reference geometry,
  Gaussian displacements and optional rotations about rotatable bonds.
* ``serving_stream``- Poisson arrivals of molecules 5-200 atoms
  (log-uniform size).

Element indices are 0..4 for H, C, N, O, F. Units are Angstrom and eV.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2206_01580

ELEMENTS = ("H", "C", "N", "O", "F")
Z_OF_ELEMENT = (1, 6, 7, 8, 9)
VALENCE = (1, 4, 3, 2, 1)
H, C, N, O, F = range(5)


def rng_for(config_index: int, stream: int = 0) -> np.random.Generator:
    """PCG64 generator for a workload: seed = 220601580 + config index."""
    return np.random.Generator(np.random.PCG64([SEED_BASE + config_index, stream]))


@dataclass
class MoleculeSet:
    """A batch of molecules in CSR layout.

    coords  float64 [n_atoms, 3]
    elem    int32   [n_atoms]     element index 0..4
    mol_ptr int32   [n_mol + 1]   atom range of molecule m is mol_ptr[m]:mol_ptr[m+1]
    bonds   list of (i, j) global atom index pairs of the growth tree (may be empty)
    """

    coords: np.ndarray
    elem: np.ndarray
    mol_ptr: np.ndarray
    bonds: list = field(default_factory=list)

    @property
    def n_mol(self) -> int:
        return len(self.mol_ptr) - 1

    @property
    def n_atoms(self) -> int:
        return int(self.mol_ptr[-1])

    def sizes(self) -> np.ndarray:
        return np.diff(self.mol_ptr)

    def molecule(self, m: int):
        a, b = int(self.mol_ptr[m]), int(self.mol_ptr[m + 1])
        return self.coords[a:b], self.elem[a:b]

    def subset(self, mols) -> "MoleculeSet":
        mols = np.asarray(mols, dtype=np.int64)
        parts_c, parts_e, ptr = [], [], [0]
        for m in mols:
            c, e = self.molecule(int(m))
            parts_c.append(c)
            parts_e.append(e)
            ptr.append(ptr[-1] + len(e))
        return MoleculeSet(np.concatenate(parts_c).astype(np.float64),
                           np.concatenate(parts_e).astype(np.int32),
                           np.asarray(ptr, dtype=np.int32))


def concat(mols: list) -> MoleculeSet:
    """Concatenate (coords, elem) pairs into one CSR batch."""
    ptr = [0]
    for c, e in mols:
        ptr.append(ptr[-1] + len(e))
    return MoleculeSet(np.concatenate([c for c, _ in mols]).astype(np.float64),
                       np.concatenate([e for _, e in mols]).astype(np.int32),
                       np.asarray(ptr, dtype=np.int32))


# ----------------------------------------------------------------------------
# geometry generators


def _min_dist_ok(pos: np.ndarray, new: np.ndarray, rmin: float) -> bool:
    if len(pos) == 0:
        return True
    return bool(np.min(np.sum((pos - new) ** 2, axis=1)) >= rmin * rmin)


def random_box(rng, n_mol: int, n_atoms: int, box: float = 4.0, rmin: float = 0.9,
               p_elem=(0.5, 0.125, 0.125, 0.125, 0.125)) -> MoleculeSet:
    """Molecules with atoms uniform in a cube, rejecting any pair closer than rmin."""
    mols = []
    for _ in range(n_mol):
        pos = []
        while len(pos) < n_atoms:
            cand = rng.uniform(0.0, box, size=3)
            if _min_dist_ok(np.asarray(pos).reshape(-1, 3), cand, rmin):
                pos.append(cand)
        elem = rng.choice(5, size=n_atoms, p=p_elem).astype(np.int32)
        mols.append((np.asarray(pos), elem))
    return concat(mols)


def _unit(rng) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def grow_molecule(rng, elements, bond_range=(1.0, 1.6), rmin: float = 0.9,
                  max_tries: int = 200):
    """Random bonded growth with a fixed element sequence.

    Heavy atoms must come before the hydrogens they carry: atom k bonds to an
    earlier heavy atom with free valence. Returns (coords [M,3], elem [M],
    bonds [(parent, child)]). Atoms that cannot be placed are dropped.
    """
    elements = list(elements)
    pos = [np.zeros(3)]
    elem = [elements[0]]
    free = [VALENCE[elements[0]]]
    bonds = []
    for e in elements[1:]:
        placed = False
        for _ in range(max_tries):
            parents = [i for i in range(len(pos)) if free[i] > 0 and elem[i] != H]
            if not parents:
                break
            p = parents[rng.integers(len(parents))]
            cand = pos[p] + rng.uniform(*bond_range) * _unit(rng)
            if _min_dist_ok(np.asarray(pos), cand, rmin):
                pos.append(cand)
                elem.append(e)
                free[p] -= 1
                free.append(VALENCE[e] - 1)
                bonds.append((p, len(pos) - 1))
                placed = True
                break
        if not placed and e != H:
            continue
    return np.asarray(pos), np.asarray(elem, dtype=np.int32), bonds


def _heavy_then_h(heavy, n_h):
    return list(heavy) + [H] * n_h


def random_composition(rng, m: int, p_h: float = 0.51,
                       heavy_mix=(0.72, 0.12, 0.15, 0.01)):
    """Element sequence for an m-atom molecule: heavy atoms first, then H.

    At least one heavy atom; the H count is capped by the free valence a
    tree of the drawn heavy atoms can offer.
    """
    n_h = int(rng.binomial(m, p_h))
    n_heavy = max(1, m - n_h)
    heavy = list(rng.choice([C, N, O, F], size=n_heavy, p=heavy_mix))
    if heavy[0] == F and n_heavy > 1:
        heavy[0] = C
    cap = sum(VALENCE[e] for e in heavy) - 2 * (n_heavy - 1)
    n_h = min(m - n_heavy, max(cap, 0))
    return _heavy_then_h(heavy, n_h)


def grow_batch(rng, compositions, bond_range=(1.0, 1.6), rmin: float = 0.9,
               max_tries: int = 64):
    """Random bonded growth of many molecules at once (same rules as
    ``grow_molecule``, vectorised over molecules). Atoms that cannot be placed
    after ``max_tries`` proposals are dropped. Returns a MoleculeSet whose
    ``bonds`` hold the growth tree in global atom indices."""
    n = len(compositions)
    lens = np.array([len(c) for c in compositions])
    mmax = int(lens.max())
    el = np.full((n, mmax), -1, dtype=np.int64)
    for i, c in enumerate(compositions):
        el[i, :len(c)] = c
    val = np.array(VALENCE)
    pos = np.full((n, mmax, 3), np.nan)
    pos[:, 0] = 0.0
    ok = np.zeros((n, mmax), dtype=bool)
    ok[:, 0] = True
    free = np.zeros((n, mmax), dtype=np.int64)
    free[:, 0] = val[el[:, 0]]
    parent = np.full((n, mmax), -1, dtype=np.int64)
    for k in range(1, mmax):
        todo = np.nonzero(lens > k)[0]
        for _ in range(max_tries):
            if len(todo) == 0:
                break
            elig = ok[todo, :k] & (free[todo, :k] > 0) & (el[todo, :k] != H)
            has = elig.any(axis=1)
            todo = todo[has]
            elig = elig[has]
            if len(todo) == 0:
                break
            keys = np.where(elig, rng.random(elig.shape), -1.0)
            p = np.argmax(keys, axis=1)
            u = rng.normal(size=(len(todo), 3))
            u /= np.linalg.norm(u, axis=1, keepdims=True)
            cand = pos[todo, p] + rng.uniform(*bond_range, size=(len(todo), 1)) * u
            d2 = np.sum((pos[todo, :k] - cand[:, None, :]) ** 2, axis=-1)
            d2 = np.where(ok[todo, :k], d2, np.inf)
            good = np.min(d2, axis=1) >= rmin * rmin
            g = todo[good]
            pos[g, k] = cand[good]
            ok[g, k] = True
            free[g, p[good]] -= 1
            free[g, k] = val[el[g, k]] - 1
            parent[g, k] = p[good]
            todo = todo[~good]
    mols, bonds, off = [], [], 0
    for i in range(n):
        keep = np.nonzero(ok[i, :lens[i]])[0]
        remap = -np.ones(mmax, dtype=np.int64)
        remap[keep] = np.arange(len(keep))
        mols.append((pos[i, keep], el[i, keep].astype(np.int32)))
        for k in keep[1:]:
            bonds.append((off + int(remap[parent[i, k]]), off + int(remap[k])))
        off += len(keep)
    s = concat(mols)
    s.bonds = bonds
    return s


def qm9_like(rng, n_mol: int, mean: float = 18.0, sd: float = 3.0,
             lo: int = 3, hi: int = 29) -> MoleculeSet:
    """QM9-shaped set: sizes round(TruncNormal(mean, sd)) on [lo, hi]."""
    sizes = []
    while len(sizes) < n_mol:
        m = np.rint(rng.normal(mean, sd, size=2 * n_mol)).astype(int)
        sizes.extend(int(v) for v in m[(m >= lo) & (m <= hi)])
    return grow_batch(rng, [random_composition(rng, m) for m in sizes[:n_mol]])


def _subtree(bonds, root_side: int, other: int, n: int):
    """Atoms reachable from `other` without crossing the bond (root_side, other)."""
    adj = [[] for _ in range(n)]
    for i, j in bonds:
        adj[i].append(j)
        adj[j].append(i)
    seen = {other}
    stack = [other]
    while stack:
        a = stack.pop()
        for b in adj[a]:
            if b == root_side and a == other:
                continue
            if b not in seen:
                seen.add(b)
                stack.append(b)
    return sorted(seen)


def _rotate_about(points, origin, axis, angle):
    axis = axis / np.linalg.norm(axis)
    p = points - origin
    c, s = math.cos(angle), math.sin(angle)
    rot = (p * c + np.cross(axis, p) * s + np.outer(p @ axis, axis) * (1.0 - c))
    return rot + origin


def conformations(rng, composition, n_conf: int, sd: float, n_rotatable: int = 0,
                  rmin: float = 0.9):
    """MD17/3BPA-shaped set: one grown reference, then per-conformation
    rotations about `n_rotatable` heavy-heavy tree bonds (angle U[-pi, pi],
    smaller side rotated) and Gaussian displacement of every coordinate; a
    rotation or displacement that brings two atoms closer than `rmin` is
    redrawn.

    Returns (MoleculeSet, reference coords, tree bonds of the reference).
    """
    while True:
        ref, elem, bonds = grow_molecule(rng, composition)
        if len(elem) == len(composition):
            break
    n = len(elem)
    heavy_bonds = [(i, j) for i, j in bonds if elem[i] != H and elem[j] != H]
    rot = []
    if n_rotatable:
        cands = [b for b in heavy_bonds
                 if 1 < len(_subtree(bonds, b[0], b[1], n)) < n - 1]
        idx = rng.choice(len(cands), size=min(n_rotatable, len(cands)), replace=False)
        rot = [cands[k] for k in idx]
    sides = []
    for i, j in rot:
        side = _subtree(bonds, i, j, n)
        if len(side) > n // 2:
            side = _subtree(bonds, j, i, n)
            i, j = j, i
        sides.append((i, j, side))
    def clashes(x):
        d2 = np.sum((x[:, None, :] - x[None, :, :]) ** 2, axis=-1) + np.eye(n) * 1e9
        return np.nonzero((d2 < rmin * rmin).any(axis=1))[0]

    mols = []
    while len(mols) < n_conf:
        # rotations first (redrawn until the rigid geometry has no contact < rmin),
        # then Gaussian displacements (redrawn for the atoms of a contact < rmin)
        for _ in range(100):
            x = ref.copy()
            for i, j, side in sides:
                x[side] = _rotate_about(x[side], x[i], x[j] - x[i],
                                        rng.uniform(-math.pi, math.pi))
            if len(clashes(x)) == 0:
                break
        else:
            continue
        y = x + rng.normal(0.0, sd, size=x.shape)
        for _ in range(100):
            bad = clashes(y)
            if len(bad) == 0:
                break
            y[bad] = x[bad] + rng.normal(0.0, sd, size=(len(bad), 3))
        else:
            continue
        mols.append((y, elem.copy()))
    s = concat(mols)
    s.bonds = bonds
    return s, ref, bonds


ASPIRIN_LIKE = [C] * 9 + [O] * 4 + [H] * 8            # C9H8O4, 21 atoms
BPA3_LIKE = [C] * 12 + [N] * 2 + [O] + [H] * 12        # C12H12N2O, 27 atoms


def serving_molecules(rng, n_mol: int, lo: int = 5, hi: int = 200) -> MoleculeSet:
    """Molecules with sizes log-uniform on [lo, hi], grown with H/C/N/O/F."""
    sizes = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_mol))).astype(int)
    return grow_batch(rng, [random_composition(rng, int(m)) for m in sizes])


# ----------------------------------------------------------------------------
# periodic systems: stand-ins for the paper's liquid water and MOF crystal


@dataclass
class PeriodicSet:
    coords: np.ndarray   # float64 [N, 3] (inside the cell)
    elem: np.ndarray     # int32 [N]
    cell: np.ndarray     # float64 [3, 3] lattice vectors as rows

    @property
    def n_atoms(self) -> int:
        return len(self.elem)


def _periodic_ok(tree_pts, pts, box, rmin):
    """True where a point of pts keeps rmin from every point of tree_pts (orthorhombic box)."""
    from scipy.spatial import cKDTree
    if len(tree_pts) == 0:
        return np.ones(len(pts), dtype=bool)
    t = cKDTree(np.mod(tree_pts, box), boxsize=box)
    d, _ = t.query(np.mod(pts, box), k=1)
    return d >= rmin


def water_box(rng, n_waters: int, density_g_cm3: float = 1.0) -> PeriodicSet:
    """Liquid-water-shaped periodic box: n rigid waters (O-H 0.957 A, H-O-H
    104.5 deg) in a cubic cell at the given density (29.9 A^3 per molecule at
    1 g/cm^3); oxygens on a jittered cubic grid, random orientations, and the
    waters with an atom closer than 1.2 A to another water's are re-oriented
    until none is."""
    from scipy.spatial import cKDTree
    L = (n_waters * 18.015 / (6.02214076e23 * density_g_cm3) * 1e24) ** (1.0 / 3.0)
    k = int(math.ceil(n_waters ** (1.0 / 3.0)))
    a = L / k
    grid = np.stack(np.meshgrid(*[np.arange(k)] * 3, indexing="ij"), axis=-1).reshape(-1, 3)[:n_waters]
    oxy = (grid + 0.5) * a + rng.uniform(-0.25, 0.25, size=(n_waters, 3))
    box = np.array([L, L, L])
    ang = math.radians(104.5)

    def orient(m):
        u = rng.normal(size=(m, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        v = rng.normal(size=(m, 3))
        v -= u * np.sum(u * v, axis=1, keepdims=True)
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        return 0.957 * u, 0.957 * (math.cos(ang) * u + math.sin(ang) * v)

    h1, h2 = orient(n_waters)
    for _ in range(100):
        pts = np.concatenate([oxy, oxy + h1, oxy + h2])            # [3n, 3]: O block, H1 block, H2 block
        pairs = cKDTree(np.mod(pts, box), boxsize=box).query_pairs(1.2, output_type="ndarray")
        mol = np.tile(np.arange(n_waters), 3)
        bad = pairs[mol[pairs[:, 0]] != mol[pairs[:, 1]]] if len(pairs) else pairs
        if len(bad) == 0:
            break
        redo = np.unique(mol[bad[:, 1]])
        h1[redo], h2[redo] = orient(len(redo))
    atoms = np.stack([oxy, oxy + h1, oxy + h2], axis=1).reshape(-1, 3)
    elem = np.tile(np.array([O, H, H], dtype=np.int32), n_waters)
    return PeriodicSet(np.mod(atoms, box), elem, np.diag(box))


def framework_crystal(rng, n_atoms: int, density: float = 0.075, rmin: float = 1.05,
                      fractions=(0.35, 0.45, 0.08, 0.12, 0.0)) -> PeriodicSet:
    """MOF-shaped periodic crystal: n atoms (H/C/N/O/F fractions) at a framework's
    number density (atoms per A^3) in an orthorhombic cell with edges in ratio
    1 : 1.1 : 1.2, positions by random sequential insertion keeping rmin."""
    vol = n_atoms / density
    a = (vol / (1.0 * 1.1 * 1.2)) ** (1.0 / 3.0)
    box = np.array([a, 1.1 * a, 1.2 * a])
    from scipy.spatial import cKDTree
    pts = np.zeros((0, 3))
    while len(pts) < n_atoms:
        cand = rng.uniform(0.0, 1.0, size=(n_atoms - len(pts) + 16, 3)) * box
        cand = cand[_periodic_ok(pts, cand, box, rmin)]
        # candidates must also keep rmin from each other: of a close pair the later one goes
        if len(cand) > 1:
            pairs = cKDTree(cand, boxsize=box).query_pairs(rmin, output_type="ndarray")
            drop = np.zeros(len(cand), dtype=bool)
            drop[pairs[:, 1] if len(pairs) else []] = True
            cand = cand[~drop]
        pts = np.concatenate([pts, cand[: n_atoms - len(pts)]])
    elem = rng.choice(5, size=n_atoms, p=np.asarray(fractions) / np.sum(fractions)).astype(np.int32)
    return PeriodicSet(pts[:n_atoms], elem, np.diag(box))


def poisson_arrivals(rng, rate_per_s: float, duration_s: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process."""
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            return np.asarray(out)
        out.append(t)


# ----------------------------------------------------------------------------
# random parameters the feature map draws (passed in to both sides)


def sorf_draw(rng, n_features: int, d: int, n_transform: int):
    """Rademacher signs [n_stack, T, d] (+1/-1, int8) and phases b ~ U[0, 2 pi) [N_F]."""
    assert n_features % d == 0
    n_stack = n_features // d
    signs = rng.choice(np.array([-1, 1], dtype=np.int8), size=(n_stack, n_transform, d))
    b = rng.uniform(0.0, 2.0 * math.pi, size=n_features)
    return signs, b


def rff_draw(rng, n_features: int, d: int):
    """Standard normal matrix G [N_F, d] and phases b ~ U[0, 2 pi)."""
    return rng.normal(size=(n_features, d)), rng.uniform(0.0, 2.0 * math.pi, size=n_features)


# ----------------------------------------------------------------------------
# synthetic targets: random pair potentials with analytic forces


@dataclass
class PairPotential:
    """Lennard-Jones between all pairs plus harmonic springs on listed bonds.

    eps, sig [5,5] symmetric per element pair; k_b, r0 per bond (or None).
    """

    eps: np.ndarray
    sig: np.ndarray
    bonds: list = field(default_factory=list)
    k_b: np.ndarray | None = None
    r0: np.ndarray | None = None
    lj_exclude_bonded: bool = False


def random_lj(rng) -> PairPotential:
    eps = np.zeros((5, 5))
    sig = np.zeros((5, 5))
    for a in range(5):
        for b in range(a, 5):
            eps[a, b] = eps[b, a] = rng.uniform(0.005, 0.05)
            sig[a, b] = sig[b, a] = rng.uniform(0.6, 0.9)
    return PairPotential(eps, sig)


def add_bonds(rng, pot: PairPotential, bonds, ref_coords=None, r0_by_pair=None, elem=None,
              k_range=(10.0, 30.0)) -> PairPotential:
    """Harmonic springs on `bonds` with k ~ U[k_range]; r0 from a reference geometry
    or from a per-element-pair table."""
    bonds = list(bonds)
    k = rng.uniform(*k_range, size=len(bonds))
    if ref_coords is not None:
        r0 = np.array([np.linalg.norm(ref_coords[i] - ref_coords[j]) for i, j in bonds])
    else:
        r0 = np.array([r0_by_pair[elem[i], elem[j]] for i, j in bonds])
    return PairPotential(pot.eps, pot.sig, bonds, k, r0, pot.lj_exclude_bonded)


def potential_energy_forces(pot: PairPotential, coords, elem, bonds_local=None,
                            k=None, r0=None, exclude=None):
    """Energy and analytic forces of one molecule (FP64)."""
    x = np.asarray(coords, dtype=np.float64)
    n = len(x)
    f = np.zeros_like(x)
    iu, ju = np.triu_indices(n, 1)
    if exclude:
        keep = np.array([(a, b) not in exclude for a, b in zip(iu, ju)], dtype=bool)
        iu, ju = iu[keep], ju[keep]
    rv = x[ju] - x[iu]
    r = np.sqrt(np.sum(rv * rv, axis=1))
    ep = pot.eps[elem[iu], elem[ju]]
    sg = pot.sig[elem[iu], elem[ju]]
    sr6 = (sg / r) ** 6
    e_tot = float(np.sum(4.0 * ep * (sr6 * sr6 - sr6)))
    g = (4.0 * ep * (-12.0 * sr6 * sr6 + 6.0 * sr6) / r)[:, None] * rv / r[:, None]
    np.add.at(f, ju, -g)
    np.add.at(f, iu, g)
    if bonds_local is not None and len(bonds_local):
        bl = np.asarray(bonds_local)
        rv = x[bl[:, 1]] - x[bl[:, 0]]
        r = np.sqrt(np.sum(rv * rv, axis=1))
        e_tot += float(np.sum(0.5 * k * (r - r0) ** 2))
        g = (k * (r - r0))[:, None] * rv / r[:, None]
        np.add.at(f, bl[:, 1], -g)
        np.add.at(f, bl[:, 0], g)
    return e_tot, f


def targets(pot: PairPotential, mols: MoleculeSet, with_forces: bool = False):
    """Energies [n_mol] (and forces [n_atoms, 3]) of every molecule in the set.

    Bonds in ``pot.bonds`` are global atom indices; they are mapped to each
    molecule. When ``pot.lj_exclude_bonded`` is set, bonded pairs carry no LJ term.
    """
    E = np.zeros(mols.n_mol)
    Fo = np.zeros((mols.n_atoms, 3))
    by_mol = [[] for _ in range(mols.n_mol)]
    if pot.bonds:
        owner = np.searchsorted(mols.mol_ptr, np.arange(mols.n_atoms), side="right") - 1
        for q, (i, j) in enumerate(pot.bonds):
            by_mol[owner[i]].append(q)
    for m in range(mols.n_mol):
        a = int(mols.mol_ptr[m])
        c, e = mols.molecule(m)
        qs = by_mol[m]
        bl = [(pot.bonds[q][0] - a, pot.bonds[q][1] - a) for q in qs]
        excl = set((min(i, j), max(i, j)) for i, j in bl) if pot.lj_exclude_bonded else None
        en, fo = potential_energy_forces(
            pot, c, e, bl if qs else None,
            pot.k_b[qs] if qs else None, pot.r0[qs] if qs else None, excl)
        E[m] = en
        Fo[a:a + len(e)] = fo
    return (E, Fo) if with_forces else E


def replicate_bonds(bonds, n_atoms_per_mol: int, n_mol: int):
    """Tree bonds of a reference molecule repeated for every conformation."""
    return [(m * n_atoms_per_mol + i, m * n_atoms_per_mol + j)
            for m in range(n_mol) for i, j in bonds]


# ----------------------------------------------------------------------------
# the five workloads


@dataclass
class Workload:
    name: str
    mols: MoleculeSet
    energies: np.ndarray
    forces: np.ndarray | None
    params_column: str          # "E" or "EF" column of the FCHL19 parameter table
    n2: int
    n3: int
    d: int
    n_features: int
    n_transform: int
    sigma: float
    lam: float
    signs: np.ndarray
    b: np.ndarray
    test: MoleculeSet | None = None
    test_energies: np.ndarray | None = None
    test_forces: np.ndarray | None = None
    potential: PairPotential | None = None


def workload(config: int, scale: float = 1.0, sigma: float | None = None) -> Workload:
    """Build one of the five workloads. ``scale`` < 1 shrinks the molecule count
    (used for bounded samples and quick tests); the shapes stay the same."""
    rng = rng_for(config)
    if config == 0:
        n_mol = max(1, int(round(64 * scale)))
        mols = random_box(rng, n_mol, 9)
        pot = random_lj(rng)
        E = targets(pot, mols)
        signs, b = sorf_draw(rng, 512, 64, 3)
        return Workload("parity-64x9", mols, E, None, "E", 24, 22, 64, 512, 3,
                        2.0 if sigma is None else sigma, 1e-6, signs, b, potential=pot)
    if config == 1:
        n_mol = max(1, int(round(100_000 * scale)))
        mols = qm9_like(rng, n_mol)
        pot = random_lj(rng)
        r0 = rng.uniform(1.0, 1.6, size=(5, 5))
        r0 = np.triu(r0) + np.triu(r0, 1).T
        pot = add_bonds(rng, pot, mols.bonds, r0_by_pair=r0, elem=mols.elem)
        pot.lj_exclude_bonded = True
        E = targets(pot, mols)
        signs, b = sorf_draw(rng, 16384, 128, 3)
        return Workload("qm9-shaped-100k", mols, E, None, "E", 24, 22, 128, 16384, 3,
                        2.0 if sigma is None else sigma, 1e-6, signs, b, potential=pot)
    if config in (2, 3):
        comp = ASPIRIN_LIKE if config == 2 else BPA3_LIKE
        n_train = 1000 if config == 2 else 500
        n_test = 0 if config == 2 else 2000
        n_train = max(1, int(round(n_train * scale)))
        n_test = int(round(n_test * scale))
        sd = 0.1 if config == 2 else 0.15
        nrot = 0 if config == 2 else 3
        allm, ref, bonds = conformations(rng, comp, n_train + n_test, sd, nrot)
        pot = random_lj(rng)
        gb = replicate_bonds(bonds, len(comp), n_train + n_test)
        pot = add_bonds(rng, pot, bonds, ref_coords=ref)
        pot = PairPotential(pot.eps, pot.sig, gb, np.tile(pot.k_b, n_train + n_test),
                            np.tile(pot.r0, n_train + n_test), True)
        E, Fo = targets(pot, allm, with_forces=True)
        nf = 8192 if config == 2 else 16384
        signs, b = sorf_draw(rng, nf, 128, 3)
        tr = allm.subset(range(n_train))
        na = int(tr.mol_ptr[-1])
        w = Workload("md17-shaped-1k" if config == 2 else "3bpa-shaped-500",
                     tr, E[:n_train], Fo[:na], "EF", 24, 22, 128, nf, 3,
                     2.0 if sigma is None else sigma, 1e-6, signs, b)
        if n_test:
            w.test = allm.subset(range(n_train, n_train + n_test))
            w.test_energies = E[n_train:]
            w.test_forces = Fo[na:]
        return w
    if config == 4:
        n_mol = max(1, int(round(2000 * scale)))
        mols = serving_molecules(rng, n_mol)
        signs, b = sorf_draw(rng, 16384, 128, 3)
        return Workload("serving-5-200", mols, np.zeros(n_mol), None, "EF", 24, 22, 128,
                        16384, 3, 2.0 if sigma is None else sigma, 1e-6, signs, b)
    raise ValueError(f"unknown workload {config}")
