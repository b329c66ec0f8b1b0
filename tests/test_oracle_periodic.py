"""Pins for the FP64 oracle's periodic FCHL19 (the paper's periodic MOF and
water systems): a molecule in a large box is the molecule, lattice
translations and supercells change nothing, a rotated crystal has the same
representation, the simple-cubic lattice's two-body block is a closed form
over its coordination shells, and forces are the derivative of the energy."""
import math

import numpy as np
import pytest
import scipy.stats
import torch

from oracle import fchl19

H, C, N, O = 0, 1, 2, 3


def P(column="E"):
    return fchl19.params(column, n2=24, n3=22)


def per(x, elem, cell, p):
    R = torch.as_tensor(np.asarray(x, dtype=np.float64))
    return fchl19.representation_periodic(R, np.asarray(elem), np.asarray(cell, dtype=np.float64), p).numpy()


# three atoms in a skewed cell whose shortest lattice vector (3.3 A) is well
# inside the cutoff: many images of every atom, including its own
CELL = np.array([[3.3, 0.0, 0.0], [0.8, 3.6, 0.0], [0.3, -0.5, 3.9]])
X3 = np.array([[0.2, 0.1, 0.3], [1.4, 0.9, 0.2], [0.7, 2.0, 1.8]])
E3 = [C, O, H]


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def test_molecule_in_a_large_box_is_the_molecule():
    p = P()
    x = np.array([[0, 0, 0], [1.09, 0, 0], [-0.36, 1.03, 0], [-0.36, -0.51, 0.89], [1.5, 1.2, -0.7]])
    e = [C, H, H, H, O]
    mol = fchl19.representation(torch.as_tensor(x), np.asarray(e), p).numpy()
    got = per(x + 5.0, e, np.eye(3) * 40.0, p)
    assert rel(got, mol) <= 1e-13


def test_lattice_translation_of_an_atom_changes_nothing():
    p = P("EF")
    ref = per(X3, E3, CELL, p)
    y = X3.copy()
    y[1] += CELL[0] - 2 * CELL[2]
    y[2] -= CELL[1]
    assert rel(per(y, E3, CELL, p), ref) <= 1e-12


def test_supercell_gives_the_same_environments():
    p = P()
    ref = per(X3, E3, CELL, p)
    xs = np.concatenate([X3, X3 + CELL[0]])
    sc = np.array([2 * CELL[0], CELL[1], CELL[2]])
    got = per(xs, E3 + E3, sc, p)
    assert rel(got[:3], ref) <= 1e-12
    assert rel(got[3:], ref) <= 1e-12


def test_rotated_crystal_has_the_same_representation():
    p = P()
    Q, _ = np.linalg.qr(np.random.default_rng(3).normal(size=(3, 3)))
    ref = per(X3, E3, CELL, p)
    assert rel(per(X3 @ Q.T, E3, CELL @ Q.T, p), ref) <= 1e-11


@pytest.mark.parametrize("a", [2.5, 3.1])
def test_simple_cubic_two_body_is_a_sum_over_shells(a):
    """One H atom in a cubic cell of side a: neighbours are the lattice points
    n a (n a nonzero integer triple) closer than r_cut; the two-body block is
    the diatomic closed form summed over them, and the three-body terms sit in
    the (H, H) pair block only."""
    p = P()
    out = per([[0.3, 0.2, 0.1]], [H], np.eye(3) * a, p)[0]
    m = int(math.ceil(p.rcut / a))
    n = np.stack(np.meshgrid(*[np.arange(-m, m + 1)] * 3, indexing="ij"), -1).reshape(-1, 3)
    r = a * np.sqrt(np.sum(n * n, axis=1))
    r = r[(r > 0) & (r < p.rcut)]
    Rs = p.rcut * np.arange(1, p.n2 + 1) / p.n2
    want = np.zeros(p.n2)
    for rr in r:
        s = math.sqrt(math.log(1 + p.eta2 / rr**2))
        mu = math.log(rr / math.sqrt(1 + p.eta2 / rr**2))
        fc = 0.5 * (math.cos(math.pi * rr / p.rcut) + 1)
        want += fc * rr ** (-p.N2) * scipy.stats.lognorm.pdf(Rs, s=s, scale=math.exp(mu))
    np.testing.assert_allclose(out[H * p.n2:(H + 1) * p.n2], want, rtol=1e-12, atol=1e-300)
    assert np.all(out[p.n2:p.n_el * p.n2] == 0.0)
    hh = p.n_el * p.n2 + fchl19.pair_index(H, H, p.n_el) * p.n3 * 2
    three = out[p.n_el * p.n2:]
    assert np.any(out[hh:hh + p.n3 * 2] != 0.0)
    mask = np.ones_like(three, dtype=bool)
    mask[hh - p.n_el * p.n2:hh - p.n_el * p.n2 + p.n3 * 2] = False
    assert np.all(three[mask] == 0.0)


def test_periodic_forces_are_the_energy_gradient():
    p = P("EF")
    w = torch.as_tensor(np.random.default_rng(5).normal(size=p.rep_dim))

    def energy(x):
        R = torch.as_tensor(x, dtype=torch.float64)
        return float((fchl19.representation_periodic(R, np.asarray(E3), CELL, p) @ w).sum())

    R = torch.tensor(X3, dtype=torch.float64, requires_grad=True)
    (g,) = torch.autograd.grad((fchl19.representation_periodic(R, np.asarray(E3), CELL, p) @ w).sum(), R)
    h = 1e-4
    fd = np.zeros_like(X3)
    for i in range(3):
        for k in range(3):
            xp, xm = X3.copy(), X3.copy()
            xp[i, k] += h
            xm[i, k] -= h
            fd[i, k] = (energy(xp) - energy(xm)) / (2 * h)
    assert rel(g.numpy(), fd) <= 1e-6
    # the energy of a crystal does not change when every atom moves together
    assert np.max(np.abs(g.numpy().sum(0))) <= 1e-9 * np.max(np.abs(g.numpy()))


def test_periodic_energy_forces_are_minus_the_energy_gradient():
    """The periodic energy + force oracle: forces equal central differences of
    its energies (h = 1e-4 A) and sum to zero (translation invariance)."""
    from oracle import model, regression, sorf
    p = P("EF")
    rng = np.random.default_rng(3)
    reps = per(X3, E3, CELL, p)
    U = regression.pca_bases(reps, np.asarray(E3), 5, 16)
    signs = rng.choice([-1, 1], size=(4, 3, 16))
    b = rng.uniform(0, 2 * math.pi, size=64)
    m = model.Model(p, U, sorf.sorf_matrix(signs, 2.0), b, rng.normal(size=64))
    E, F = model.periodic_energy_forces(X3, E3, CELL, m)
    h = 1e-4
    for k in range(3):
        for a in range(3):
            xp, xm = X3.copy(), X3.copy()
            xp[k, a] += h
            xm[k, a] -= h
            fd = -(model.periodic_energy_forces(xp, E3, CELL, m)[0] -
                   model.periodic_energy_forces(xm, E3, CELL, m)[0]) / (2 * h)
            assert abs(fd - F[k, a]) <= 1e-6 * max(1.0, np.abs(F).max()), (k, a, fd, F[k, a])
    assert np.max(np.abs(F.sum(axis=0))) <= 1e-9 * max(1.0, np.abs(F).max())
