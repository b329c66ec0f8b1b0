"""Pins for the FP64 model oracle: forces and force rows against central finite
differences, conservation laws, and the atomic energy partition."""
import math

import numpy as np
import pytest

from oracle import fchl19, model, regression
from paper_2206_01580_gb300 import synth


@pytest.fixture(scope="module")
def small():
    rng = np.random.default_rng(11)
    mols = synth.random_box(rng, 3, 6)
    p = fchl19.params("EF", n2=24, n3=22)
    reps = fchl19.representation_batch(mols.coords, mols.elem, mols.mol_ptr, p)
    U = rng.normal(size=(5, p.rep_dim, 16)) * 0.1
    signs, b = synth.sorf_draw(rng, 64, 16, 3)
    m = model.sorf_model(p, U, signs, b, sigma=1.5, alpha=rng.normal(size=64))
    return mols, m


def test_forces_match_central_differences(small):
    mols, m = small
    E, F = model.energies_forces(mols.coords, mols.elem, mols.mol_ptr, m)
    h = 1e-4
    for mol in range(mols.n_mol):
        a, b = int(mols.mol_ptr[mol]), int(mols.mol_ptr[mol + 1])
        for k in range(a, b):
            for ax in range(3):
                xp, xm = mols.coords.copy(), mols.coords.copy()
                xp[k, ax] += h
                xm[k, ax] -= h
                ep = model.energies_forces(xp, mols.elem, mols.mol_ptr, m, forces=False)[mol]
                em = model.energies_forces(xm, mols.elem, mols.mol_ptr, m, forces=False)[mol]
                assert -(ep - em) / (2 * h) == pytest.approx(F[k, ax], rel=1e-5, abs=1e-7)


def test_forces_sum_and_torque_vanish(small):
    mols, m = small
    _, F = model.energies_forces(mols.coords, mols.elem, mols.mol_ptr, m)
    for mol in range(mols.n_mol):
        a, b = int(mols.mol_ptr[mol]), int(mols.mol_ptr[mol + 1])
        scale = np.abs(F[a:b]).max()
        np.testing.assert_allclose(F[a:b].sum(0), 0, atol=1e-12 * scale)
        np.testing.assert_allclose(np.cross(mols.coords[a:b], F[a:b]).sum(0), 0, atol=1e-11 * scale)


def test_force_rows_match_finite_differences(small):
    mols, m = small
    rows = model.force_rows(mols.coords, mols.elem, mols.mol_ptr, m)
    h = 1e-4
    for k, ax in [(0, 0), (2, 1), (7, 2), (12, 0)]:
        mol = int(np.searchsorted(mols.mol_ptr, k, side="right") - 1)
        xp, xm = mols.coords.copy(), mols.coords.copy()
        xp[k, ax] += h
        xm[k, ax] -= h
        Zp = model.feature_matrix(xp, mols.elem, mols.mol_ptr, m)[mol]
        Zm = model.feature_matrix(xm, mols.elem, mols.mol_ptr, m)[mol]
        np.testing.assert_allclose(rows[3 * k + ax], -(Zp - Zm) / (2 * h), rtol=1e-5,
                                   atol=1e-8 * np.abs(rows[3 * k + ax]).max())


def test_energy_is_sum_of_atomic_energies_and_z_alpha(small):
    mols, m = small
    E = model.energies_forces(mols.coords, mols.elem, mols.mol_ptr, m, forces=False)
    eps = model.atom_energies(mols.coords, mols.elem, mols.mol_ptr, m)
    Z = model.feature_matrix(mols.coords, mols.elem, mols.mol_ptr, m)
    np.testing.assert_allclose(E, np.add.reduceat(eps, mols.mol_ptr[:-1]), rtol=1e-12)
    np.testing.assert_allclose(E, Z @ m.alpha, rtol=1e-12)


def test_feature_pipeline_is_project_then_map(small):
    """Z rows equal sum over atoms of z(rho^T U_e), assembled from the separate stages."""
    mols, m = small
    reps = fchl19.representation_batch(mols.coords, mols.elem, mols.mol_ptr, m.p)
    x = regression.project(reps, mols.elem, m.U)
    z = math.sqrt(2 / m.n_features) * np.cos(x @ m.W.T + m.b)
    want = regression.segment_sum(z, mols.mol_ptr)
    np.testing.assert_allclose(model.feature_matrix(mols.coords, mols.elem, mols.mol_ptr, m),
                               want, rtol=1e-12, atol=1e-14)


def test_training_interpolates_when_features_exceed_data():
    """Energy-only training on the parity workload: N_F = 512 > 64 molecules, so
    with lambda = 1e-6 the fit reproduces the training energies closely."""
    w = synth.workload(0, scale=0.5)
    p = fchl19.params("E", n2=24, n3=22)
    reps = fchl19.representation_batch(w.mols.coords, w.mols.elem, w.mols.mol_ptr, p)
    U = regression.pca_bases(reps, w.mols.elem, 5, w.d)
    m = model.sorf_model(p, U, w.signs, w.b, w.sigma)
    alpha, res = model.train(w.mols.coords, w.mols.elem, w.mols.mol_ptr, w.energies, m, w.lam)
    m.alpha = alpha
    E = model.energies_forces(w.mols.coords, w.mols.elem, w.mols.mol_ptr, m, forces=False)
    assert res < 1e-10
    assert np.mean(np.abs(E - w.energies)) < 1e-3 * np.mean(np.abs(w.energies))


def test_energy_force_training_fits_forces():
    """Energy+force rows: the fitted model's forces match the training forces
    better than the zero model does."""
    w = synth.workload(2, scale=0.01)          # 10 conformations x 21 atoms
    p = fchl19.params("EF", n2=24, n3=22)
    reps = fchl19.representation_batch(w.mols.coords, w.mols.elem, w.mols.mol_ptr, p)
    U = regression.pca_bases(reps, w.mols.elem, 5, 16)
    signs, b = synth.sorf_draw(np.random.default_rng(0), 256, 16, 3)
    m = model.sorf_model(p, U, signs, b, sigma=2.0)
    alpha, res = model.train(w.mols.coords, w.mols.elem, w.mols.mol_ptr, w.energies, m, 1e-6,
                             forces=w.forces)
    m.alpha = alpha
    E, F = model.energies_forces(w.mols.coords, w.mols.elem, w.mols.mol_ptr, m)
    assert np.mean(np.abs(F - w.forces)) < 0.5 * np.mean(np.abs(w.forces))
