"""GPU parity at the production configuration (N_F = 16384, d = 128, T = 3,
sigma = 2), through the C ABI, against the FP64 oracle:

* energy + force prediction on molecules of 5 to ~200 atoms (sizes on both
  sides of the 32-atom switch of the FCHL19 adjoint), weights of unit scale;
* force rows -dZ/dr of two 27-atom 3BPA-shaped conformations (E+F training rows);
* the SORF segment sum on projected representations of QM9-shaped molecules
  (the feature kernels' inputs as training meets them), and the range check
  of the phase reduction.

Tolerances: energies <= 1e-4 eV per atom, forces <= 1e-3 eV/A (the stated
bounds); force rows <= 2e-4 of the molecule block's largest entry (the FP32
forward-mode chain, as at smaller N_F); Z <= 2e-5 sqrt(2/N_F) per atom summed.
"""
import math

import numpy as np
import pytest
import torch

from oracle import fchl19 as o_fchl19
from oracle import model as o_model
from oracle import regression as o_reg
from oracle import sorf as o_sorf
from paper_2206_01580_gb300 import synth

pytestmark = pytest.mark.gpu

NF, D, T, SIGMA = 16384, 128, 3, 2.0


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_01580_gb300 import qmlr
    qmlr.lib()
    return qmlr


def gpu_params(column):
    from paper_2206_01580_gb300.params import from_table
    return from_table(column, n2=24, n3=22)


def sizes_5_to_200():
    """Eleven serving-shaped molecules whose sizes spread over 5..~200 atoms."""
    pool = synth.serving_molecules(synth.rng_for(4, 71), 400, lo=5, hi=200)
    sz = pool.sizes()
    pick = []
    for t in (5, 12, 24, 31, 33, 47, 64, 90, 130, 170, 199):
        cost = np.abs(sz - t).astype(float)
        cost[pick] = np.inf
        pick.append(int(np.argmin(cost)))
    return synth.concat([pool.molecule(i) for i in pick])


def test_predict_ef_production_config_5_to_200_atoms(q):
    mols = sizes_5_to_200()
    n = mols.sizes()
    assert n.min() <= 6 and n.max() >= 180 and np.any((n > 32) & (n < 60))
    po = o_fchl19.params("EF", n2=24, n3=22)
    reps = o_fchl19.representation_batch(mols.coords, mols.elem, mols.mol_ptr, po)
    U = o_reg.pca_bases(reps, mols.elem, 5, D).astype(np.float32)
    rng = np.random.default_rng(5)
    signs, b = synth.sorf_draw(rng, NF, D, T)
    b = b.astype(np.float32)
    alpha = rng.normal(size=NF).astype(np.float32)
    om = o_model.sorf_model(po, U.astype(np.float64), signs, b.astype(np.float64), SIGMA, alpha.astype(np.float64))
    E_ref, F_ref = o_model.energies_forces(mols.coords, mols.elem, mols.mol_ptr, om)
    m = q.Model(gpu_params("EF"), int(n.max()), U, signs, T, b, SIGMA, alpha)
    E, F = m.predict(mols.coords, mols.elem, mols.mol_ptr)
    E, F = E.cpu().numpy(), F.cpu().numpy()
    assert q.device_status() == 0
    m.close()
    assert np.all(np.abs(E - E_ref) <= 1e-4 * n), np.max(np.abs(E - E_ref) / n)
    err = np.abs(F - F_ref).max(axis=1)
    assert np.max(err) <= 1e-3, (np.max(err), np.abs(F_ref).max())
    # the largest molecules are not the easy ones: their forces are large too
    big = np.repeat(n, n) >= 130
    assert np.abs(F_ref[big]).max() > 1.0


def test_predict_ef_tensor_core_sorf_on_a_large_batch(q):
    """Batches of >= 8192 atoms take the tensor-core SORF energies + gradients:
    twelve shuffled copies of the 5-200-atom set (~9.6 k atoms) against the
    oracle (same bounds), against the FWHT kernel of the same model, and every
    copy of a molecule bitwise equal to the others (the result does not depend
    on the molecule's place in the batch)."""
    base = sizes_5_to_200()
    nb = base.sizes()
    po = o_fchl19.params("EF", n2=24, n3=22)
    reps = o_fchl19.representation_batch(base.coords, base.elem, base.mol_ptr, po)
    U = o_reg.pca_bases(reps, base.elem, 5, D).astype(np.float32)
    rng = np.random.default_rng(6)
    signs, b = synth.sorf_draw(rng, NF, D, T)
    b = b.astype(np.float32)
    alpha = rng.normal(size=NF).astype(np.float32)
    om = o_model.sorf_model(po, U.astype(np.float64), signs, b.astype(np.float64), SIGMA, alpha.astype(np.float64))
    E_ref, F_ref = o_model.energies_forces(base.coords, base.elem, base.mol_ptr, om)
    order = np.random.default_rng(7).permutation(np.tile(np.arange(base.n_mol), 12))
    mols = synth.concat([base.molecule(int(i)) for i in order])
    assert mols.n_atoms >= 8192
    m = q.Model(gpu_params("EF"), int(nb.max()), U, signs, T, b, SIGMA, alpha)
    assert m.sorf_tc
    E, F = (t.cpu().numpy() for t in m.predict(mols.coords, mols.elem, mols.mol_ptr))
    m.set_sorf_tc(False)
    E2, F2 = (t.cpu().numpy() for t in m.predict(mols.coords, mols.elem, mols.mol_ptr))
    assert q.device_status() == 0
    m.close()
    ptr = mols.mol_ptr
    first = {}
    for k, i in enumerate(order):
        a, e = int(ptr[k]), int(ptr[k + 1])
        ra, re_ = int(base.mol_ptr[i]), int(base.mol_ptr[i + 1])
        assert abs(E[k] - E_ref[i]) <= 1e-4 * nb[i]
        assert np.max(np.abs(F[a:e] - F_ref[ra:re_])) <= 1e-3
        assert abs(E[k] - E2[k]) <= 1e-4 * nb[i] and np.max(np.abs(F[a:e] - F2[a:e])) <= 1e-3
        if i in first:
            k0, a0, e0 = first[i]
            assert E[k] == E[k0] and np.array_equal(F[a:e], F[a0:e0])
        else:
            first[i] = (k, a, e)


def test_force_rows_production_config_3bpa_shaped(q):
    from paper_2206_01580_gb300 import pipeline
    w = synth.workload(3, scale=0.004)                  # two 27-atom conformations
    mols = w.mols
    assert mols.n_mol == 2 and np.all(mols.sizes() == 27)
    po = o_fchl19.params("EF", n2=24, n3=22)
    reps = o_fchl19.representation_batch(mols.coords, mols.elem, mols.mol_ptr, po)
    U = o_reg.pca_bases(reps, mols.elem, 5, D).astype(np.float32)
    b = w.b.astype(np.float32)
    om = o_model.sorf_model(po, U.astype(np.float64), w.signs, b.astype(np.float64), SIGMA)
    ref = o_model.force_rows(mols.coords, mols.elem, mols.mol_ptr, om)
    Zref = o_model.feature_matrix(mols.coords, mols.elem, mols.mol_ptr, om)
    spec = pipeline.spec_from(gpu_params("EF"), D, w.signs, b, SIGMA)
    batch = pipeline.Batch.from_host(mols.coords, mols.elem, mols.mol_ptr)
    rows = pipeline.energy_force_rows(batch, spec, torch.as_tensor(U).cuda()).cpu().numpy()
    assert q.device_status() == 0
    assert rows.shape == (2 + 3 * 54, NF)
    np.testing.assert_allclose(rows[:2], Zref, atol=2e-5 * math.sqrt(2.0 / NF) * 27)
    for m in range(2):
        blk_ref = ref[3 * 27 * m:3 * 27 * (m + 1)]
        blk = rows[2 + 3 * 27 * m:2 + 3 * 27 * (m + 1)]
        assert np.max(np.abs(blk - blk_ref)) <= 2e-4 * np.max(np.abs(blk_ref)), m


@pytest.fixture(scope="module")
def qm9_projected():
    """Projected representations x = rho U_e (FP64 oracle, rounded to FP32) of
    300 QM9-shaped molecules; U from the oracle's per-element PCA."""
    mols = synth.qm9_like(synth.rng_for(1, 12), 300)
    po = o_fchl19.params("E", n2=24, n3=22)
    reps = o_fchl19.representation_batch(mols.coords, mols.elem, mols.mol_ptr, po)
    U = o_reg.pca_bases(reps, mols.elem, 5, D)
    x = o_reg.project(reps, mols.elem, U).astype(np.float32)
    return mols, x


def test_sorf_segment_sum_on_projected_qm9_inputs(q, qm9_projected):
    mols, x = qm9_projected
    rng = np.random.default_rng(8)
    signs, b = synth.sorf_draw(rng, NF, D, T)
    b = b.astype(np.float32)
    W = o_sorf.sorf_matrix(signs, SIGMA)
    # the phases these inputs produce stay far inside the exactly reduced range
    umax = (math.sqrt(D) / SIGMA) * np.linalg.norm(x.astype(np.float64), axis=1).max() + 2 * math.pi
    assert umax < 2 ** 17 * math.pi / 100, umax
    Z = q.sorf(x, mols.mol_ptr, q.pack_signs(signs), T, b, SIGMA, q.SORF_PER_MOL).cpu().numpy()
    assert q.device_status() == 0
    xd = x.astype(np.float64)
    zd = o_sorf.features(xd, W, b.astype(np.float64))
    Zref = np.add.reduceat(zd, mols.mol_ptr[:-1], axis=0)
    tol = 2e-5 * math.sqrt(2.0 / NF) * mols.sizes()[:, None]
    assert np.all(np.abs(Z - Zref) <= tol), np.max(np.abs(Z - Zref) / tol)


def test_sorf_range_check_records_a_device_error(q, qm9_projected):
    """An atom whose phases would leave the exactly reduced range is reported
    (device error 6); in-range atoms are not."""
    mols, x = qm9_projected
    rng = np.random.default_rng(8)
    signs, b = synth.sorf_draw(rng, 1024, D, T)
    bits = q.pack_signs(signs)
    b = b.astype(np.float32)
    q.sorf(x, mols.mol_ptr, bits, T, b, SIGMA, q.SORF_PER_MOL)
    assert q.device_status() == 0
    bad = x.copy()
    lim = (2 ** 17 - 4) * math.pi * SIGMA / math.sqrt(D)       # largest |x|_2 accepted
    bad[7] *= np.float32(1.01 * lim / np.linalg.norm(x[7].astype(np.float64)))
    q.sorf(bad, mols.mol_ptr, bits, T, b, SIGMA, q.SORF_PER_MOL)
    assert q.device_status() == 6
    bad[7] = np.nan
    q.sorf(bad, mols.mol_ptr, bits, T, b, SIGMA, q.SORF_ENERGY, alpha=np.ones(1024, np.float32))
    assert q.device_status() == 6
    assert q.device_status() == 0          # reading the status clears it
