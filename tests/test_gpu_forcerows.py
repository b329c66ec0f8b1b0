"""GPU parity of the energy+force training rows through the C ABI against the
FP64 oracle: FCHL19 Jacobian rows (forward mode), the force rows -dZ/dr, and
energy+force training (trained-model MAE within 1 % of the oracle's).

Tolerances: Jacobian and force rows max error <= 2e-4 of the largest entry of
the molecule's block (FP32 forward-mode chain through exp/log/pow)."""
import numpy as np
import pytest
import torch
from torch.func import jacfwd

from oracle import fchl19 as o_fchl19
from oracle import model as o_model
from oracle import regression as o_reg
from paper_2206_01580_gb300 import synth

pytestmark = pytest.mark.gpu


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


def small_mixed():
    a = synth.workload(2, scale=0.003).mols          # 3 aspirin-like conformations (21 atoms)
    b = synth.random_box(synth.rng_for(0, 5), 3, 9)  # 9-atom boxes (some pairs beyond the cutoff? no: 4 A box)
    c = synth.serving_molecules(synth.rng_for(4, 5), 2, lo=30, hi=45)   # larger: pairs beyond r_cut
    return synth.concat([m.molecule(i) for m in (a, b, c) for i in range(m.n_mol)])


def test_jacobian_rows_match_oracle(q):
    mols = small_mixed()
    p = o_fchl19.params("EF", n2=24, n3=22)
    jac_ptr, J, _ = q.fchl19_jacobian(mols.coords, mols.elem, mols.mol_ptr, int(mols.sizes().max()),
                                      gpu_params("EF"))
    J = J.cpu().numpy()
    ptr = jac_ptr.cpu().numpy()
    assert q.device_status() == 0
    for m in range(mols.n_mol):
        a, b = int(mols.mol_ptr[m]), int(mols.mol_ptr[m + 1])
        M = b - a
        x = mols.coords[a:b]
        R = torch.as_tensor(x, dtype=torch.float64)
        jref = jacfwd(lambda r: o_fchl19.representation(r, mols.elem[a:b], p, x))(R).numpy()  # [M,780,M,3]
        got = J[ptr[m]:ptr[m + 1], :780].reshape(M, M, 3, 780)                              # [I,k,x,bin]
        want = np.transpose(jref, (0, 2, 3, 1))
        scale = np.max(np.abs(want))
        assert np.max(np.abs(got - want)) <= 2e-4 * scale, m


def test_force_rows_match_oracle(q):
    from paper_2206_01580_gb300 import pipeline
    mols = small_mixed()
    po = o_fchl19.params("EF", n2=24, n3=22)
    reps = o_fchl19.representation_batch(mols.coords, mols.elem, mols.mol_ptr, po)
    U = o_reg.pca_bases(reps, mols.elem, 5, 128)
    rng = np.random.default_rng(4)
    signs, b = synth.sorf_draw(rng, 1024, 128, 3)
    bf = b.astype(np.float32)
    om = o_model.sorf_model(po, U.astype(np.float32).astype(np.float64), signs, bf.astype(np.float64), 2.0)
    ref = o_model.force_rows(mols.coords, mols.elem, mols.mol_ptr, om)
    Zref = o_model.feature_matrix(mols.coords, mols.elem, mols.mol_ptr, om)
    spec = pipeline.spec_from(gpu_params("EF"), 128, signs, bf, 2.0)
    batch = pipeline.Batch.from_host(mols.coords, mols.elem, mols.mol_ptr)
    rows = pipeline.energy_force_rows(batch, spec, torch.as_tensor(U.astype(np.float32)).cuda()).cpu().numpy()
    assert q.device_status() == 0
    nm = mols.n_mol
    np.testing.assert_allclose(rows[:nm], Zref, atol=2e-5 * np.max(np.abs(Zref)))
    for m in range(nm):
        a, bb = int(mols.mol_ptr[m]), int(mols.mol_ptr[m + 1])
        blk_ref = ref[3 * a:3 * bb]
        blk = rows[nm + 3 * a:nm + 3 * bb]
        assert np.max(np.abs(blk - blk_ref)) <= 2e-4 * np.max(np.abs(blk_ref)), m


def test_energy_force_training_matches_oracle_mae(q):
    """MD17-shaped sample (12 train / 12 held-out conformations of a 21-atom
    molecule, N_F = 1024, E+F parameters, lambda = 1e-6): the GPU-trained model's
    energy and force MAE on held-out conformations are within 1 % of the
    oracle-trained model's (same U for both, from the oracle fit)."""
    from paper_2206_01580_gb300 import pipeline
    w = synth.workload(2, scale=0.024)          # 24 conformations
    tr, te = w.mols.subset(range(12)), w.mols.subset(range(12, 24))
    na = tr.n_atoms
    E_tr, F_tr = w.energies[:12], w.forces[:na]
    E_te, F_te = w.energies[12:24], w.forces[na:2 * na]
    po = o_fchl19.params("EF", n2=24, n3=22)
    reps = o_fchl19.representation_batch(tr.coords, tr.elem, tr.mol_ptr, po)
    U = o_reg.pca_bases(reps, tr.elem, 5, 128).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(9)
    signs, b = synth.sorf_draw(rng, 1024, 128, 3)
    bf = b.astype(np.float32).astype(np.float64)
    om = o_model.sorf_model(po, U, signs, bf, 2.0)
    alpha_o, _ = o_model.train(tr.coords, tr.elem, tr.mol_ptr, E_tr, om, 1e-6, forces=F_tr, refine=2)
    om.alpha = alpha_o
    Eo, Fo = o_model.energies_forces(te.coords, te.elem, te.mol_ptr, om)
    spec = pipeline.spec_from(gpu_params("EF"), 128, signs, bf, 2.0)
    batch = pipeline.Batch.from_host(tr.coords, tr.elem, tr.mol_ptr)
    alpha, _, it, rel = pipeline.train_energy_force(batch, E_tr, F_tr, spec, 1e-6,
                                                    U=torch.as_tensor(U.astype(np.float32)).cuda(),
                                                    max_iter=300, tol=1e-10)
    assert rel <= 1e-10, (it, rel)
    om.alpha = alpha.cpu().numpy()
    Eg, Fg = o_model.energies_forces(te.coords, te.elem, te.mol_ptr, om)
    mae_e_o, mae_e_g = np.mean(np.abs(Eo - E_te)), np.mean(np.abs(Eg - E_te))
    mae_f_o, mae_f_g = np.mean(np.abs(Fo - F_te)), np.mean(np.abs(Fg - F_te))
    assert abs(mae_e_g - mae_e_o) <= 0.01 * mae_e_o, (mae_e_g, mae_e_o)
    assert abs(mae_f_g - mae_f_o) <= 0.01 * mae_f_o, (mae_f_g, mae_f_o)
