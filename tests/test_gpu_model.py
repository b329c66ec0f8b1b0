"""GPU parity of the setup and end-to-end paths through the C ABI against the
FP64 oracle: the PCA basis, energy + force prediction with a model handle,
and energy-only training (trained-model MAE within 1 % of the oracle's)."""
import math

import numpy as np
import pytest
import torch

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


def test_pca_fit_matches_oracle(q):
    mols = synth.qm9_like(synth.rng_for(1, 3), 300)
    p = o_fchl19.params("E", n2=24, n3=22)
    reps = o_fchl19.representation_batch(mols.coords, mols.elem, mols.mol_ptr, p).astype(np.float32)
    repd = np.zeros((mols.n_atoms, 780), np.float32)
    repd[:] = reps
    perm, offs = q.group_by_element(mols.elem, 5)
    d, cap = 64, 2000
    U = q.pca_fit(repd, 780, perm, offs, 5, d, cap).cpu().numpy()
    assert q.device_status() == 0
    for e in range(5):
        idx = np.nonzero(mols.elem == e)[0][:cap]
        if len(idx) == 0:
            assert np.all(U[e] == 0)
            continue
        Ur = o_reg.pca_basis(reps[idx].astype(np.float64), d)
        kept = np.nonzero(np.any(Ur != 0, axis=0))[0]
        # kept columns are orthonormal
        G = U[e][:, kept].T.astype(np.float64) @ U[e][:, kept]
        assert np.max(np.abs(G - np.eye(len(kept)))) < 1e-5
        # leading, well-separated directions agree column by column (same sign rule)
        w = np.linalg.eigvalsh(reps[idx].astype(np.float64).T @ reps[idx])[::-1]
        for c in range(min(8, len(kept))):
            gap = min(abs(w[c] - w[c + 1]), abs(w[c] - w[c - 1]) if c else np.inf) / w[0]
            if gap > 1e-3:
                assert np.max(np.abs(U[e][:, c] - Ur[:, c])) < 1e-4, (e, c)
        # the span of the kept columns captures the oracle's leading subspace
        P = U[e][:, kept].astype(np.float64)
        top = Ur[:, kept[: max(1, len(kept) // 2)]]
        overlap = np.linalg.norm(P.T @ top) ** 2 / top.shape[1]
        assert overlap > 0.999, (e, overlap)


@pytest.fixture(scope="module")
def ef_model(q):
    """A random-weight model on a mixed-size set (E+F parameters, N_F = 1024)."""
    a = synth.workload(0, scale=0.125).mols
    b = synth.serving_molecules(synth.rng_for(4, 11), 5, lo=5, hi=60)
    mols = synth.concat([a.molecule(i) for i in range(a.n_mol)] + [b.molecule(i) for i in range(b.n_mol)])
    po = o_fchl19.params("EF", n2=24, n3=22)
    reps = o_fchl19.representation_batch(mols.coords, mols.elem, mols.mol_ptr, po)
    U = o_reg.pca_bases(reps, mols.elem, 5, 128).astype(np.float32)
    rng = np.random.default_rng(3)
    signs, bb = synth.sorf_draw(rng, 1024, 128, 3)
    alpha = (rng.normal(size=1024) * 0.02).astype(np.float32)
    om = o_model.sorf_model(po, U.astype(np.float64), signs, bb.astype(np.float32).astype(np.float64), 2.0,
                            alpha.astype(np.float64))
    E_ref, F_ref = o_model.energies_forces(mols.coords, mols.elem, mols.mol_ptr, om)
    return mols, U, signs, bb.astype(np.float32), alpha, E_ref, F_ref


def test_predict_ef_matches_oracle(q, ef_model):
    mols, U, signs, bb, alpha, E_ref, F_ref = ef_model
    m = q.Model(gpu_params("EF"), int(mols.sizes().max()), U, signs, 3, bb, 2.0, alpha)
    E, F = m.predict(mols.coords, mols.elem, mols.mol_ptr)
    E, F = E.cpu().numpy(), F.cpu().numpy()
    assert q.device_status() == 0
    n = mols.sizes()
    assert np.all(np.abs(E - E_ref) <= 1e-4 * n), np.max(np.abs(E - E_ref) / n)
    assert np.max(np.abs(F - F_ref)) <= 1e-3, np.max(np.abs(F - F_ref))
    # energies only
    E2, _ = m.predict(mols.coords, mols.elem, mols.mol_ptr, forces=False)
    assert np.all(np.abs(E2.cpu().numpy() - E_ref) <= 1e-4 * n)
    m.close()


def test_predict_forces_are_conservative(q, ef_model):
    """Net force and torque vanish per molecule (translation/rotation invariance)."""
    mols, U, signs, bb, alpha, _, _ = ef_model
    m = q.Model(gpu_params("EF"), int(mols.sizes().max()), U, signs, 3, bb, 2.0, alpha)
    _, F = m.predict(mols.coords, mols.elem, mols.mol_ptr)
    F = F.cpu().numpy().astype(np.float64)
    for k in range(mols.n_mol):
        a, b = int(mols.mol_ptr[k]), int(mols.mol_ptr[k + 1])
        scale = np.abs(F[a:b]).max() + 1e-30
        assert np.max(np.abs(F[a:b].sum(0))) <= 1e-4 * scale * (b - a)
        c = mols.coords[a:b] - mols.coords[a:b].mean(0)
        assert np.max(np.abs(np.cross(c, F[a:b]).sum(0))) <= 1e-3 * scale * (b - a)
    m.close()


def test_energy_training_matches_oracle_mae(q):
    """Parity workload (64 x 9, N_F = 512, sigma = 2, lambda = 1e-6): the GPU-trained
    model's MAE on held-out molecules is within 1 % of the oracle-trained model's
    (same U for both, taken from the oracle fit)."""
    from paper_2206_01580_gb300 import pipeline
    w = synth.workload(0)
    test_mols = synth.random_box(synth.rng_for(0, 99), 32, 9)
    E_test = synth.targets(w.potential, test_mols)
    po = o_fchl19.params("E", n2=24, n3=22)
    reps = o_fchl19.representation_batch(w.mols.coords, w.mols.elem, w.mols.mol_ptr, po)
    U = o_reg.pca_bases(reps, w.mols.elem, 5, w.d)
    om = o_model.sorf_model(po, U, w.signs, w.b, w.sigma)
    alpha_o, _ = o_model.train(w.mols.coords, w.mols.elem, w.mols.mol_ptr, w.energies, om, w.lam, refine=2)
    om.alpha = alpha_o
    mae_o = np.mean(np.abs(o_model.energies_forces(test_mols.coords, test_mols.elem, test_mols.mol_ptr, om,
                                                   forces=False) - E_test))
    spec = pipeline.spec_from(gpu_params("E"), w.d, w.signs, w.b, w.sigma)
    batch = pipeline.Batch.from_host(w.mols.coords, w.mols.elem, w.mols.mol_ptr)
    alpha, _, it, rel = pipeline.train_energy(batch, w.energies, spec, w.lam,
                                              U=torch.as_tensor(U.astype(np.float32)).cuda(),
                                              max_iter=300, tol=1e-10)
    assert rel <= 1e-10, (it, rel)
    om.alpha = alpha.cpu().numpy()
    mae_g = np.mean(np.abs(o_model.energies_forces(test_mols.coords, test_mols.elem, test_mols.mol_ptr, om,
                                                   forces=False) - E_test))
    assert abs(mae_g - mae_o) <= 0.01 * mae_o, (mae_g, mae_o)


def test_split_prediction_matches_one_call():
    """qmlr_predict_features + qmlr_predict_ef_from_features give the results
    of qmlr_predict_ef bitwise, also with the first half on another stream."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_01580_gb300 import qmlr
    from paper_2206_01580_gb300.params import from_table
    mols = synth.serving_molecules(synth.rng_for(4, 33), 30, lo=5, hi=60)
    rng = np.random.default_rng(3)
    p = from_table("EF", n2=24, n3=22)
    U = (rng.normal(size=(5, 780, 64)) * 0.05).astype(np.float32)
    signs, b = synth.sorf_draw(rng, 1024, 64, 3)
    alpha = (rng.normal(size=1024) * 0.02).astype(np.float32)
    model = qmlr.Model(p, 60, U, signs, 3, b.astype(np.float32), 2.0, alpha)
    E1, F1 = model.predict(mols.coords, mols.elem, mols.mol_ptr)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        model.predict_features(mols.coords, mols.elem, mols.mol_ptr)
    torch.cuda.current_stream().wait_stream(side)
    E2, F2 = model.predict_from_features(mols.coords, mols.elem, mols.mol_ptr)
    torch.cuda.synchronize()
    assert torch.equal(E1, E2) and torch.equal(F1, F2)
    model.close()
