"""Energies as a differentiable function of the coordinates (the
FCHL19SORFEnergy autograd.Function over the C ABI): the gradient torch.autograd
returns is the hand-written adjoint's, and it matches both the FP64 oracle's
forces and central differences of the GPU energies.

Tolerances: forces <= 1e-3 eV/A against the oracle (the stated force bound).
The central differences use h = 2^-13 A (about 1e-4 A) and divide by the
step the FP32 coordinates actually took; the energies they difference are
FP32 sums of N_F terms, whose rounding (about 1e-6 eV on these molecules)
limits the difference quotient to about 1e-2 eV/A, so that comparison is
relative to the largest force of the set."""
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


@pytest.fixture(scope="module")
def setup(q):
    from paper_2206_01580_gb300.params import from_table
    a = synth.workload(2, scale=0.003).mols                              # 21-atom conformations
    b = synth.serving_molecules(synth.rng_for(4, 21), 3, lo=5, hi=40)
    mols = synth.concat([m.molecule(i) for m in (a, b) for i in range(m.n_mol)])
    po = o_fchl19.params("EF", n2=24, n3=22)
    reps = o_fchl19.representation_batch(mols.coords, mols.elem, mols.mol_ptr, po)
    U = o_reg.pca_bases(reps, mols.elem, 5, 128).astype(np.float32)
    rng = np.random.default_rng(17)
    signs, bb = synth.sorf_draw(rng, 4096, 128, 3)
    bb = bb.astype(np.float32)
    alpha = (rng.normal(size=4096) * 0.5).astype(np.float32)
    om = o_model.sorf_model(po, U.astype(np.float64), signs, bb.astype(np.float64), 2.0, alpha.astype(np.float64))
    E_ref, F_ref = o_model.energies_forces(mols.coords, mols.elem, mols.mol_ptr, om)
    model = q.Model(from_table("EF", n2=24, n3=22), int(mols.sizes().max()), U, signs, 3, bb, 2.0, alpha)
    yield mols, model, E_ref, F_ref
    model.close()


def test_autograd_gradient_is_minus_the_oracle_forces(q, setup):
    mols, model, E_ref, F_ref = setup
    R = torch.tensor(mols.coords, dtype=torch.float32, device="cuda", requires_grad=True)
    E = q.FCHL19SORFEnergy.apply(R, model, mols.elem, mols.mol_ptr)
    assert E.dtype == torch.float64 and E.requires_grad
    (g,) = torch.autograd.grad(E.sum(), R)
    assert q.device_status() == 0
    n = mols.sizes()
    assert np.all(np.abs(E.detach().cpu().numpy() - E_ref) <= 1e-4 * n)
    assert np.max(np.abs(-g.cpu().numpy() - F_ref)) <= 1e-3, np.max(np.abs(-g.cpu().numpy() - F_ref))


def test_autograd_weights_each_molecule_by_its_upstream_gradient(q, setup):
    """L = sum_m w_m E_m: dL/dr_k = -w_{mol(k)} F_k."""
    mols, model, _, F_ref = setup
    R = torch.tensor(mols.coords, dtype=torch.float32, device="cuda", requires_grad=True)
    E = q.energy(R, model, mols.elem, mols.mol_ptr)
    w = torch.linspace(-2.0, 3.0, mols.n_mol, dtype=torch.float64, device="cuda")
    (g,) = torch.autograd.grad((w * E).sum(), R)
    wa = np.repeat(w.cpu().numpy(), mols.sizes())[:, None]
    assert np.max(np.abs(g.cpu().numpy() - (-wa * F_ref))) <= 1e-3 * max(1.0, np.abs(wa).max())


def test_autograd_gradient_matches_central_differences(q, setup):
    mols, model, _, _ = setup
    R = torch.tensor(mols.coords, dtype=torch.float32, device="cuda", requires_grad=True)
    E = q.energy(R, model, mols.elem, mols.mol_ptr)
    (g,) = torch.autograd.grad(E.sum(), R)
    g = g.cpu().numpy().astype(np.float64)
    h = 2.0 ** -13
    rng = np.random.default_rng(5)
    picks = rng.choice(mols.n_atoms, size=min(12, mols.n_atoms), replace=False)
    fd = np.zeros((len(picks), 3))
    x0 = mols.coords.astype(np.float32)
    with torch.no_grad():
        for r, k in enumerate(picks):
            for ax in range(3):
                xp, xm = x0.copy(), x0.copy()
                xp[k, ax] += np.float32(h)
                xm[k, ax] -= np.float32(h)
                step = float(xp[k, ax]) - float(xm[k, ax])             # the FP32 step actually taken
                Ep = q.energy(torch.as_tensor(xp).cuda(), model, mols.elem, mols.mol_ptr).sum().item()
                Em = q.energy(torch.as_tensor(xm).cuda(), model, mols.elem, mols.mol_ptr).sum().item()
                fd[r, ax] = (Ep - Em) / step
    scale = np.abs(g).max()
    assert np.max(np.abs(fd - g[picks])) <= 2e-2 * scale, (np.max(np.abs(fd - g[picks])), scale)


def test_no_gradient_requested_computes_energies_only(q, setup):
    mols, model, E_ref, _ = setup
    R = torch.tensor(mols.coords, dtype=torch.float32, device="cuda")
    E = q.energy(R, model, mols.elem, mols.mol_ptr)
    assert not E.requires_grad
    assert np.all(np.abs(E.cpu().numpy() - E_ref) <= 1e-4 * mols.sizes())
