"""GPU parity of periodic FCHL19 (the paper's periodic MOF and water systems)
through the C ABI against the FP64 oracle: representation rows over lattice
images (a skewed cell shorter than the cutoff, a water-shaped box and a
framework-shaped crystal), and energies and forces of the periodic atomic
energy partition (periodic FCHL19 -> projection -> SORF -> adjoint).

Tolerances: representation rel <= 1e-5 per row; energy <= 1e-4 eV per atom;
forces <= 1e-3 eV/A; the forces of the cell sum to zero."""
import math

import numpy as np
import pytest
import torch

from oracle import fchl19 as o_fchl19
from oracle import model as o_model
from oracle import regression as o_reg
from paper_2206_01580_gb300 import synth

pytestmark = pytest.mark.gpu

H, C, N, O = 0, 1, 2, 3
CELL = np.array([[3.3, 0.0, 0.0], [0.8, 3.6, 0.0], [0.3, -0.5, 3.9]])
X3 = np.array([[0.2, 0.1, 0.3], [1.4, 0.9, 0.2], [0.7, 2.0, 1.8]])
E3 = np.array([C, O, H], np.int32)


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


def systems():
    w = synth.water_box(synth.rng_for(5, 1), 8)                    # 24 atoms, 6.2 A cube
    m = synth.framework_crystal(synth.rng_for(5, 2), 40)           # 40 atoms, ~8 A cell
    return [("skewed-3", X3.astype(np.float32).astype(np.float64), E3, CELL),
            ("water-8", w.coords.astype(np.float32).astype(np.float64), w.elem, w.cell),
            ("framework-40", m.coords.astype(np.float32).astype(np.float64), m.elem, m.cell)]


@pytest.mark.parametrize("column", ["E", "EF"])
def test_periodic_representation_matches_oracle(q, column):
    po = o_fchl19.params(column, n2=24, n3=22)
    for name, x, el, cell in systems():
        ref = o_fchl19.representation_periodic(torch.as_tensor(x), el, cell, po).numpy()
        sysg = q.PeriodicSystem(x, el, cell, po.rcut)
        rep = q.fchl19_periodic(sysg, gpu_params(column)).cpu().numpy()
        assert q.device_status() == 0
        assert np.all(rep[:, 780:] == 0)
        for i in range(len(el)):
            rel = np.max(np.abs(rep[i, :780] - ref[i])) / np.max(np.abs(ref[i]))
            assert rel <= 1e-5, (name, i, rel)


def test_periodic_energy_and_forces_match_oracle(q):
    from paper_2206_01580_gb300 import pipeline
    po = o_fchl19.params("EF", n2=24, n3=22)
    rng = np.random.default_rng(11)
    for name, x, el, cell in systems():
        reps = o_fchl19.representation_periodic(torch.as_tensor(x), el, cell, po).numpy()
        U = o_reg.pca_bases(reps, el, 5, 64).astype(np.float32)
        signs, b = synth.sorf_draw(rng, 1024, 64, 3)
        b = b.astype(np.float32)
        alpha = (rng.normal(size=1024) * 0.5).astype(np.float32)
        om = o_model.sorf_model(po, U.astype(np.float64), signs, b.astype(np.float64), 2.0, alpha.astype(np.float64))
        E_ref, F_ref = o_model.periodic_energy_forces(x, el, cell, om)
        spec = pipeline.spec_from(gpu_params("EF"), 64, signs, b, 2.0)
        sysg = q.PeriodicSystem(x, el, cell, po.rcut)
        E, F = pipeline.predict_periodic(sysg, spec, torch.as_tensor(U).cuda(), torch.as_tensor(alpha).cuda())
        E, F = float(E.cpu()[0]), F.cpu().numpy()
        assert q.device_status() == 0
        assert abs(E - E_ref) <= 1e-4 * len(el), (name, E, E_ref)
        assert np.max(np.abs(F - F_ref)) <= 1e-3, (name, np.max(np.abs(F - F_ref)))
        assert np.max(np.abs(F.astype(np.float64).sum(0))) <= 1e-4 * max(1.0, np.abs(F).max()) * len(el)


def test_periodic_environment_larger_than_sized_is_reported(q):
    """An atom with more environment entries than max_env is recorded as device
    error 1 and its row is zero; the others are computed."""
    po = o_fchl19.params("E", n2=24, n3=22)
    sysg = q.PeriodicSystem(X3, E3, CELL, po.rcut)
    full = q.fchl19_periodic(sysg, gpu_params("E")).cpu().numpy()
    assert q.device_status() == 0
    n_env = np.diff(sysg.env_ptr.cpu().numpy())
    sysg.max_env = int(n_env.max()) - 1      # the largest environments no longer fit
    rep = q.fchl19_periodic(sysg, gpu_params("E")).cpu().numpy()
    assert q.device_status() == 1
    for i in range(3):
        if n_env[i] > sysg.max_env:
            assert np.all(rep[i] == 0)
        else:
            assert np.array_equal(rep[i], full[i])
