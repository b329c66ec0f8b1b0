"""Continuous-batching server through the C ABI: every molecule's energy and
forces are the same (bitwise) when it is served alone and when it is served in
a mixed stream with other molecules; they match the FP64 oracle within the
energy/force tolerances; admission, size limits and bounded waits behave."""
import time

import numpy as np
import pytest
import torch

from oracle import fchl19 as o_fchl19
from oracle import model as o_model
from oracle import regression as o_reg
from paper_2206_01580_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_01580_gb300 import qmlr
    from paper_2206_01580_gb300.params import from_table
    mols = synth.serving_molecules(synth.rng_for(4, 21), 40, lo=5, hi=200)
    po = o_fchl19.params("EF", n2=24, n3=22)
    fit = mols.subset(range(8))
    reps = o_fchl19.representation_batch(fit.coords, fit.elem, fit.mol_ptr, po)
    U = o_reg.pca_bases(reps, fit.elem, 5, 128).astype(np.float32)
    rng = np.random.default_rng(31)
    signs, b = synth.sorf_draw(rng, 2048, 128, 3)
    b = b.astype(np.float32)
    alpha = (rng.normal(size=2048) * 0.02).astype(np.float32)
    model = qmlr.Model(from_table("EF", n2=24, n3=22), 200, U, signs, 3, b, 2.0, alpha)
    return qmlr, model, mols, (po, U, signs, b, alpha)


def _serve_all(srv, mols, alone: bool):
    out = {}
    if alone:
        for m in range(mols.n_mol):
            c, e = mols.molecule(m)
            t = srv.submit(c, e)
            rc, E, F = srv.poll(t, len(e))
            assert rc == 0
            out[m] = (E, F)
    else:
        tickets = []
        for m in range(mols.n_mol):
            c, e = mols.molecule(m)
            tickets.append((m, srv.submit(c, e), len(e)))
        for m, t, n in tickets:
            rc, E, F = srv.poll(t, n)
            assert rc == 0
            out[m] = (E, F)
    return out


@pytest.mark.parametrize("use_graphs", [True, False])
def test_result_is_the_same_alone_and_in_the_mix(setup, use_graphs):
    qmlr, model, mols, _ = setup
    srv = qmlr.Server(model, n_lanes=2, max_batch_atoms=2048, max_batch_mols=512, use_graphs=use_graphs)
    alone = _serve_all(srv, mols, alone=True)
    mixed = _serve_all(srv, mols, alone=False)
    mixed2 = _serve_all(srv, mols, alone=False)   # graphs replayed
    for m in range(mols.n_mol):
        assert alone[m][0] == mixed[m][0] == mixed2[m][0], m
        assert np.array_equal(alone[m][1], mixed[m][1]) and np.array_equal(alone[m][1], mixed2[m][1]), m
    st = srv.stats()
    assert st["completed"] == 3 * mols.n_mol and st["batches"] < 3 * mols.n_mol
    # the direct batched prediction agrees as well
    E, F = model.predict(mols.coords, mols.elem, mols.mol_ptr)
    E, F = E.cpu().numpy(), F.cpu().numpy()
    for m in range(mols.n_mol):
        a, b = int(mols.mol_ptr[m]), int(mols.mol_ptr[m + 1])
        assert E[m] == alone[m][0]
        assert np.array_equal(F[a:b], alone[m][1])
    srv.close()


def test_served_results_match_oracle(setup):
    qmlr, model, mols, (po, U, signs, b, alpha) = setup
    srv = qmlr.Server(model, n_lanes=2, max_batch_atoms=2048, max_batch_mols=512)
    sub = mols.subset([0, 1, 2, 3])
    om = o_model.sorf_model(po, U.astype(np.float64), signs, b.astype(np.float64), 2.0, alpha.astype(np.float64))
    E_ref, F_ref = o_model.energies_forces(sub.coords, sub.elem, sub.mol_ptr, om)
    got = _serve_all(srv, sub, alone=False)
    for m in range(sub.n_mol):
        n = int(sub.mol_ptr[m + 1] - sub.mol_ptr[m])
        a = int(sub.mol_ptr[m])
        assert abs(got[m][0] - E_ref[m]) <= 1e-4 * n
        assert np.max(np.abs(got[m][1] - F_ref[a:a + n])) <= 1e-3
    srv.close()


def test_admission_limits_and_bounded_waits(setup):
    qmlr, model, mols, _ = setup
    srv = qmlr.Server(model, n_lanes=1, max_batch_atoms=256, max_batch_mols=128, max_slots=4,
                      use_graphs=False)
    c, e = mols.molecule(0)
    tickets = [srv.submit(c, e) for _ in range(4)]
    rc, _ = srv.try_submit(c, e)
    assert rc == qmlr.EBUSY
    for t in tickets:
        assert srv.poll(t, len(e))[0] == 0
    assert srv.try_submit(c, e)[0] == 0
    # a molecule larger than the model allows is refused before queuing
    big = np.zeros((201, 3), np.float32)
    assert srv.try_submit(big, np.zeros(201, np.int32))[0] == qmlr.EINVAL
    srv.close()
    # a bounded poll runs out while work is still queued, and the ticket stays valid
    srv = qmlr.Server(model, n_lanes=1, max_batch_atoms=256, max_batch_mols=128, use_graphs=False)
    bigm = [m for m in range(mols.n_mol) if mols.sizes()[m] > 150][:1]
    cb, eb = mols.molecule(bigm[0])
    ts = [srv.submit(cb, eb) for _ in range(40)]
    rc, _, _ = srv.poll(ts[-1], len(eb), timeout_us=0)
    assert rc == qmlr.ETIMEOUT
    for t in ts:
        assert srv.poll(t, len(eb))[0] == 0
    with pytest.raises(Exception):
        srv.submit(np.zeros((0, 3), np.float32), np.zeros(0, np.int32))
    srv.close()


def test_trace_replay_completes_every_admitted_request(setup):
    qmlr, model, mols, _ = setup
    srv = qmlr.Server(model, n_lanes=2, max_batch_atoms=2048, max_batch_mols=512)
    rng = np.random.default_rng(5)
    arrivals = synth.poisson_arrivals(rng, 2000.0, 0.2)
    picks = rng.integers(0, mols.n_mol, size=len(arrivals))
    st = srv.replay(mols.coords, mols.elem, mols.mol_ptr, arrivals, picks)
    assert st["completed"] + st["rejected"] == len(arrivals)
    assert st["completed"] > 0 and 0 < st["p50_us"] <= st["p99_us"]
    srv.close()
