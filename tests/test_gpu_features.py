"""GPU parity of the feature path through the C ABI against the FP64 oracle:
FCHL19 forward and VJP, element grouping, projection and its transpose, SORF
per-atom features, per-molecule segment sums, energies and the SORF backward.

Tolerances (float32 kernels against the float64 oracle):
* representation, projection: rel <= 1e-5 per atom row (|delta|_inf / |ref|_inf)
* features: |delta z| <= 2e-5 * sqrt(2/N_F) (cos of an argument with ~1e-6 error)
* energies: <= 1e-4 eV per atom; gradients: rel <= 1e-4 per molecule
"""
import math

import numpy as np
import pytest
import torch

from oracle import fchl19 as o_fchl19
from oracle import regression as o_reg
from oracle import sorf as o_sorf
from paper_2206_01580_gb300 import synth

pytestmark = pytest.mark.gpu

REP_REL = 1e-5


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_01580_gb300 import qmlr
    qmlr.lib()
    return qmlr


def gpu_params(column="E"):
    from paper_2206_01580_gb300.params import from_table
    return from_table(column, n2=24, n3=22)


def oracle_params(column="E"):
    return o_fchl19.params(column, n2=24, n3=22)


def row_rel(got, ref):
    num = np.max(np.abs(got - ref), axis=1)
    den = np.maximum(np.max(np.abs(ref), axis=1), 1e-30)
    return num / den


def mixed_set():
    """Molecules of several shapes: box (9), QM9-like (3-29), serving-like (up to 120)."""
    a = synth.workload(0, scale=0.25).mols
    b = synth.qm9_like(synth.rng_for(1, 7), 12)
    c = synth.serving_molecules(synth.rng_for(4, 7), 6, lo=30, hi=120)
    return synth.concat([a.molecule(i) for i in range(a.n_mol)] + [b.molecule(i) for i in range(b.n_mol)]
                        + [c.molecule(i) for i in range(c.n_mol)])


@pytest.mark.parametrize("column", ["E", "EF"])
def test_fchl19_forward_matches_oracle(q, column):
    mols = mixed_set()
    ref = o_fchl19.representation_batch(mols.coords, mols.elem, mols.mol_ptr, oracle_params(column))
    got = q.fchl19(mols.coords, mols.elem, mols.mol_ptr, int(mols.sizes().max()),
                   gpu_params(column)).cpu().numpy()
    assert got.shape[1] == 780
    assert q.device_status() == 0
    nz = np.max(np.abs(ref), axis=1) > 0
    assert np.all(row_rel(got[nz, :780], ref[nz]) <= REP_REL)
    assert np.all(got[~nz] == 0)


def test_fchl19_padding_and_degenerate_molecules(q):
    # single atom, an empty molecule, a diatomic beyond the cutoff, a normal molecule
    coords = np.array([[0, 0, 0], [0, 0, 0], [7.0, 0, 0], [0, 0, 0], [1.1, 0, 0], [0, 1.0, 0]], float)
    elem = np.array([1, 0, 1, 2, 0, 3], np.int32)
    mol_ptr = np.array([0, 1, 1, 3, 6], np.int32)
    got = q.fchl19(coords, elem, mol_ptr, 8, gpu_params(), rep_ld=800).cpu().numpy()
    assert q.device_status() == 0
    assert np.all(got[:3] == 0)
    assert np.all(got[:, 780:] == 0)
    ref = o_fchl19.representation_batch(coords, elem, mol_ptr, oracle_params())
    assert np.all(row_rel(got[3:, :780], ref[3:]) <= REP_REL)


def test_fchl19_molecule_too_large_is_reported(q):
    mols = synth.workload(0, scale=0.1).mols
    got = q.fchl19(mols.coords, mols.elem, mols.mol_ptr, 4, gpu_params()).cpu().numpy()
    assert q.device_status() == 1
    assert np.all(got == 0)
    assert q.device_status() == 0


def test_fchl19_vjp_matches_oracle_autograd(q):
    mols = mixed_set()
    p = oracle_params("EF")
    rng = np.random.default_rng(0)
    g = rng.normal(size=(mols.n_atoms, 780))
    ref = np.zeros((mols.n_atoms, 3))
    for m in range(mols.n_mol):
        a, b = int(mols.mol_ptr[m]), int(mols.mol_ptr[m + 1])
        R = torch.tensor(mols.coords[a:b], dtype=torch.float64, requires_grad=True)
        (gr,) = torch.autograd.grad((o_fchl19.representation(R, mols.elem[a:b], p)
                                     * torch.as_tensor(g[a:b])).sum(), R)
        ref[a:b] = gr.numpy()
    gpad = np.zeros((mols.n_atoms, 780), np.float32)
    gpad[:] = g
    got = q.fchl19_vjp(mols.coords, mols.elem, mols.mol_ptr, int(mols.sizes().max()),
                       gpu_params("EF"), gpad).cpu().numpy()
    assert q.device_status() == 0
    got2 = q.fchl19_vjp_atoms(mols.coords, mols.elem, mols.mol_ptr, int(mols.sizes().max()),
                              gpu_params("EF"), gpad, scale=-1.0).cpu().numpy()
    assert q.device_status() == 0
    for m in range(mols.n_mol):
        a, b = int(mols.mol_ptr[m]), int(mols.mol_ptr[m + 1])
        scale = np.max(np.abs(ref[a:b]))
        assert np.max(np.abs(got[a:b] - ref[a:b])) <= 1e-4 * scale, m
        assert np.max(np.abs(-got2[a:b] - ref[a:b])) <= 1e-4 * scale, m


def test_group_by_element_is_stable_counting_sort(q):
    rng = np.random.default_rng(1)
    for n in (0, 1, 1000, 1024, 5000):
        elem = rng.integers(0, 5, size=n).astype(np.int32)
        perm, offs = q.group_by_element(elem, 5)
        want = np.argsort(elem, kind="stable")
        assert np.array_equal(perm.cpu().numpy(), want)
        assert np.array_equal(offs.cpu().numpy(), np.concatenate([[0], np.cumsum(np.bincount(elem, minlength=5))]))


@pytest.mark.parametrize("d", [64, 128])
def test_project_and_transpose_match_oracle(q, d):
    mols = mixed_set()
    rng = np.random.default_rng(2)
    reps = o_fchl19.representation_batch(mols.coords, mols.elem, mols.mol_ptr, oracle_params())
    U = rng.normal(size=(5, 780, d)) / math.sqrt(780)
    Uf = U.astype(np.float32)
    repf = np.zeros((mols.n_atoms, 780), np.float32)
    repf[:] = reps
    perm, offs = q.group_by_element(mols.elem, 5)
    x = q.project(repf, 780, perm, offs, 5, Uf).cpu().numpy()
    ref = o_reg.project(repf.astype(np.float64), mols.elem, Uf.astype(np.float64))
    assert np.all(row_rel(x, ref) <= REP_REL)
    gx = rng.normal(size=(2, mols.n_atoms, d)).astype(np.float32)
    gr = q.project_t(gx, perm, offs, 5, Uf, 780, rep_ld=784).cpu().numpy()
    gsum = gx.astype(np.float64).sum(0)
    want = np.stack([Uf[e].astype(np.float64) @ gsum[i] for i, e in enumerate(mols.elem)])
    assert np.all(row_rel(gr[:, :780], want) <= REP_REL)
    assert np.all(gr[:, 780:] == 0)


def _sorf_inputs(d, nf, T, n_mol=10, seed=3):
    rng = np.random.default_rng(seed)
    sizes = rng.integers(1, 12, size=n_mol)
    sizes[3] = 0
    mol_ptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    x = (rng.normal(size=(int(mol_ptr[-1]), d)) * 0.5).astype(np.float32)
    signs, b = synth.sorf_draw(rng, nf, d, T)
    return x, mol_ptr, signs, b.astype(np.float32)


SORF_CASES = [(16, 64, 1), (32, 256, 2), (64, 512, 3), (128, 1024, 3), (128, 16384, 3), (128, 32768, 2)]


@pytest.mark.parametrize("d,nf,T", SORF_CASES)
def test_sorf_per_atom_and_per_molecule_match_oracle(q, d, nf, T):
    x, mol_ptr, signs, b = _sorf_inputs(d, nf, T)
    sigma = 1.7
    W = o_sorf.sorf_matrix(signs, sigma)
    ref = o_sorf.features(x.astype(np.float64), W, b.astype(np.float64))
    bits = q.pack_signs(signs)
    pref = math.sqrt(2 / nf)
    z = q.sorf(x, mol_ptr, bits, T, b, sigma, q.SORF_PER_ATOM).cpu().numpy()
    assert np.max(np.abs(z - ref)) <= 2e-5 * pref
    Z = q.sorf(x, mol_ptr, bits, T, b, sigma, q.SORF_PER_MOL).cpu().numpy()
    Zref = o_reg.segment_sum(ref, mol_ptr)
    sizes = np.diff(mol_ptr)
    assert np.all(np.max(np.abs(Z - Zref), axis=1) <= 2e-5 * pref * np.maximum(sizes, 1))
    assert np.all(Z[sizes == 0] == 0)


RFF_CASES = [(16, 64), (64, 512), (128, 1000), (128, 4096), (200, 300), (256, 129)]


@pytest.mark.parametrize("d,nf", RFF_CASES)
def test_rff_per_atom_and_per_molecule_match_oracle(q, d, nf):
    """Dense RFF (W = G / sigma) against the FP64 oracle, including feature
    counts that end in a partial 128-feature tile and d that is not a power of
    two. Bound from the FP32 arithmetic: the dot product's rounding
    (d 2^-24 sum_k |G_fk x_k|, divided by sigma), one rounding of the scale and
    phase add (2^-24 |u|), cosf (a few ulp); the molecule sums add their own
    FP32 rounding."""
    rng = np.random.default_rng(41 + d)
    sizes = rng.integers(1, 12, size=9)
    sizes[2] = 0
    mol_ptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    x = (rng.normal(size=(int(mol_ptr[-1]), d)) * 0.5).astype(np.float32)
    G, b = synth.rff_draw(rng, nf, d)
    G, b = G.astype(np.float32), b.astype(np.float32)
    sigma = 1.7
    xd, Gd, bd = x.astype(np.float64), G.astype(np.float64), b.astype(np.float64)
    ref = o_sorf.features(xd, o_sorf.rff_matrix(Gd, sigma), bd)
    pref = math.sqrt(2 / nf)
    u = xd @ Gd.T / sigma + bd
    bound = pref * (d * 2.0 ** -24 * (np.abs(xd) @ np.abs(Gd).T) / sigma + 2.0 ** -23 * np.abs(u) + 1e-6)
    z = q.rff(x, mol_ptr, G, b, sigma, q.SORF_PER_ATOM).cpu().numpy()
    assert np.all(np.abs(z - ref) <= bound)
    Z = q.rff(x, mol_ptr, G, b, sigma, q.SORF_PER_MOL).cpu().numpy()
    Zref = o_reg.segment_sum(ref, mol_ptr)
    Zbound = o_reg.segment_sum(bound, mol_ptr) + pref * 2.0 ** -22 * sizes[:, None] ** 2
    assert np.all(np.abs(Z - Zref) <= Zbound)
    assert np.all(Z[sizes == 0] == 0)
    # deterministic
    assert np.array_equal(Z, q.rff(x, mol_ptr, G, b, sigma, q.SORF_PER_MOL).cpu().numpy())


@pytest.mark.parametrize("d,nf,T", SORF_CASES)
def test_sorf_energy_and_gradient_match_oracle(q, d, nf, T):
    x, mol_ptr, signs, b = _sorf_inputs(d, nf, T, seed=4)
    sigma = 1.3
    rng = np.random.default_rng(5)
    alpha = (rng.normal(size=nf) * 0.05).astype(np.float32)
    W = o_sorf.sorf_matrix(signs, sigma)
    xt = torch.tensor(x.astype(np.float64), requires_grad=True)
    zt = o_sorf.features(xt, W, b.astype(np.float64))
    e_atom = zt @ torch.as_tensor(alpha.astype(np.float64))
    (gref,) = torch.autograd.grad(e_atom.sum(), xt)
    Eref = np.add.reduceat(np.append(e_atom.detach().numpy(), 0.0), mol_ptr[:-1])
    sizes = np.diff(mol_ptr)
    Eref[sizes == 0] = 0.0
    bits = q.pack_signs(signs)
    E = q.sorf(x, mol_ptr, bits, T, b, sigma, q.SORF_ENERGY, alpha=alpha).cpu().numpy()
    assert np.all(np.abs(E - Eref) <= 1e-4 * np.maximum(sizes, 1))
    E2, gx = q.sorf_grad(x, mol_ptr, bits, T, b, sigma, alpha)
    E2, gx = E2.cpu().numpy(), gx.cpu().numpy().sum(0)
    assert np.all(np.abs(E2 - Eref) <= 1e-4 * np.maximum(sizes, 1))
    scale = np.max(np.abs(gref.numpy()))
    assert np.max(np.abs(gx - gref.numpy())) <= 1e-4 * scale


SORF_TC_CASES = [(128, 1, 10), (384, 3, 60), (1024, 2, 60), (16384, 3, 60), (32768, 2, 10), (512, 3, 2000)]


@pytest.mark.parametrize("nf,T,n_mol", SORF_TC_CASES)
def test_sorf_tensor_core_energy_and_gradient_match_oracle(q, nf, T, n_mol):
    """Both Hadamard chains on the tensor cores (FP16 chain tables, two-part
    FP16 operands, FP32 accumulation) against the FP64 oracle: the same bounds
    as the FWHT kernel. Cases span one to 150+ tiles of 128 atoms (several
    tiles per CTA in the last), a ragged last tile, an empty molecule, odd stack
    counts (backward promotion every 2 half stacks), atoms whose x spans six
    orders of magnitude, a zero row, and weights spanning four."""
    d = 128
    x, mol_ptr, signs, b = _sorf_inputs(d, nf, T, n_mol=n_mol, seed=6 + nf)
    rng = np.random.default_rng(7 + nf)
    x *= (10.0 ** rng.uniform(-3, 3, size=(x.shape[0], 1))).astype(np.float32)
    x[min(5, x.shape[0] - 1)] = 0.0
    x = np.ascontiguousarray(x)
    sigma = 1.3 * float(np.sqrt(np.mean(np.sum(x.astype(np.float64) ** 2, axis=1))))
    alpha = (rng.normal(size=nf) * 0.05 * 10.0 ** rng.uniform(-2, 2, size=nf)).astype(np.float32)
    W = o_sorf.sorf_matrix(signs, sigma)
    xt = torch.tensor(x.astype(np.float64), requires_grad=True)
    zt = o_sorf.features(xt, W, b.astype(np.float64))
    e_atom = zt @ torch.as_tensor(alpha.astype(np.float64))
    (gref,) = torch.autograd.grad(e_atom.sum(), xt)
    gref = gref.numpy()
    sizes = np.diff(mol_ptr)
    Eref = np.array([e_atom[mol_ptr[k]:mol_ptr[k + 1]].sum().item() for k in range(len(sizes))])
    bits = q.pack_signs(signs)
    tables = q.sorf_tc_tables(bits, T, nf)
    E, gx = q.sorf_grad_tc(x, mol_ptr, tables, T, b, sigma, alpha)
    E, gx = E.cpu().numpy(), gx.cpu().numpy()[0]
    # per atom: phase error <= 2^-18 of its bound (sqrt(d)/sigma)|x| plus 2^-20
    # (sin/cos), weighted by sqrt(2/N_F) sum |alpha|; summed over the molecule
    a1 = math.sqrt(2 / nf) * float(np.sum(np.abs(alpha.astype(np.float64))))
    xn = np.linalg.norm(x.astype(np.float64), axis=1)
    tol_a = a1 * (2.0 ** -18 * math.sqrt(d) / sigma * xn + 2.0 ** -20)
    tol = np.array([tol_a[mol_ptr[k]:mol_ptr[k + 1]].sum() for k in range(len(sizes))])
    assert np.all(np.abs(E - Eref) <= tol)
    assert np.max(np.abs(gx - gref)) <= 1e-4 * np.max(np.abs(gref))
    # deterministic
    E2, gx2 = q.sorf_grad_tc(x, mol_ptr, tables, T, b, sigma, alpha)
    assert np.array_equal(E, E2.cpu().numpy()) and np.array_equal(gx, gx2.cpu().numpy()[0])
    assert q.device_status() == 0


def _ragged_molecules(rng, n_mol, big=()):
    sizes = rng.integers(1, 30, size=n_mol)
    for i, n in big:
        sizes[i] = n
    sizes[[0, n_mol // 2, n_mol - 1]] = 0          # empty first, middle and last molecules
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)


@pytest.mark.parametrize("nf,T,n_mol,big", [(128, 1, 9, ()), (1024, 3, 40, ((5, 300),)),
                                            (16384, 3, 30, ((3, 129), (7, 200))), (384, 2, 3000, ((11, 700),))])
def test_sorf_tensor_core_segment_sums_match_oracle(q, nf, T, n_mol, big):
    """Z on the tensor cores against the FP64 oracle's segment sums: molecules
    of 1-29 atoms, empty molecules (first, middle, last), molecules spanning
    two to six 128-atom tiles, up to 150+ CTAs; Z written into a row block of
    a wider matrix; every row of a molecule identical to the row the same
    molecule gets in another batch (the sum order does not depend on tiling)."""
    d = 128
    rng = np.random.default_rng(17 + nf + n_mol)
    mol_ptr = _ragged_molecules(rng, n_mol, big)
    n_atoms = int(mol_ptr[-1])
    x = (rng.normal(size=(n_atoms, d)) * 0.5).astype(np.float32)
    signs, b = synth.sorf_draw(rng, nf, d, T)
    b = b.astype(np.float32)
    sigma = 1.7
    W = o_sorf.sorf_matrix(signs, sigma)
    ref = o_sorf.features(x.astype(np.float64), W, b.astype(np.float64))
    Zref = o_reg.segment_sum(ref, mol_ptr)
    sizes = np.diff(mol_ptr)
    bits = q.pack_signs(signs)
    tables = q.sorf_tc_tables(bits, T, nf)
    big_out = torch.full((n_mol, nf + 32), float("nan"), device="cuda")
    q.sorf_segment_sum_tc(x, mol_ptr, tables, T, b, sigma, out=big_out[:, :nf])
    Z = big_out[:, :nf].cpu().numpy()
    assert torch.isnan(big_out[:, nf:]).all()
    pref = math.sqrt(2 / nf)
    assert np.all(np.max(np.abs(Z - Zref), axis=1) <= 2e-5 * pref * np.maximum(sizes, 1))
    assert np.all(Z[sizes == 0] == 0)
    # the same molecules in a different batch (shifted start, other neighbours)
    lo = n_mol // 3
    sub_ptr = (mol_ptr[lo:] - mol_ptr[lo]).astype(np.int32)
    Zs = q.sorf_segment_sum_tc(x[mol_ptr[lo]:], sub_ptr, tables, T, b, sigma).cpu().numpy()
    assert np.array_equal(Zs, Z[lo:])
    assert q.device_status() == 0


def test_sorf_tensor_core_tables_are_the_integer_chain(q):
    """The FP16 tables hold M_s = H D_T ... H D_1 exactly (unnormalised
    Hadamard, integer entries), forward [s][i][j] and backward [s][j][i]."""
    nf, d, T = 384, 128, 3
    rng = np.random.default_rng(11)
    signs, _ = synth.sorf_draw(rng, nf, d, T)
    tables = q.sorf_tc_tables(q.pack_signs(signs), T, nf).view(torch.float16).float().cpu().numpy()
    mf = tables[:nf * d].reshape(nf // d, d, d)
    mb = tables[nf * d:].reshape(nf // d, d, d)
    W = o_sorf.sorf_matrix(signs, 1.0)            # (sqrt(d)) d^{-T/2} M_s stacked
    M = W * d ** (T / 2) / math.sqrt(d)
    assert np.array_equal(mf.reshape(nf, d), np.round(M))
    assert np.allclose(M, np.round(M), atol=1e-9)
    assert np.array_equal(mb, np.transpose(mf, (0, 2, 1)))
    assert np.max(np.abs(mf)) <= d ** (T / 2)


@pytest.mark.parametrize("d,nf,n_mol", [(16, 64, 9), (64, 512, 9), (128, 1000, 9), (128, 4096, 9),
                                        (200, 300, 9), (256, 129, 9), (16, 64, 10001)])
def test_rff_tensor_core_matches_oracle(q, d, nf, n_mol):
    """Dense RFF on the tensor cores (split-BF16 GEMM, FP32 accumulation)
    against the FP64 oracle; the last case has 70 000 atoms, so the GEMM runs
    in two chunks and molecules straddle the chunk boundary. Bound: four times
    the FP32 dot-product bound of the SIMT form (the split products and the
    accumulator's adds), plus the phase add and cosf."""
    rng = np.random.default_rng(43 + d + n_mol)
    sizes = rng.integers(1, 12, size=n_mol) if n_mol < 100 else np.full(n_mol, 7)
    sizes[2] = 0
    mol_ptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    x = (rng.normal(size=(int(mol_ptr[-1]), d)) * 0.5).astype(np.float32)
    G, b = synth.rff_draw(rng, nf, d)
    G, b = G.astype(np.float32), b.astype(np.float32)
    sigma = 1.7
    xd, Gd, bd = x.astype(np.float64), G.astype(np.float64), b.astype(np.float64)
    ref = o_sorf.features(xd, o_sorf.rff_matrix(Gd, sigma), bd)
    pref = math.sqrt(2 / nf)
    u = xd @ Gd.T / sigma + bd
    bound = pref * (4 * d * 2.0 ** -24 * (np.abs(xd) @ np.abs(Gd).T) / sigma + 2.0 ** -23 * np.abs(u) + 1e-6)
    z = q.rff_tc(x, mol_ptr, G, b, sigma, q.SORF_PER_ATOM).cpu().numpy()
    assert q.device_status() == 0
    assert np.all(np.abs(z - ref) <= bound), np.max(np.abs(z - ref) / bound)
    Z = q.rff_tc(x, mol_ptr, G, b, sigma, q.SORF_PER_MOL).cpu().numpy()
    Zref = o_reg.segment_sum(ref, mol_ptr)
    Zbound = o_reg.segment_sum(bound, mol_ptr) + pref * 2.0 ** -22 * (sizes[:, None] + 1) ** 2
    assert np.all(np.abs(Z - Zref) <= Zbound), np.max(np.abs(Z - Zref) / Zbound)
    assert np.all(Z[sizes == 0] == 0)
    assert np.array_equal(Z, q.rff_tc(x, mol_ptr, G, b, sigma, q.SORF_PER_MOL).cpu().numpy())
