"""Pins for the FP64 FCHL19 oracle: closed forms, special geometries and invariances.

Each test checks the oracle against something other than itself: scipy's
log-normal and normal densities, hand-built triangles whose angles are known
in closed form, the paper's parameter table, and the symmetries the paper
claims for FCHL19 (Representation section: permutation and rotation
invariance).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.stats
import torch

from oracle import fchl19

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fchl19_params.json")
H, C, N, O, F = range(5)


def rep(x, elem, p):
    return fchl19.representation(torch.as_tensor(np.asarray(x, dtype=np.float64)),
                                 np.asarray(elem), p).numpy()


def P(column="E"):
    return fchl19.params(column, n2=24, n3=22)


def test_table_matches_paper():
    g = json.load(open(GOLDEN))
    for col in ("E", "EF"):
        for k, v in g[col].items():
            want = math.pi if v == "pi" else v
            assert fchl19.PAPER_TABLE[col][k] == pytest.approx(want, rel=0, abs=0), (col, k)


def test_rep_dim_is_780():
    assert P().rep_dim == 5 * 24 + 15 * 22 * 2 == 780


def test_cutoff_values():
    p = P()
    r = torch.tensor([0.0, p.rcut / 2, p.rcut, p.rcut + 1.0, 2 * p.rcut], dtype=torch.float64)
    assert fchl19.cutoff(r, p.rcut).tolist() == pytest.approx([1.0, 0.5, 0.0, 0.0, 0.0], abs=1e-15)


@pytest.mark.parametrize("column", ["E", "EF"])
@pytest.mark.parametrize("r", [0.74, 1.1, 2.3, 4.9])
def test_two_body_diatomic_is_lognormal_pdf(column, r):
    p = P(column)
    x = [[0, 0, 0], [r, 0, 0]]
    out = rep(x, [N, F], p)
    Rs = p.rcut * np.arange(1, p.n2 + 1) / p.n2
    s = math.sqrt(math.log(1 + p.eta2 / r**2))
    mu = math.log(r / math.sqrt(1 + p.eta2 / r**2))
    fc = 0.5 * (math.cos(math.pi * r / p.rcut) + 1)
    want = fc * r ** (-p.N2) * scipy.stats.lognorm.pdf(Rs, s=s, scale=math.exp(mu))
    # atom 0 (N) sees an F neighbour: block of element F only
    np.testing.assert_allclose(out[0, F * p.n2:(F + 1) * p.n2], want, rtol=1e-13, atol=1e-300)
    np.testing.assert_allclose(out[1, N * p.n2:(N + 1) * p.n2], want, rtol=1e-13, atol=1e-300)
    mask = np.ones(p.rep_dim, dtype=bool)
    mask[F * p.n2:(F + 1) * p.n2] = False
    assert np.all(out[0, mask] == 0.0)          # no other element block, no three-body
    mask = np.ones(p.rep_dim, dtype=bool)
    mask[N * p.n2:(N + 1) * p.n2] = False
    assert np.all(out[1, mask] == 0.0)


def test_two_body_same_element_pair_adds():
    p = P()
    x = [[0, 0, 0], [1.0, 0, 0], [-1.7, 0, 0]]
    out = rep(x, [C, H, H], p)
    two = out[0, H * p.n2:(H + 1) * p.n2]
    a = rep([[0, 0, 0], [1.0, 0, 0]], [C, H], p)[0, H * p.n2:(H + 1) * p.n2]
    b = rep([[0, 0, 0], [-1.7, 0, 0]], [C, H], p)[0, H * p.n2:(H + 1) * p.n2]
    np.testing.assert_allclose(two, a + b, rtol=1e-14)


def test_beyond_cutoff_is_zero_and_continuous():
    p = P()
    out = rep([[0, 0, 0], [p.rcut, 0, 0]], [C, O], p)
    assert np.all(out == 0.0)
    near = rep([[0, 0, 0], [p.rcut - 1e-6, 0, 0]], [C, O], p)
    assert np.max(np.abs(near)) < 1e-12


def _three_body_block(out_row, p, a, b):
    off = p.n_el * p.n2 + fchl19.pair_index(a, b, p.n_el) * p.n3 * 2
    return out_row[off:off + 2 * p.n3].reshape(p.n3, 2)


@pytest.mark.parametrize("column", ["E", "EF"])
@pytest.mark.parametrize("side", [1.2, 2.0, 3.1])
def test_equilateral_triangle_closed_form(column, side):
    p = P(column)
    x = [[0, 0, 0], [side, 0, 0], [side / 2, side * math.sqrt(3) / 2, 0]]
    out = rep(x, [C, H, O], p)
    Rs = p.rcut * np.arange(1, p.n3 + 1) / p.n3
    fc = 0.5 * (math.cos(math.pi * side / p.rcut) + 1)
    atm = p.c3 * (1 + 3 * 0.125) / side ** (3 * p.N3)          # cos 60 deg = 1/2 at every vertex
    radial = scipy.stats.norm.pdf(side, loc=Rs, scale=1 / math.sqrt(2 * p.eta3))
    ang = math.exp(-p.zeta**2 / 2) * np.array([1.0, math.sqrt(3.0)])   # [2 cos 60, 2 sin 60]
    want = atm * fc**3 * radial[:, None] * ang[None, :]
    # centre C sees the pair {H, O}; centre H sees {C, O}; centre O sees {H, C}
    for centre, (a, b) in [(0, (H, O)), (1, (C, O)), (2, (C, H))]:
        got = _three_body_block(out[centre], p, a, b)
        np.testing.assert_allclose(got, want, rtol=1e-12)
        three = out[centre, p.n_el * p.n2:].copy()
        off = fchl19.pair_index(a, b, p.n_el) * p.n3 * 2
        three[off:off + 2 * p.n3] = 0
        assert np.all(three == 0.0)


def test_right_angle_triangle_angle_at_centre():
    """Right angle at atom 0: for that centre G^cos = 0 and G^sin = 2 exp(-zeta^2/2);
    the radial term is centred at (r_ij + r_ik)/2 of the two sides that meet at the centre."""
    p = P("EF")
    a, b = 1.3, 2.1
    hyp = math.hypot(a, b)
    x = [[0, 0, 0], [a, 0, 0], [0, b, 0]]
    out = rep(x, [N, C, C], p)
    Rs = p.rcut * np.arange(1, p.n3 + 1) / p.n3
    fc = lambda r: 0.5 * (math.cos(math.pi * r / p.rcut) + 1)
    fcs = fc(a) * fc(b) * fc(hyp)
    atm = p.c3 * 1.0 / (a * b * hyp) ** p.N3                   # one cosine is zero
    damp = math.exp(-p.zeta**2 / 2)
    # centre 0 (right angle)
    got = _three_body_block(out[0], p, C, C)
    rad = scipy.stats.norm.pdf((a + b) / 2, loc=Rs, scale=1 / math.sqrt(2 * p.eta3))
    np.testing.assert_allclose(got[:, 0], 0.0, atol=1e-14 * np.max(np.abs(got)))
    np.testing.assert_allclose(got[:, 1], atm * fcs * rad * 2 * damp, rtol=1e-12)
    # centre 1: angle between the sides of length a and hyp, cos = a / hyp
    got = _three_body_block(out[1], p, N, C)
    rad = scipy.stats.norm.pdf((a + hyp) / 2, loc=Rs, scale=1 / math.sqrt(2 * p.eta3))
    c1 = a / hyp
    s1 = b / hyp
    np.testing.assert_allclose(got[:, 0], atm * fcs * rad * 2 * damp * c1, rtol=1e-12)
    np.testing.assert_allclose(got[:, 1], atm * fcs * rad * 2 * damp * s1, rtol=1e-12)


def test_three_body_needs_r_jk_inside_cutoff():
    """f_cut(r_jk) as printed: two neighbours of i farther than r_cut apart add no three-body term."""
    p = P()
    x = [[0, 0, 0], [3.5, 0, 0], [-3.5, 0, 0]]
    out = rep(x, [C, H, H], p)
    assert np.all(out[0, p.n_el * p.n2:] == 0.0)
    assert np.any(out[0, :p.n_el * p.n2] != 0.0)


def _random_molecule(rng, n=11):
    x = rng.uniform(0, 4.5, size=(n, 3))
    e = rng.integers(0, 5, size=n)
    return x, e


def test_rotation_translation_invariance():
    rng = np.random.default_rng(7)
    x, e = _random_molecule(rng)
    p = P()
    base = rep(x, e, p)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    moved = x @ Q.T + rng.normal(size=3) * 10
    np.testing.assert_allclose(rep(moved, e, p), base, rtol=1e-11, atol=1e-12 * np.abs(base).max())


def test_permutation_equivariance():
    rng = np.random.default_rng(8)
    x, e = _random_molecule(rng)
    p = P()
    base = rep(x, e, p)
    perm = rng.permutation(len(e))
    np.testing.assert_allclose(rep(x[perm], e[perm], p), base[perm], rtol=1e-12,
                               atol=1e-13 * np.abs(base).max())


def test_far_atom_changes_nothing():
    rng = np.random.default_rng(9)
    x, e = _random_molecule(rng, 7)
    p = P()
    base = rep(x, e, p)
    far = np.concatenate([x, [[40.0, 40.0, 40.0]]])
    out = rep(far, np.concatenate([e, [C]]), p)
    np.testing.assert_allclose(out[:-1], base, rtol=0, atol=0)
    assert np.all(out[-1] == 0.0)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(10)
    x, e = _random_molecule(rng, 6)
    p = P("EF")
    R = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    g = torch.as_tensor(rng.normal(size=(6, p.rep_dim)))
    (grad,) = torch.autograd.grad((fchl19.representation(R, e, p) * g).sum(), R)
    h = 1e-4
    fd = np.zeros_like(x)
    for k in range(6):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, a] += h
            xm[k, a] -= h
            fd[k, a] = (np.sum(rep(xp, e, p) * g.numpy()) - np.sum(rep(xm, e, p) * g.numpy())) / (2 * h)
    np.testing.assert_allclose(grad.numpy(), fd, rtol=1e-6, atol=1e-7 * np.abs(fd).max())


# The three-body block layout (the representation's concatenation order, read
# as row-major upper-triangular order over unordered element pairs a <= b),
# written out by hand for five elements so that the pin does not depend on the
# oracle's own pair_index.
PAIR_TABLE_5 = {
    (0, 0): 0, (0, 1): 1, (0, 2): 2, (0, 3): 3, (0, 4): 4,
    (1, 1): 5, (1, 2): 6, (1, 3): 7, (1, 4): 8,
    (2, 2): 9, (2, 3): 10, (2, 4): 11,
    (3, 3): 12, (3, 4): 13,
    (4, 4): 14,
}


def test_pair_index_is_the_upper_triangular_order():
    seen = set()
    for a in range(5):
        for b in range(5):
            want = PAIR_TABLE_5[(min(a, b), max(a, b))]
            assert fchl19.pair_index(a, b, 5) == want, (a, b)
            seen.add(want)
    assert seen == set(range(15))          # a bijection onto 0..14


@pytest.mark.parametrize("pair", sorted(PAIR_TABLE_5))
def test_three_body_block_lands_at_its_table_offset(pair):
    """A centre with exactly one triplet of neighbour elements (a, b): every
    non-zero three-body entry of its row lies in the block the table names."""
    p = P()
    a, b = pair
    x = [[0, 0, 0], [1.3, 0, 0], [0.4, 1.2, 0]]
    out = rep(x, [C, a, b], p)[0]
    off = p.n_el * p.n2 + PAIR_TABLE_5[pair] * p.n3 * 2
    three = out[p.n_el * p.n2:]
    nz = np.nonzero(three)[0] + p.n_el * p.n2
    assert len(nz) > 0
    assert nz.min() >= off and nz.max() < off + 2 * p.n3, (pair, nz.min(), nz.max(), off)
