"""The library's host cell list for periodic systems against the oracle's
brute-force image enumeration (CPU only): the same (j, n) entries for every
atom, in (j, n) order, for large and small (r_cut longer than the cell)
triclinic cells and for coordinates outside the cell; the entries reproduce
the oracle's periodic representation; bad inputs are rejected."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import fchl19


@pytest.fixture(scope="module")
def q():
    from paper_2206_01580_gb300 import qmlr
    qmlr.lib()
    return qmlr


def brute(x, cell, rcut):
    """Oracle: every (j, n) with |x_j + n . cell - x_i| < rcut, i itself excluded."""
    T = fchl19.lattice_translations(cell, rcut)
    span = np.max(np.abs(x @ np.linalg.inv(cell)), axis=0)         # fractional extent of the inputs
    g = np.arange(-int(np.max(np.abs(T))) - int(np.ceil(span.max())) - 1,
                  int(np.max(np.abs(T))) + int(np.ceil(span.max())) + 2)
    n = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    sh = n @ cell
    out = []
    for i in range(len(x)):
        rel = x[None, :, :] + sh[:, None, :] - x[i][None, None, :]
        keep = np.sum(rel * rel, axis=-1) < rcut * rcut
        keep[np.all(n == 0, axis=1), i] = False
        kk, jj = np.nonzero(keep)
        out.append(sorted((int(j), *map(int, n[k])) for k, j in zip(kk, jj)))
    return out


def lib_entries(q, x, cell, rcut):
    ptr, atom, shift = q.periodic_environment(x, cell, rcut)
    return [sorted((int(atom[e]), *map(int, shift[e])) for e in range(ptr[i], ptr[i + 1])) for i in range(len(x))], \
        (ptr, atom, shift)


CELLS = {
    "cubic-large": np.eye(3) * 13.0,
    "triclinic-large": np.array([[12.5, 0, 0], [3.1, 13.2, 0], [-2.2, 1.7, 12.9]]),
    "triclinic-small": np.array([[3.3, 0.0, 0.0], [0.8, 3.6, 0.0], [0.3, -0.5, 3.9]]),
    "slab": np.array([[14.0, 0, 0], [0, 2.9, 0], [0.7, 0.4, 15.0]]),
}


@pytest.mark.parametrize("name", sorted(CELLS))
def test_cell_list_matches_brute_force(q, name):
    cell = CELLS[name]
    rng = np.random.default_rng(len(name))
    n = 40 if "large" in name or name == "slab" else 5
    x = rng.uniform(0, 1, size=(n, 3)) @ cell
    got, (ptr, atom, shift) = lib_entries(q, x, cell, 6.0)
    assert got == brute(x, cell, 6.0)
    # entries of one atom come sorted by (j, n)
    for i in range(n):
        seg = [(int(atom[e]), *map(int, shift[e])) for e in range(ptr[i], ptr[i + 1])]
        assert seg == sorted(seg)


def test_coordinates_outside_the_cell(q):
    cell = CELLS["triclinic-small"]
    rng = np.random.default_rng(9)
    s = rng.uniform(-1.5, 2.5, size=(6, 3))
    x = s @ cell
    got, _ = lib_entries(q, x, cell, 6.0)
    assert got == brute(x, cell, 6.0)


def test_entries_reproduce_the_oracle_periodic_representation(q):
    p = fchl19.params("EF", n2=24, n3=22)
    cell = CELLS["triclinic-small"]
    x = np.array([[0.2, 0.1, 0.3], [1.4, 0.9, 0.2], [0.7, 2.0, 1.8]])
    elem = np.array([1, 3, 0])
    ref = fchl19.representation_periodic(torch.as_tensor(x), elem, cell, p).numpy()
    ptr, atom, shift = q.periodic_environment(x, cell, p.rcut)
    rows = []
    for i in range(3):
        e = slice(ptr[i], ptr[i + 1])
        v = x[atom[e]] + shift[e] @ cell - x[i]
        rows.append(fchl19.environment_row(torch.as_tensor(v), elem[atom[e]], p).numpy())
    got = np.stack(rows)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_empty_system_and_bad_inputs(q):
    ptr, atom, shift = q.periodic_environment(np.zeros((0, 3)), np.eye(3) * 5, 6.0)
    assert list(ptr) == [0] and len(atom) == 0
    with pytest.raises(q.QMLRError, match="singular"):
        q.periodic_environment(np.zeros((2, 3)), np.array([[1.0, 0, 0], [2.0, 0, 0], [0, 0, 1.0]]), 6.0)
    with pytest.raises(q.QMLRError, match="r_cut"):
        q.periodic_environment(np.zeros((2, 3)), np.eye(3) * 5, -1.0)
    # offsets that do not match the coordinates
    L = q.lib()
    x = np.ascontiguousarray(np.random.default_rng(1).uniform(0, 5, size=(3, 3)))
    A = np.ascontiguousarray(np.eye(3) * 5.0)
    ptr = np.zeros(4, np.int64)
    assert L.qmlr_periodic_environment_count(x.ctypes.data, 3, A.ctypes.data, 6.0, ptr.ctypes.data) == 0
    ptr[1:] += 1
    atom = np.zeros(int(ptr[-1]) + 8, np.int32)
    shift = np.zeros((int(ptr[-1]) + 8, 3), np.int32)
    rc = L.qmlr_periodic_environment(x.ctypes.data, 3, A.ctypes.data, 6.0, ptr.ctypes.data, atom.ctypes.data,
                                     shift.ctypes.data)
    assert rc == q.EINVAL
    assert b"env_ptr does not match" in L.qmlr_last_error()
