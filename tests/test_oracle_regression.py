"""Pins for the FP64 regression oracle: library least squares, SVD, reductions."""
import numpy as np
import pytest

from oracle import regression


def test_ridge_solve_matches_augmented_lstsq():
    rng = np.random.default_rng(0)
    n, f, lam = 200, 64, 1e-3
    Z = rng.normal(size=(n, f))
    y = rng.normal(size=n)
    alpha, res = regression.ridge_solve(Z, y, lam)
    aug = np.concatenate([Z, np.sqrt(lam) * np.eye(f)])
    want = np.linalg.lstsq(aug, np.concatenate([y, np.zeros(f)]), rcond=None)[0]
    np.testing.assert_allclose(alpha, want, rtol=1e-9, atol=1e-12)
    assert res < 1e-12


def test_ridge_solve_underdetermined_tiny_lambda():
    rng = np.random.default_rng(1)
    n, f, lam = 40, 64, 1e-6
    Z = rng.normal(size=(n, f))
    y = rng.normal(size=n)
    alpha, res = regression.ridge_solve(Z, y, lam, refine=2)
    aug = np.concatenate([Z, np.sqrt(lam) * np.eye(f)])
    want = np.linalg.lstsq(aug, np.concatenate([y, np.zeros(f)]), rcond=None)[0]
    np.testing.assert_allclose(Z @ alpha, Z @ want, rtol=1e-8, atol=1e-10)
    assert res < 1e-10


def test_normal_equation_residual():
    rng = np.random.default_rng(2)
    Z = rng.normal(size=(300, 50))
    y = rng.normal(size=300)
    alpha, _ = regression.ridge_solve(Z, y, 1e-6)
    A = Z.T @ Z + 1e-6 * np.eye(50)
    r = Z.T @ y - A @ alpha
    assert np.linalg.norm(r) / np.linalg.norm(Z.T @ y) < 1e-12


def test_pca_basis_matches_svd_up_to_sign():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(500, 40)) * np.linspace(3, 0.1, 40)   # distinct singular values
    U = regression.pca_basis(X, 16)
    Us = np.linalg.svd(X.T, full_matrices=False)[0][:, :16]   # columns of Z~ are the reps
    for c in range(16):
        assert abs(abs(U[:, c] @ Us[:, c]) - 1) < 1e-10
        k = np.argmax(np.abs(U[:, c]))
        assert U[k, c] > 0
    np.testing.assert_allclose(U.T @ U, np.eye(16), atol=1e-12)


def test_pca_basis_zero_fills_beyond_rank():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(5, 30))                    # rank 5
    U = regression.pca_basis(X, 8)
    assert np.all(U[:, 5:] == 0)
    np.testing.assert_allclose(U[:, :5].T @ U[:, :5], np.eye(5), atol=1e-10)


def test_project_uses_element_basis():
    rng = np.random.default_rng(5)
    reps = rng.normal(size=(6, 10))
    elem = np.array([0, 1, 2, 1, 0, 2])
    U = rng.normal(size=(3, 10, 4))
    x = regression.project(reps, elem, U)
    for i in range(6):
        np.testing.assert_allclose(x[i], np.einsum("k,kd->d", reps[i], U[elem[i]]), rtol=1e-14)


def test_segment_sum_matches_reduceat():
    rng = np.random.default_rng(6)
    z = rng.normal(size=(20, 7))
    ptr = np.array([0, 3, 3, 11, 20])
    Z = regression.segment_sum(z, ptr)
    want = np.add.reduceat(z, [0, 3, 11], axis=0)
    np.testing.assert_allclose(Z[[0, 2, 3]], want, rtol=1e-14)
    assert np.all(Z[1] == 0)
