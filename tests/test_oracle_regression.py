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


def test_round_to_format_bf16_is_torch_bfloat16():
    """bfloat16 rounding (ties to even) against torch's conversion of FP32 values."""
    import torch
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-20, 20, size=5000),
                        [0.0, 1.0, -1.0, 1.00390625, 1.01171875, 3.0e38]]).astype(np.float32)
    want = torch.as_tensor(x).to(torch.bfloat16).float().numpy().astype(np.float64)
    got = regression.round_to_format(x, regression.BF16_FORMAT)
    assert np.array_equal(got, want)


def test_round_to_format_e4m3_values_of_the_format():
    """e4m3 (3 fraction bits, exponent bias 7, largest finite 448, subnormals 2^-9):
    hand-worked ties, saturation and subnormals, and torch's float8_e4m3fn on in-range values."""
    import torch
    f = regression.E4M3_FORMAT
    cases = {1.0625: 1.0, 1.1875: 1.25, 448.0: 448.0, 460.0: 448.0, 1e6: 448.0, -500.0: -448.0,
             2.0 ** -9: 2.0 ** -9, 2.0 ** -10: 0.0, 3 * 2.0 ** -10: 2.0 ** -8, 0.3: 0.3125, 17.0: 16.0,
             19.0: 20.0, 240.0: 240.0, 232.0: 224.0}
    for x, want in cases.items():
        assert regression.round_to_format(x, f) == want, (x, regression.round_to_format(x, f))
    rng = np.random.default_rng(4)
    x = (rng.normal(size=4000) * 4.0 ** rng.integers(-5, 4, size=4000)).astype(np.float32)
    x = x[np.abs(x) < 440]
    want = torch.as_tensor(x).to(torch.float8_e4m3fn).float().numpy().astype(np.float64)
    assert np.array_equal(regression.round_to_format(x, f), want)


def test_quantized_gram_definitions():
    """Q^T Q of the rounded operand: exact for values the formats hold; per-feature
    power-of-two scales for e4m3 cancel exactly; scaled columns keep their largest
    entry within 448 and above 224."""
    rng = np.random.default_rng(5)
    Z = rng.integers(-8, 9, size=(40, 6)).astype(np.float64) / 4.0       # exactly representable in both
    assert np.array_equal(regression.quantized_gram(Z, "bf16"), Z.T @ Z)
    assert np.allclose(regression.quantized_gram(Z, "e4m3"), Z.T @ Z, rtol=0, atol=0)
    Y = rng.normal(size=(300, 9)) * np.exp(rng.normal(size=9) * 3)
    s = regression.fp8_feature_scales(Y)
    amax = np.max(np.abs(Y), axis=0)
    assert np.all(amax * s <= 448.0) and np.all(amax * s > 224.0)
    assert np.all(np.log2(s) == np.round(np.log2(s)))
    G = regression.quantized_gram(Y, "e4m3")
    rel = np.abs(G - Y.T @ Y) / np.sqrt(np.outer(np.diag(Y.T @ Y), np.diag(Y.T @ Y)))
    assert np.max(rel) < 2 ** -3                       # 3 fraction bits: products within ~2^-3
    assert np.max(np.abs(regression.quantized_gram(Y, "bf16") - Y.T @ Y) /
                  np.sqrt(np.outer(np.diag(Y.T @ Y), np.diag(Y.T @ Y)))) < 2 ** -7
