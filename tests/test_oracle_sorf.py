"""Pins for the FP64 SORF/RFF oracle: explicit Hadamard matrices, orthogonality,
textbook special cases and convergence to the Gaussian kernel (RFF and SORF
sections of the paper)."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import sorf


@pytest.mark.parametrize("d", [1, 2, 4, 8, 16, 64])
def test_hadamard_is_sylvester(d):
    H = sorf.hadamard(d)
    np.testing.assert_array_equal(H, scipy.linalg.hadamard(d))
    np.testing.assert_array_equal(H @ H, d * np.eye(d))


def test_hadamard_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        sorf.hadamard(12)


def test_single_transform_is_h_d_over_sigma():
    """N_transform = 1: W = (sqrt(d)/sigma) (H/sqrt(d)) D = H D / sigma."""
    rng = np.random.default_rng(0)
    d, sigma = 16, 1.7
    s = rng.choice([-1, 1], size=(3, 1, d))
    W = sorf.sorf_matrix(s, sigma)
    for k in range(3):
        np.testing.assert_allclose(W[k * d:(k + 1) * d],
                                   scipy.linalg.hadamard(d) @ np.diag(s[k, 0]) / sigma, rtol=1e-14)


def test_two_transforms_apply_first_diagonal_first():
    """N_transform = 2: W x = (1/(sigma sqrt(d))) H D_2 H D_1 x."""
    rng = np.random.default_rng(1)
    d, sigma = 32, 0.9
    s = rng.choice([-1, 1], size=(1, 2, d))
    x = rng.normal(size=d)
    Hd = scipy.linalg.hadamard(d)
    want = Hd @ (s[0, 1] * (Hd @ (s[0, 0] * x))) / (sigma * math.sqrt(d))
    np.testing.assert_allclose(sorf.sorf_matrix(s, sigma) @ x, want, rtol=1e-13)


@pytest.mark.parametrize("T", [1, 2, 3])
def test_stack_rows_are_orthogonal(T):
    rng = np.random.default_rng(2)
    d, sigma = 64, 2.0
    s = rng.choice([-1, 1], size=(4, T, d))
    W = sorf.sorf_matrix(s, sigma)
    for k in range(4):
        Wk = W[k * d:(k + 1) * d]
        np.testing.assert_allclose(Wk @ Wk.T, d / sigma**2 * np.eye(d), atol=1e-11)


def _kernel_error(W, b, xs, ys, sigma):
    zx = sorf.features(xs, W, b)
    zy = sorf.features(ys, W, b)
    approx = np.sum(zx * zy, axis=1)
    exact = np.array([sorf.gaussian_kernel(x, y, sigma) for x, y in zip(xs, ys)])
    return np.sqrt(np.mean((approx - exact) ** 2))


def _pairs(rng, d, sigma, n=64):
    xs = rng.normal(size=(n, d)) * 0.3
    dirs = rng.normal(size=(n, d))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    ys = xs + dirs * rng.uniform(0.2, 2.0, size=(n, 1)) * sigma
    return xs, ys


def test_sorf_converges_to_gaussian_kernel():
    rng = np.random.default_rng(3)
    d, sigma = 64, 1.5
    xs, ys = _pairs(rng, d, sigma)
    errs = []
    for nf in (256, 4096, 65536):
        s = rng.choice([-1, 1], size=(nf // d, 3, d))
        b = rng.uniform(0, 2 * math.pi, size=nf)
        errs.append(_kernel_error(sorf.sorf_matrix(s, sigma), b, xs, ys, sigma))
    # Monte Carlo error ~ N_F^{-1/2}: 256x more features -> ~16x smaller error
    assert errs[-1] < 0.01
    assert errs[0] / errs[-1] > 6.0


def test_rff_converges_to_gaussian_kernel():
    rng = np.random.default_rng(4)
    d, sigma = 64, 1.5
    xs, ys = _pairs(rng, d, sigma)
    errs = []
    for nf in (256, 4096, 65536):
        G = rng.normal(size=(nf, d))
        b = rng.uniform(0, 2 * math.pi, size=nf)
        errs.append(_kernel_error(sorf.rff_matrix(G, sigma), b, xs, ys, sigma))
    assert errs[-1] < 0.01
    assert errs[0] / errs[-1] > 6.0


def test_sorf_kernel_width_is_sigma():
    """A wrong scale (e.g. dropping sqrt(d)) changes the kernel width: fit it back."""
    rng = np.random.default_rng(5)
    d, sigma, nf = 64, 2.0, 65536
    s = rng.choice([-1, 1], size=(nf // d, 3, d))
    b = rng.uniform(0, 2 * math.pi, size=nf)
    W = sorf.sorf_matrix(s, sigma)
    x = np.zeros(d)
    u = rng.normal(size=d)
    u /= np.linalg.norm(u)
    rs = np.linspace(0.5, 4.0, 8)
    k = [float(np.sum(sorf.features(x[None], W, b) * sorf.features((x + r * u)[None], W, b)))
         for r in rs]
    # -2 ln k = r^2 / sigma^2  -> slope 1/sigma^2
    slope = np.polyfit(rs**2, -2 * np.log(np.clip(k, 1e-6, None)), 1)[0]
    assert slope == pytest.approx(1 / sigma**2, rel=0.1)


def test_features_bounded():
    rng = np.random.default_rng(6)
    s = rng.choice([-1, 1], size=(4, 3, 16))
    b = rng.uniform(0, 2 * math.pi, size=64)
    z = sorf.features(rng.normal(size=(10, 16)), sorf.sorf_matrix(s, 1.0), b)
    assert np.max(np.abs(z)) <= math.sqrt(2 / 64) + 1e-15
