"""GPU parity of the normal-equation path through the C ABI: split-BF16
operands, the plain-FP32 and tensor-core Gram, Z^T y, the FP64 Cholesky
factor and solves, and the refined ridge solve against the FP64 oracle.

Tolerances: Gram max-abs error <= 4e-5 * max|G| for plain FP32 (accumulation)
and the 2-way BF16 split (products ~2^-16 relative), <= 1e-5 for the 3-way
split (~2^-24 products, FP32 accumulation); Z^T y and Cholesky: FP64 round-off
(rel 1e-10); solves: relative normal-equation residual <= tol with the exact
FP64 operator, and predictions Z alpha within 1e-6 relative of the oracle's.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import torch

from oracle import regression as o_reg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_01580_gb300 import qmlr
    qmlr.lib()
    return qmlr


def _features(n_rows, nf, seed=0):
    """Rows shaped like per-molecule SORF sums: sums of a few bounded cosines."""
    rng = np.random.default_rng(seed)
    atoms = rng.integers(3, 12, size=n_rows)
    Z = np.zeros((n_rows, nf), np.float32)
    pref = math.sqrt(2 / nf)
    for r in range(n_rows):
        Z[r] = pref * np.cos(rng.normal(size=(atoms[r], nf)) * 2 + rng.uniform(0, 6.3, nf)).sum(0)
    return Z


@pytest.mark.parametrize("n_split", [1, 2, 3])
def test_gram_operand_is_bf16_split(q, n_split):
    Z = _features(100, 256)
    zt = q.gram_operand(Z, n_split).cpu()
    assert zt.shape == (n_split, 256, 128)
    rem = torch.as_tensor(Z).T.contiguous()
    for k in range(n_split):
        want = rem.to(torch.bfloat16)
        assert torch.equal(zt[k, :, :100].view(torch.bfloat16), want)
        assert torch.all(zt[k, :, 100:] == 0)
        rem = rem - want.float()


GRAM_TOL = {0: 4e-5, 1: 4e-5, 2: 1e-5}


def test_fp8_operand_matches_oracle_rounding(q):
    """e4m3 operand: per-feature power-of-two scales and round-to-nearest-even
    values equal the oracle's definition bit for bit; K padding is zero."""
    Z = _features(300, 256, seed=31)
    Z[:, 5] = 0.0                                   # an all-zero feature keeps scale 1
    Z[:, 7] *= 1e-3
    zt, inv = q.gram_operand_fp8(Z)
    assert zt.shape == (256, 384)
    s = o_reg.fp8_feature_scales(Z.astype(np.float64))
    assert np.array_equal(1.0 / inv.cpu().numpy().astype(np.float64), s)
    got = zt.cpu().view(torch.float8_e4m3fn).float().numpy().astype(np.float64)
    want = o_reg.round_to_format(Z.astype(np.float64) * s[None, :], o_reg.E4M3_FORMAT).T
    assert np.array_equal(got[:, :300], want)
    assert np.all(got[:, 300:] == 0)


# (precision, promote, tile_n) of the configurable tensor-core Gram
REDUCED_FORMS = [(3, 0, 256), (3, 0, 128), (3, 2, 256), (4, 0, 256), (4, 3, 128)]


@pytest.mark.parametrize("n_rows,nf", [(1000, 256), (777, 512), (4096, 768)])
@pytest.mark.parametrize("form", REDUCED_FORMS)
def test_reduced_precision_gram_matches_quantized_oracle(q, n_rows, nf, form):
    """One-part BF16 and e4m3 Grams equal Q^T Q of the oracle's rounded operand
    up to the FP32 accumulation (bound: K 2^-23 of the largest diagonal entry,
    the worst case of truncating adds)."""
    precision, promote, tile = form
    Z = _features(n_rows, nf, seed=n_rows + 3 * nf)
    ref = o_reg.quantized_gram(Z.astype(np.float64), "bf16" if precision == 3 else "e4m3")
    G = q.gram_tc(Z, precision, promote=promote, tile_n=tile).cpu().numpy()
    assert q.device_status() == 0
    scale = np.max(np.diag(ref))
    err = np.max(np.abs(G - ref)) / scale
    assert err <= n_rows * 2.0 ** -23, err
    assert np.array_equal(G, G.T)


@pytest.mark.parametrize("form", [(3, 0, 256), (4, 0, 256), (1, 0, 256), (1, 1, 128)])
def test_reduced_precision_gram_several_waves(q, form):
    """380 tiles of 128 x 256 (or 703 of 128 x 128): several waves of the
    persistent launch; the 2-way split without per-block promotion against FP64."""
    precision, promote, tile = form
    Z = _features(600, 4864, seed=41)
    G = q.gram_tc(Z, precision, promote=promote, tile_n=tile).cpu().numpy()
    assert q.device_status() == 0
    if precision == 1:
        Zd = Z.astype(np.float64)
        ref = Zd.T @ Zd
        tol = GRAM_TOL[1] + 600 * 2.0 ** -23
    else:
        ref = o_reg.quantized_gram(Z.astype(np.float64), "bf16" if precision == 3 else "e4m3")
        tol = 600 * 2.0 ** -23
    err = np.max(np.abs(G - ref)) / np.max(np.diag(ref))
    assert err <= tol, err
    assert np.array_equal(G, G.T)
    if form == (1, 1, 128):            # the default 2-way form: bitwise the qmlr_gram result
        assert np.array_equal(G, q.gram(Z, q.GRAM_BF16X3).cpu().numpy())


@pytest.mark.parametrize("n_rows,nf", [(64, 128), (1000, 256), (777, 384), (4096, 1024), (130, 512)])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_gram_matches_fp64(q, n_rows, nf, precision):
    Z = _features(n_rows, nf, seed=n_rows + nf)
    ref = Z.astype(np.float64).T @ Z.astype(np.float64)
    G = q.gram(Z, precision).cpu().numpy()
    assert q.device_status() == 0
    err = np.max(np.abs(G - ref)) / np.max(np.abs(ref))
    assert err <= GRAM_TOL[precision], err
    assert np.array_equal(G, G.T)


@pytest.mark.parametrize("precision", [1, 2])
def test_persistent_gram_matches_fp64(q, precision):
    """Enough tiles (37 x 38 / 2 = 703 >= 4 per SM) for the persistent,
    wave-aligned tensor-core Gram; a ragged K (600 rows, not a multiple of 64)."""
    Z = _features(600, 4736, seed=17)
    Zd = torch.as_tensor(Z, dtype=torch.float64)
    ref = (Zd.T @ Zd).numpy()
    G = q.gram(Z, precision).cpu().numpy()
    assert q.device_status() == 0
    err = np.max(np.abs(G - ref)) / np.max(np.abs(ref))
    assert err <= GRAM_TOL[precision], err
    assert np.array_equal(G, G.T)


@pytest.mark.parametrize("tc_form", [None, (1, 256)])
def test_gram_at_full_size_on_sampled_entries(q, tc_form):
    """The 2-way tensor-core Gram at the training size (100,000 molecules x
    16,384 features): qmlr_gram's form (Kahan sums, 128-wide tiles) and the
    training step's (every K block promoted into plain FP32 sums, 256-wide
    tiles). 256 sampled entries, every tile row and column touched, against
    FP64 dot products of the sampled columns."""
    n_rows, nf = 100_000, 16_384
    g = torch.Generator(device="cuda").manual_seed(23)
    Z = (torch.rand(n_rows, nf, device="cuda", generator=g) - 0.5) * 0.1
    if tc_form is None:
        G = q.gram(Z, q.GRAM_BF16X3)
    else:
        G = q.gram_tc(Z, q.GRAM_BF16X3, promote=tc_form[0], tile_n=tc_form[1])
    assert q.device_status() == 0
    rng = np.random.default_rng(24)
    ii = np.concatenate([np.arange(0, nf, 128), np.arange(127, nf, 128)])[:256]
    jj = rng.integers(0, nf, size=ii.size)
    jj[:128] = ii[:128]   # diagonal entries
    cols = np.unique(np.concatenate([ii, jj]))
    Zc = Z[:, torch.as_tensor(cols, device="cuda")].double().cpu().numpy()
    pos = {c: k for k, c in enumerate(cols)}
    ref = np.array([Zc[:, pos[i]] @ Zc[:, pos[j]] for i, j in zip(ii, jj)])
    got = G[torch.as_tensor(ii, device="cuda"), torch.as_tensor(jj, device="cuda")].double().cpu().numpy()
    scale = np.max(np.abs(np.diag(Zc.T @ Zc)))
    assert np.max(np.abs(got - ref)) <= GRAM_TOL[1] * scale
    sym = G[torch.as_tensor(jj, device="cuda"), torch.as_tensor(ii, device="cuda")].double().cpu().numpy()
    assert np.array_equal(got, sym)


def test_tensor_core_gram_is_unbiased_on_long_sums(q):
    """Tensor-core accumulator adds truncate; the kernel promotes every 64-row K
    block into FP32 Kahan sums, so the diagonal (sums of 6000 positive terms)
    carries no systematic relative bias beyond FP32 rounding."""
    Z = _features(6000, 256, seed=21)
    ref = np.einsum("ij,ij->j", Z.astype(np.float64), Z.astype(np.float64))
    for precision, tol in ((0, 1e-6), (2, 1e-6)):
        G = q.gram(Z, precision).cpu().numpy()
        bias = np.mean(np.diag(G) / ref - 1.0)
        assert abs(bias) <= tol, (precision, bias)


@pytest.mark.parametrize("n_rows,nf", [(1, 7), (4099, 300), (2500, 1024)])
def test_normal_apply_matches_fp64(q, n_rows, nf):
    """The solve's exact operator Z^T (Z p) + lam p (compensated FP32 pairs
    folded into FP64) against FP64 numpy: error <= 1e-12 of the sum of |terms|
    elementwise; repeated calls agree bitwise."""
    Z = _features(n_rows, nf, seed=n_rows)
    rng = np.random.default_rng(nf)
    pv = rng.normal(size=nf) * np.exp(rng.normal(size=nf))
    lam = 1e-3
    Zd = Z.astype(np.float64)
    ref = Zd.T @ (Zd @ pv) + lam * pv
    scale = np.abs(Zd).T @ (np.abs(Zd) @ np.abs(pv)) + lam * np.abs(pv)
    got = q.normal_apply(Z, pv, lam).cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-12 * scale), np.max(np.abs(got - ref) / scale)
    again = q.normal_apply(Z, pv, lam).cpu().numpy()
    assert np.array_equal(got, again)


def test_zty_matches_fp64(q):
    Z = _features(3000, 384, seed=5)
    y = np.random.default_rng(6).normal(size=3000)
    c = q.zty(Z, y).cpu().numpy()
    ref = Z.astype(np.float64).T @ y
    np.testing.assert_allclose(c, ref, rtol=1e-10, atol=1e-12 * np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [1, 63, 64, 100, 300])
def test_cholesky_matches_lapack(q, n):
    rng = np.random.default_rng(n)
    X = rng.normal(size=(n + 5, n))
    A = X.T @ X + 0.1 * np.eye(n)
    L, info = q.cholesky(A)
    assert info == 0
    L = np.tril(L.cpu().numpy())
    ref = np.linalg.cholesky(A)
    np.testing.assert_allclose(L, ref, rtol=1e-10, atol=1e-12 * np.max(np.abs(ref)))
    v = rng.normal(size=n)
    x = q.cholesky_solve(torch.as_tensor(L).cuda(), v).cpu().numpy()
    np.testing.assert_allclose(x, scipy.linalg.cho_solve((ref, True), v), rtol=1e-9)


@pytest.mark.parametrize("n", [1, 200, 256, 300, 600, 1000, 1333])
def test_mixed_cholesky_reconstructs_matrix(q, n):
    """Mixed factor: panels of 256 columns in FP64, tensor-core trailing updates
    from 3-way BF16 splits. L L^T reproduces A to ~1e-7 of max|A| (FP64
    round-off while n <= 256, where no tensor-core update runs), and its
    triangular solves match the FP64 factor's to the same relative order.
    The bound comes from the tensor cores' truncating accumulator: per 64-deep
    K block four large adds of ~2^-23 relative each (small split products are
    added first), over the panels that touch an element."""
    rng = np.random.default_rng(100 + n)
    X = rng.normal(size=(n + 5, n))
    A = X.T @ X + 0.1 * np.eye(n)
    L, info = q.cholesky_mixed(A)
    assert info == 0
    assert q.device_status() == 0
    L = L.cpu().numpy()
    assert np.all(np.triu(L, 1) == np.triu(A, 1))     # strict upper triangle untouched
    L = np.tril(L)
    err = np.max(np.abs(L @ L.T - A)) / np.max(np.abs(A))
    assert err <= (1e-13 if n <= 256 else 5e-7), err
    v = rng.normal(size=n)
    x = q.cholesky_solve(torch.as_tensor(L).cuda(), v).cpu().numpy()
    ref = scipy.linalg.cho_solve((np.linalg.cholesky(A), True), v)
    cond_bound = 1e-10 if n <= 256 else 1e-7 * np.linalg.cond(A)
    assert np.max(np.abs(x - ref)) <= cond_bound * np.max(np.abs(ref))


def test_mixed_cholesky_reports_indefinite_matrix(q):
    A = np.eye(700)
    A[400, 400] = -1.0          # met after two tensor-core trailing updates
    _, info = q.cholesky_mixed(A)
    assert info == 401
    assert q.device_status() == 5
    assert q.device_status() == 0


def test_cholesky_reports_indefinite_matrix(q):
    A = np.eye(80)
    A[50, 50] = -1.0
    _, info = q.cholesky(A)
    assert info == 51
    assert q.device_status() == 5
    assert q.device_status() == 0


@pytest.mark.parametrize("factor", [0, 1])
@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_ridge_solve_matches_oracle(q, method, precision, factor):
    Z = _features(1500, 640, seed=9)
    y = np.random.default_rng(10).normal(size=1500)
    lam = 1e-6
    alpha_ref, _ = o_reg.ridge_solve(Z.astype(np.float64), y, lam, refine=2)
    G = q.gram(Z, precision)
    alpha, it, rel = q.gram_solve(G, Z, y, lam, method=method, max_iter=30, tol=1e-11, factor=factor)
    assert rel <= 1e-11, (it, rel)
    alpha = alpha.cpu().numpy()
    pz, pr = Z.astype(np.float64) @ alpha, Z.astype(np.float64) @ alpha_ref
    assert np.max(np.abs(pz - pr)) <= 1e-6 * np.max(np.abs(pr))


@pytest.mark.parametrize("factor", [0, 1])
def test_ridge_solve_ragged_feature_count(q, factor):
    """N_F = 300: four 64-row blocks and a 44-row tail in the factor and in the
    preconditioner's double-float dataflow sweeps (plain FP32 Gram, which takes
    any feature count), against the FP64 oracle."""
    Z = _features(1000, 300, seed=31)
    y = np.random.default_rng(32).normal(size=1000)
    lam = 1e-6
    alpha_ref, _ = o_reg.ridge_solve(Z.astype(np.float64), y, lam, refine=2)
    G = q.gram(Z, q.GRAM_FP32)
    alpha, it, rel = q.gram_solve(G, Z, y, lam, max_iter=40, tol=1e-11, factor=factor)
    assert rel <= 1e-11, (it, rel)
    pz = Z.astype(np.float64) @ alpha.cpu().numpy()
    pr = Z.astype(np.float64) @ alpha_ref
    assert np.max(np.abs(pz - pr)) <= 1e-6 * np.max(np.abs(pr))


def test_mixed_factor_preconditions_as_well_as_fp64(q):
    """On a Gram large enough for several tensor-core panel updates the mixed
    factor needs at most two more PCG iterations than the FP64 one."""
    Z = _features(3000, 1024, seed=13)
    y = np.random.default_rng(14).normal(size=3000)
    G = q.gram(Z, 2)
    its = {}
    for f in (q.FACTOR_FP64, q.FACTOR_MIXED):
        alpha, it, rel = q.gram_solve(G, Z, y, 1e-6, max_iter=60, tol=1e-10, factor=f)
        assert rel <= 1e-10
        its[f] = it
    assert its[q.FACTOR_MIXED] <= its[q.FACTOR_FP64] + 2, its


def test_ridge_solve_underdetermined_with_shift(q):
    """Fewer rows than features (the parity workload's shape): G is rank
    deficient, so the factor is taken of G + (lambda + shift) I and the exact
    operator recovers the lambda-regularised solution."""
    Z = _features(64, 512, seed=11)
    y = np.random.default_rng(12).normal(size=64)
    lam = 1e-6
    alpha_ref, _ = o_reg.ridge_solve(Z.astype(np.float64), y, lam, refine=2)
    G = q.gram(Z, 2)
    alpha, it, rel = q.gram_solve(G, Z, y, lam, method=0, max_iter=200, tol=1e-10, shift=1e-4,
                                  factor=q.FACTOR_FP64)
    assert rel <= 1e-10, (it, rel)
    pz = Z.astype(np.float64) @ alpha.cpu().numpy()
    pr = Z.astype(np.float64) @ alpha_ref
    assert np.max(np.abs(pz - pr)) <= 1e-6 * np.max(np.abs(pr))


def test_unit_rates_are_plausible(q):
    """The diagnostic unit-rate probe: FP32 FMA and add rates within a factor of
    SMs x 128 lanes x clock, FP64 far below FP32, all rates positive."""
    r = q.unit_rates()
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 128 * 2.2e9
    assert all(v > 0 and math.isfinite(v) for v in r.values())
    assert 0.2 * nominal < r["ffma"] < 1.2 * nominal
    assert 0.2 * nominal < r["fadd"] < 1.2 * nominal
    assert r["dfma"] < r["ffma"]
