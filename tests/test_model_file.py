"""The model file (checkpoint of a trained model) through the C ABI, on the
host only: a written model reads back bit for bit, and damaged files are
rejected before anything is handed out."""
import os

import numpy as np
import pytest

from paper_2206_01580_gb300 import synth


@pytest.fixture(scope="module")
def q():
    from paper_2206_01580_gb300 import qmlr
    qmlr.lib()
    return qmlr


def _model(d, n_features, T, seed=0):
    from paper_2206_01580_gb300.params import from_table
    rng = np.random.default_rng(seed)
    p = from_table("EF", n2=24, n3=22)
    U = rng.normal(size=(5, 780, d)).astype(np.float32)
    signs, b = synth.sorf_draw(rng, n_features, d, T)
    alpha = rng.normal(size=n_features) * np.exp(rng.normal(size=n_features))
    return p, U, signs, T, b.astype(np.float32), 1.7, 1e-6, alpha


@pytest.mark.parametrize("d,n_features,T", [(64, 512, 3), (16, 48, 1), (128, 1024, 2)])
def test_model_file_round_trip(q, tmp_path, d, n_features, T):
    p, U, signs, T, b, sigma, lam, alpha = _model(d, n_features, T)
    path = tmp_path / "model.qmlr"
    q.save_model(path, p, U, signs, T, b, sigma, lam, alpha)
    m = q.load_model(path)
    assert m["params"] == p
    assert m["T"] == T and m["sigma"] == sigma and m["lam"] == lam
    assert np.array_equal(m["U"], U)
    assert np.array_equal(m["signs"], signs.astype(np.int8))
    assert np.array_equal(m["b"], b)
    assert np.array_equal(m["alpha"], alpha)          # FP64 weights kept exactly
    assert np.array_equal(q.pack_signs_host(m["signs"]), q.pack_signs_host(signs))


def _written(q, tmp_path):
    p, U, signs, T, b, sigma, lam, alpha = _model(32, 256, 3, seed=1)
    path = tmp_path / "m.qmlr"
    q.save_model(path, p, U, signs, T, b, sigma, lam, alpha)
    return path, path.read_bytes()


def test_model_file_rejects_a_flipped_byte(q, tmp_path):
    path, raw = _written(q, tmp_path)
    bad = bytearray(raw)
    bad[len(bad) // 2] ^= 0x01                       # one bit inside U
    path.write_bytes(bytes(bad))
    with pytest.raises(q.QMLRError, match="checksum"):
        q.load_model(path)


def test_model_file_rejects_truncation_and_bad_magic(q, tmp_path):
    path, raw = _written(q, tmp_path)
    path.write_bytes(raw[:-3])
    with pytest.raises(q.QMLRError, match="bytes"):
        q.load_model(path)
    path.write_bytes(raw[:100])
    with pytest.raises(q.QMLRError, match="truncated"):
        q.load_model(path)
    path.write_bytes(b"NOTAMODEL" + raw[9:])
    with pytest.raises(q.QMLRError, match="magic"):
        q.load_model(path)
    with pytest.raises(q.QMLRError, match="cannot open"):
        q.load_model(os.path.join(str(tmp_path), "missing.qmlr"))


def test_model_file_rejects_inconsistent_sizes_on_write(q, tmp_path):
    import ctypes
    p, U, signs, T, b, sigma, lam, alpha = _model(64, 512, 3)
    cp = q.c_params(p)
    L = q.lib()
    # N_F not a multiple of d
    rc = L.qmlr_model_file_write(str(tmp_path / "x").encode(), ctypes.byref(cp), 780, 64, 3, 500, 1.7, 1e-6,
                                 U.ctypes.data, q.pack_signs_host(signs).ctypes.data, b.ctypes.data,
                                 alpha.ctypes.data)
    assert rc == q.EINVAL
    assert b"bad model sizes" in L.qmlr_last_error()
    assert not (tmp_path / "x").exists()


@pytest.mark.parametrize("rep_dim,d,T", [(700, 64, 3), (781, 64, 3), (780, 48, 3), (780, 64, 5), (780, 256, 3)])
def test_model_file_write_rejects_what_a_model_cannot_hold(q, tmp_path, rep_dim, d, T):
    """rep_dim must be the one the FCHL19 parameters define, d a power of two in
    16..128 and T in 1..4 (what qmlr_model_create accepts)."""
    import ctypes
    p, U, signs, _, b, sigma, lam, alpha = _model(64, 512, 3)
    cp = q.c_params(p)
    L = q.lib()
    big = np.zeros(5 * 781 * 256, np.float32)            # large enough for any size asked above
    bits = np.zeros(512 * 5 * 8, np.uint32)
    rc = L.qmlr_model_file_write(str(tmp_path / "x").encode(), ctypes.byref(cp), rep_dim, d, T, 512, 1.7, 1e-6,
                                 big.ctypes.data, bits.ctypes.data, b.ctypes.data, alpha.ctypes.data)
    assert rc == q.EINVAL
    assert b"bad model sizes" in L.qmlr_last_error()
    assert not (tmp_path / "x").exists()


def _fnv1a64(data: bytes) -> int:
    h = 14695981039346656037
    for c in data:
        h = ((h ^ c) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def test_model_file_read_rejects_a_rep_dim_the_params_do_not_define(q, tmp_path):
    """A file whose checksum is valid but whose rep_dim disagrees with its FCHL19
    parameters is refused before any array is sized from it."""
    path, raw = _written(q, tmp_path)
    off = 8 + 4 + 4 + 4 * 4 + 7 * 8                       # rep_dim field after the FCHL19 parameters
    assert int.from_bytes(raw[off:off + 4], "little") == 780
    bad = bytearray(raw[:-8])
    bad[off:off + 4] = (700).to_bytes(4, "little")
    bad += _fnv1a64(bytes(bad)).to_bytes(8, "little")
    path.write_bytes(bytes(bad))
    with pytest.raises(q.QMLRError, match="inconsistent sizes"):
        q.load_model(path)
