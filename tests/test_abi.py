"""The C-ABI library loads and exports every entry point include/qmlr.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qmlr.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qmlr_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2206_01580_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared()
    for must in ("qmlr_fchl19", "qmlr_fchl19_vjp", "qmlr_project", "qmlr_sorf", "qmlr_sorf_grad"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2206_01580_gb300 import qmlr
    missing = [n for n in declared() if n not in qmlr.declared_symbols()]
    assert not missing, missing


def test_host_side_validation_without_gpu(lib):
    """Argument errors are caught on the host before any launch."""
    from paper_2206_01580_gb300 import qmlr
    L = qmlr.lib()
    cp = qmlr.c_params(qmlr.FCHL19Params())
    rd = ctypes.c_int32(0)
    assert L.qmlr_fchl19_rep_dim(ctypes.byref(cp), ctypes.byref(rd)) == 0
    assert rd.value == 780
    bad = qmlr.c_params(qmlr.FCHL19Params(nfourier=2))
    assert L.qmlr_fchl19_rep_dim(ctypes.byref(bad), ctypes.byref(rd)) == qmlr.EINVAL
    assert b"nfourier" in L.qmlr_last_error()
    # rep_ld smaller than rep_dim
    assert L.qmlr_fchl19(None, None, None, 0, 0, 16, ctypes.byref(cp), None, 10, None) == qmlr.EINVAL
    # SORF: d not supported
    assert L.qmlr_sorf(None, 48, None, 1, 1, None, 3, None, 96, 1.0, None, 0, None, None) == qmlr.EINVAL
    assert qmlr.sorf_parts(16384, 128) == 1 and qmlr.sorf_parts(32768, 128) == 2


def test_rff_validation_without_gpu(lib):
    """qmlr_rff rejects bad modes, feature widths and sigma before any launch."""
    from paper_2206_01580_gb300 import qmlr
    L = qmlr.lib()
    # energy mode is not offered by the dense map
    assert L.qmlr_rff(None, 64, None, 1, 1, None, None, 128, 1.0, qmlr.SORF_ENERGY, None, None) == qmlr.EINVAL
    assert b"mode" in L.qmlr_last_error()
    # d above the shared-memory slice of G
    assert L.qmlr_rff(None, 300, None, 1, 1, None, None, 128, 1.0, qmlr.SORF_PER_MOL, None, None) == qmlr.EINVAL
    assert b"d must be" in L.qmlr_last_error()
    # sigma must be positive
    assert L.qmlr_rff(None, 64, None, 1, 1, None, None, 128, 0.0, qmlr.SORF_PER_MOL, None, None) == qmlr.EINVAL
    # NULL buffers
    assert L.qmlr_rff(None, 64, None, 1, 1, None, None, 128, 1.0, qmlr.SORF_PER_MOL, None, None) == qmlr.EINVAL
    assert b"NULL" in L.qmlr_last_error()
