"""The element grouping entry point that allocates nothing, called through the
C ABI, gives the same permutation and offsets as the workspace version.

Callers that cannot allocate device memory when they group atoms (a framework
that owns all device memory through its own pool, a service that must not wait
on the allocator in its request path) use qmlr_group_by_element_noalloc; it
keeps its scratch in a fixed array inside the library. This file is collected
last so that a failure here does not hide the other tests' results.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_01580_gb300 import qmlr
    qmlr.lib()
    return qmlr


def _noalloc(q, elem, n_el):
    e = torch.as_tensor(elem, dtype=torch.int32).cuda()
    n = e.shape[0]
    perm = torch.full((max(n, 1),), -7, device="cuda", dtype=torch.int32)
    offs = torch.full((n_el + 1,), -7, device="cuda", dtype=torch.int32)
    rc = q.lib().qmlr_group_by_element_noalloc(C.c_void_p(e.data_ptr()), n, n_el, C.c_void_p(perm.data_ptr()),
                                               C.c_void_p(offs.data_ptr()), q._stream())
    assert rc == 0, q.lib().qmlr_last_error()
    return perm[:n].cpu().numpy(), offs.cpu().numpy()


def test_noalloc_grouping_matches_workspace_version_twice(q):
    rng = np.random.default_rng(123)
    # two calls in a row with different inputs: the second must not see the first's scratch
    for n, n_el in ((300_000, 5), (2_049, 3)):
        elem = rng.integers(0, n_el, size=n).astype(np.int32)
        perm_ref, offs_ref = q.group_by_element(elem, n_el)
        perm, offs = _noalloc(q, elem, n_el)
        assert np.array_equal(perm, perm_ref.cpu().numpy())
        assert np.array_equal(offs, offs_ref.cpu().numpy())
    assert q.device_status() == 0


def test_noalloc_grouping_rejects_oversize_input(q):
    n = 4194304 + 1
    rc = q.lib().qmlr_group_by_element_noalloc(None, n, 5, None, None, None)
    assert rc == q.EINVAL
    assert b"QMLR_GROUP_NOALLOC_MAX_ATOMS" in q.lib().qmlr_last_error()
