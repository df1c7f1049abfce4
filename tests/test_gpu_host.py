"""Host-convention SpMV (lilac_spmv_host): the paper's harness calling
convention with library-side marshaling and explicit change tracking."""
import numpy as np
import pytest

from paper_2001_07938_gb300 import inputs
from paper_2001_07938_gb300 import lilac as L
from lilac_testutil import assert_spmv_close, torch_cuda

pytestmark = pytest.mark.gpu


def _fresh():
    torch_cuda()
    L.lilac_host_cache_clear()


def test_cached_uploads_once_and_tracks_value_and_structure_changes():
    _fresh()
    A = inputs.random_csr(3000, 2000, 20, 0.1, seed=2)
    x = inputs.uniform(3, A.ncols)
    y = np.zeros(A.n)
    for _ in range(3):
        L.spmv_host(A, x, y)
        assert_spmv_close(A, x, y, False, "cached")
    st = L.lilac_host_cache_stats()
    assert st["uploads"] == 1 and st["hits"] == 2 and st["resident"] == 1
    # values changed in place (same pointers): found by the content hash
    A.vals[:] = inputs.uniform(4, A.nnz)
    L.spmv_host(A, x, y)
    assert_spmv_close(A, x, y, False, "after value change")
    assert L.lilac_host_cache_stats()["value_updates"] == 1
    # structure changed in place: the resident copy is rebuilt
    A.col_ind[:] = A.col_ind[::-1].copy()
    L.spmv_host(A, x, y)
    assert_spmv_close(A, x, y, False, "after structure change")
    st = L.lilac_host_cache_stats()
    assert st["structure_changes"] == 1 and st["uploads"] == 2
    L.lilac_host_cache_clear()
    assert L.lilac_host_cache_stats()["resident"] == 0


def test_version_numbers_skip_the_hash():
    _fresh()
    A = inputs.laplacian2d(40)
    x = inputs.uniform(5, A.ncols)
    y = np.zeros(A.n)
    L.spmv_host(A, x, y, version=7)
    assert_spmv_close(A, x, y, False, "v7")
    old = A.vals.copy()
    A.vals *= 2.0
    # same version number: the caller promises nothing changed (no host pass)
    L.spmv_host(A, x, y, version=7)
    B = inputs.CSR(A.n, A.ncols, A.row_ptr, A.col_ind, old)
    assert_spmv_close(B, x, y, False, "v7 stale by contract")
    L.spmv_host(A, x, y, version=8)
    assert_spmv_close(A, x, y, False, "v8")
    st = L.lilac_host_cache_stats()
    one_pass = (A.n + 1 + A.nnz) * 4 + A.nnz * 8
    # hashed at the upload and at the new number only, never on the repeat
    assert st["hashed_bytes"] == 2 * one_pass
    assert st["value_updates"] == 1 and st["hits"] == 1 and st["uploads"] == 1


def test_naive_mode_and_fp32():
    _fresh()
    A = inputs.banded_spd(5000, 8, 1.0, seed=1).astype(np.float32)
    x = inputs.uniform(6, A.ncols, dtype=np.float32)
    y = np.zeros(A.n, np.float32)
    for _ in range(2):
        L.spmv_host(A, x, y, naive=True)
        assert_spmv_close(A, x.astype(np.float64), y, True, "naive fp32")
    st = L.lilac_host_cache_stats()
    assert st["uploads"] == 2 and st["resident"] == 0
    L.spmv_host(A, x, y)
    assert_spmv_close(A, x.astype(np.float64), y, True, "cached fp32")
    with pytest.raises(L.LilacError):
        L.lilac_spmv_host(A.n, A.ncols, A.nnz, A.row_ptr.ctypes.data, A.col_ind.ctypes.data,
                          A.vals.ctypes.data, L.LILAC_F32, x.ctypes.data, y.ctypes.data, 0, 9)
    L.lilac_host_cache_clear()
