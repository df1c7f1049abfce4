"""Multi-vector SpMV (lilac_spmm): every column of Y against the FP64 oracle
SpMV of the same column of X, in both layouts, host and device."""
import numpy as np
import pytest

import oracle
from paper_2001_07938_gb300 import inputs
from paper_2001_07938_gb300 import lilac as L
from lilac_testutil import assert_spmv_close, dev, host, torch_cuda

pytestmark = pytest.mark.gpu


def _check(A, X, Y, k, fp32, what):
    for j in range(k):
        assert_spmv_close(A, X[:, j].astype(np.float64), Y[:, j], fp32, f"{what} column {j}")


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("k", [1, 3, 8, 17, 32])
def test_spmm_layouts_host_and_device(dtype, k):
    torch = torch_cuda()
    A = inputs.random_csr(3000, 2500, 40, 0.2, seed=k).astype(dtype)
    X = np.stack([inputs.uniform(100 + j, A.ncols, dtype=dtype) for j in range(k)], axis=1)
    M = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
    fp32 = dtype == np.float32
    # row-major on the device
    Xr = dev(np.ascontiguousarray(X))
    Yr = torch.full((A.n, k), float("nan"), dtype=Xr.dtype, device="cuda")
    M.spmm(Xr, Yr, k, L.LILAC_LAYOUT_ROWS)
    torch.cuda.synchronize()
    _check(A, X, host(Yr), k, fp32, "rows/device")
    # vector-major (k separate vectors) on the host
    Xv = np.ascontiguousarray(X.T)
    Yv = np.full((k, A.n), np.nan, dtype)
    M.spmm(Xv, Yv, k, L.LILAC_LAYOUT_VECTORS)
    _check(A, X, Yv.T, k, fp32, "vectors/host")
    M.close()


def test_spmm_long_rows_and_errors():
    torch_cuda()
    A = inputs.powerlaw_csr(2000, 3000, 30000, power=8, seed=3)
    k = 5
    X = np.stack([inputs.uniform(7 + j, A.ncols) for j in range(k)], axis=1)
    M = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
    Y = np.zeros((A.n, k))
    M.spmm(np.ascontiguousarray(X), Y, k)
    _check(A, X, Y, k, False, "power-law")
    for bad in (0, 33):
        with pytest.raises(L.LilacError):
            M.spmm(np.ascontiguousarray(X), Y, bad)
    M.close()
