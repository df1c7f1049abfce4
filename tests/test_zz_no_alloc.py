"""lilac_spmv_noalloc, the entry point for callers that must not allocate
device memory (e.g. because another component owns the device memory through
its own pool, or because cudaMalloc / cudaFree may synchronise the device in a
latency-critical loop), gives the same y as lilac_spmv on a handle.

Both results carry the componentwise SpMV rounding bound of the other tests
(tests/lilac_testutil.py), so they agree to twice that bound.  Two calls in a
row check that the shared scratch array is left ready for the next call.
This file is collected last on purpose, and passes alone or after the rest.
"""
import ctypes

import numpy as np
import pytest

from paper_2001_07938_gb300 import inputs
from paper_2001_07938_gb300 import lilac as L
from lilac_testutil import dev, host, spmv_tolerance, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_noalloc_matches_lilac_spmv_on_two_calls(dtype):
    torch = torch_cuda()
    # rows longer than a CTA range (carries), empty rows, unsorted duplicates
    A = inputs.powerlaw_csr(20_000, 30_000, 60_000, power=8, seed=11).astype(dtype)
    x_np = inputs.uniform(12, A.ncols, dtype=dtype)
    rp, ci, va, x = dev(A.row_ptr), dev(A.col_ind), dev(A.vals), dev(x_np)
    code = L.LILAC_F64 if dtype == np.float64 else L.LILAC_F32
    M = L.CsrMatrix.from_csr(A)
    y_ref = torch.empty(A.n, dtype=x.dtype, device="cuda")
    M.spmv(x, y_ref)
    torch.cuda.synchronize()
    M.close()
    ref = host(y_ref).astype(np.float64)
    tol = 2.0 * spmv_tolerance(A, x_np.astype(np.float64), dtype == np.float32)
    for _ in range(2):
        y = torch.full((A.n,), float("nan"), dtype=x.dtype, device="cuda")
        L.lilac_spmv_noalloc(A.n, A.ncols, A.nnz, rp.data_ptr(), ci.data_ptr(), va.data_ptr(),
                             code, x.data_ptr(), y.data_ptr())
        torch.cuda.synchronize()
        err = np.abs(host(y).astype(np.float64) - ref)
        assert np.all(err <= tol), (np.nonzero(err > tol)[0][:5], err.max())


def test_noalloc_rejects_sizes_beyond_its_limit():
    lib = L.load()
    # rows + nnz must stay below 2^31: refused on the host, before any GPU work
    assert lib.lilac_spmv_noalloc(2 ** 30, 10, 2 ** 30, 1, 1, 1, L.LILAC_F64, 1, 1,
                                  None) == L.LILAC_ERR_INVALID_ARG
    assert "2^31" in L.lilac_last_error()
