"""lilac_spmv_noalloc, the entry point for callers that must not allocate
device memory (e.g. because another component owns the device memory through
its own pool, or because cudaMalloc / cudaFree may synchronise the device in a
latency-critical loop), gives the same y as lilac_spmv on a handle and as the
FP64 oracle.

Against the oracle, y carries the componentwise SpMV rounding bound of the
other tests (tests/lilac_testutil.py); against lilac_spmv, whose result has
the same bound, twice that bound.  Two calls in a row check that the shared
scratch array is left ready for the next call; the device's free memory and
an armed allocation-failure hook show that the calls allocate nothing.  This
file is collected last on purpose, and passes alone or after the rest.
"""
import numpy as np
import pytest

import oracle
from paper_2001_07938_gb300 import inputs
from paper_2001_07938_gb300 import lilac as L
from lilac_testutil import dev, host, spmv_tolerance, torch_cuda

pytestmark = pytest.mark.gpu


def _noalloc(A, rp, ci, va, x, y, code):
    L.lilac_spmv_noalloc(A.n, A.ncols, A.nnz, rp, ci, va, code, x, y)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_noalloc_matches_lilac_spmv_and_the_oracle_on_two_calls(dtype):
    torch = torch_cuda()
    fp32 = dtype == np.float32
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
    x64 = x_np.astype(np.float64)
    yo = oracle.spmv(A.row_ptr, A.col_ind, A.vals, x64)
    tol = spmv_tolerance(A, x64, fp32)
    ys = [torch.full((A.n,), float("nan"), dtype=x.dtype, device="cuda") for _ in range(2)]
    # the first call on the device may load the library's module; the
    # following ones must leave the device's free memory as it is
    _noalloc(A, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), x.data_ptr(), ys[0].data_ptr(), code)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    L.lilac_debug_inject(None, L.LILAC_INJECT_ALLOC_FAIL, 1)  # the next library allocation fails
    try:
        _noalloc(A, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), x.data_ptr(), ys[1].data_ptr(),
                 code)
        torch.cuda.synchronize()
        # still armed: the hook was not consumed by the call above
        with pytest.raises(L.LilacError) as e:
            L.CsrMatrix.from_csr(inputs.laplacian2d(4))
        assert e.value.status == L.LILAC_ERR_OOM
    finally:
        L.lilac_debug_inject(None, L.LILAC_INJECT_ALLOC_FAIL, 0)
    assert torch.cuda.mem_get_info()[0] == free_before
    for y in ys:
        yh = host(y).astype(np.float64)
        err_ref = np.abs(yh - ref)
        assert np.all(err_ref <= 2.0 * tol), (np.nonzero(err_ref > 2.0 * tol)[0][:5], err_ref.max())
        err_or = np.abs(yh - yo)
        assert np.all(err_or <= tol), (np.nonzero(err_or > tol)[0][:5], err_or.max())


def test_noalloc_degenerate_shapes_match_the_oracle():
    """nnz = 0 (x may be NULL) and a matrix whose rows are all empty give
    y = 0; one nonempty row among many empty ones gives its dot product."""
    torch = torch_cuda()
    n = 5000
    rp = dev(np.zeros(n + 1, np.int32))
    y = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    L.lilac_spmv_noalloc(n, 7, 0, rp.data_ptr(), None, None, L.LILAC_F64, None, y.data_ptr())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(y), np.zeros(n))
    row_ptr = np.zeros(n + 1, np.int32)
    row_ptr[4001:] = 300  # row 4000 holds 300 nonzeros, all others none
    col = np.arange(300, dtype=np.int32) * 3
    val = inputs.uniform(31, 300)
    A = inputs.CSR(n, 900, row_ptr, col, val)
    xv = inputs.uniform(32, 900)
    d = [dev(a) for a in (A.row_ptr, A.col_ind, A.vals, xv)]
    y2 = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        L.lilac_spmv_noalloc(n, 900, 300, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(),
                             L.LILAC_F64, d[3].data_ptr(), y2.data_ptr())
        torch.cuda.synchronize()
        ref = oracle.spmv(A.row_ptr, A.col_ind, A.vals, xv)
        tol = spmv_tolerance(A, xv, False)
        assert np.all(np.abs(host(y2) - ref) <= tol)


def test_noalloc_rejects_sizes_beyond_its_limit():
    lib = L.load()
    # rows + nnz must stay below 2^31: refused on the host, before any GPU work
    assert lib.lilac_spmv_noalloc(2 ** 30, 10, 2 ** 30, 1, 1, 1, L.LILAC_F64, 1, 1,
                                  None) == L.LILAC_ERR_INVALID_ARG
    assert "2^31" in L.lilac_last_error()
