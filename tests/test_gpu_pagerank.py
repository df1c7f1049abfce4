"""GPU PageRank (lilac_pagerank through the C ABI) against the FP64 oracle.

FP32 PageRank: ||x_gpu - x_oracle||_1 <= 1e-5 after the same iterations,
per-iteration L1 changes alike, mass close to 1; FP64 PageRank to 1e-12.
"""
import numpy as np
import pytest

import oracle
from paper_2001_07938_gb300 import inputs
from paper_2001_07938_gb300 import lilac as L
from lilac_testutil import ALL_VARIANTS, dev, host, torch_cuda

pytestmark = pytest.mark.gpu


def _pr(A, iters=20, d=0.85, dtype=np.float32, variant=None, x0=None):
    torch = torch_cuda()
    M = L.CsrMatrix.from_csr(A.astype(dtype))
    if variant:
        M.set_variant(*variant)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    x = torch.empty(A.n, dtype=tdt, device="cuda") if x0 is None else dev(x0.astype(dtype))
    l1 = M.pagerank(x, iters=iters, damping=d, init_uniform=x0 is None)
    torch.cuda.synchronize()
    out = host(x)
    M.close()
    return out, l1


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_small_rmat_fp32_all_variants(variant):
    A = inputs.rmat_transposed(11, 8, seed=2)
    xr, l1r = oracle.pagerank(A.row_ptr, A.col_ind, A.vals, iters=20)
    x, l1 = _pr(A, variant=variant)
    assert np.abs(x.astype(np.float64) - xr).sum() <= 1e-5
    np.testing.assert_allclose(l1, l1r, rtol=1e-4, atol=1e-6)
    assert abs(x.astype(np.float64).sum() - xr.sum()) <= 1e-5


def test_sell_split_epilogue_on_many_sorted_rows():
    """SELL on a graph with many short rows sorted by length stores the rows
    in one kernel and takes the L1 / dangling sums in a row-order pass."""
    A = inputs.rmat_transposed(17, 8, seed=5)
    xr, l1r = oracle.pagerank(A.row_ptr, A.col_ind, A.vals, iters=20)
    torch = torch_cuda()
    M = L.CsrMatrix.from_csr(A)
    M.set_variant(L.LILAC_VARIANT_SELL, 1)
    info = M.info()
    assert info["active_variant"] == L.LILAC_VARIANT_SELL and info["spmv_kernels"] == 2
    assert info["sell_split_rows"] > 0
    x = torch.empty(A.n, dtype=torch.float32, device="cuda")
    l1 = M.pagerank(x, iters=20)
    torch.cuda.synchronize()
    x = host(x).astype(np.float64)
    M.close()
    assert np.abs(x - xr).sum() <= 1e-5
    np.testing.assert_allclose(l1, l1r, rtol=1e-4, atol=1e-6)


@pytest.mark.parametrize("permute", [True, False])
def test_hub_pagerank_matches_oracle_and_repeats(permute):
    """PageRank on the HUB copies (hub gather, slab pieces, cold sliced ELL
    adding the slab sums, row-order reduction), relabelled and unpermuted
    R-MAT: within the FP32 tolerance of the oracle, bitwise run to run."""
    torch = torch_cuda()
    A = inputs.rmat_transposed(19, 8, seed=6, permute=permute)
    xr, l1r = oracle.pagerank(A.row_ptr, A.col_ind, A.vals, iters=20)
    M = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
    M.set_variant(L.LILAC_VARIANT_HUB, 1)
    assert M.info()["active_variant"] == L.LILAC_VARIANT_HUB
    xs = []
    for _ in range(2):
        x = torch.empty(A.n, dtype=torch.float32, device="cuda")
        l1 = M.pagerank(x, iters=20)
        torch.cuda.synchronize()
        xs.append(host(x))
    M.close()
    np.testing.assert_array_equal(xs[0], xs[1])
    assert np.abs(xs[0].astype(np.float64) - xr).sum() <= 1e-5
    np.testing.assert_allclose(l1, l1r, rtol=1e-4, atol=1e-6)


def test_fp64_pagerank_matches_oracle_tightly():
    A = inputs.rmat_transposed(12, 8, seed=4)
    xr, l1r = oracle.pagerank(A.row_ptr, A.col_ind, A.vals.astype(np.float64), iters=30)
    x, l1 = _pr(A, iters=30, dtype=np.float64)
    assert np.abs(x - xr).sum() <= 1e-12
    # each |y_i - x_i| carries the iterate's rounding (~ t eps x_i after t
    # iterations), so the L1 changes agree to ~ t eps sum(x) in absolute terms
    np.testing.assert_allclose(l1, l1r, rtol=1e-9, atol=30 * 2.3e-16)


def test_cycle_uniform_edgeless_and_start_vector():
    N = 1000
    rp = np.arange(N + 1, dtype=np.int32)
    ci = ((np.arange(N) - 1) % N).astype(np.int32)  # edge i-1 -> i
    A = inputs.CSR(N, N, rp, ci, np.ones(N, np.float32))
    x, l1 = _pr(A, iters=5)
    np.testing.assert_allclose(x, 1.0 / N, rtol=1e-6)
    E = inputs.CSR(N, N, np.zeros(N + 1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32))
    x0 = inputs.uniform(3, N, 0.0, 1.0)
    x0 /= x0.sum()
    x, _ = _pr(E, iters=1, x0=x0)
    np.testing.assert_allclose(x, 1.0 / N, rtol=1e-6)
    A2 = inputs.rmat_transposed(10, 6, seed=9)
    x02 = inputs.uniform(4, A2.n, 0.0, 1.0)
    x02 /= x02.sum()
    xr, _ = oracle.pagerank(A2.row_ptr, A2.col_ind, A2.vals, iters=7, x0=x02)
    x, _ = _pr(A2, iters=7, x0=x02)
    assert np.abs(x - xr).sum() <= 1e-5


def test_host_vector_mode_and_odd_iterations():
    A = inputs.rmat_transposed(10, 8, seed=1)
    M = L.CsrMatrix.from_csr(A)
    xh = np.zeros(A.n, np.float32)
    l1 = M.pagerank(xh, iters=7)
    M.close()
    xr, l1r = oracle.pagerank(A.row_ptr, A.col_ind, A.vals, iters=7)
    assert np.abs(xh - xr).sum() <= 1e-5
    np.testing.assert_allclose(l1, l1r, rtol=1e-4, atol=1e-7)


@pytest.mark.slow
def test_full_rmat22_20_iterations():
    """The PageRank workload: R-MAT scale 22 (4,194,304 vertices, ~65M edges), FP32, 20 iterations."""
    A = inputs.workload_rmat_pagerank()
    x, l1 = _pr(A, iters=20)
    xr, l1r = oracle.pagerank(A.row_ptr, A.col_ind, A.vals, iters=20)
    assert np.abs(x.astype(np.float64) - xr).sum() <= 1e-5
    np.testing.assert_allclose(l1, l1r, rtol=1e-3, atol=1e-6)
