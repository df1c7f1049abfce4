"""GPU conjugate gradient (lilac_cg through the C ABI) against the FP64 oracle.

The GPU and the oracle reduce in different orders, so their CG iterates
differ at rounding level; the GPU result is checked by its own true residual
||b - A x|| / ||b|| computed by the oracle's SpMV (tolerance 1e-10), by the
iteration count against the oracle's, and by the distance to the oracle's
solution on well-conditioned systems.
"""
import numpy as np
import pytest

import oracle
from paper_2001_07938_gb300 import inputs
from paper_2001_07938_gb300 import lilac as L
from lilac_testutil import dev, host, torch_cuda, true_rel_residual

pytestmark = pytest.mark.gpu


def _solve(A, b, dtype=np.float64, **kw):
    torch = torch_cuda()
    M = L.CsrMatrix.from_csr(A.astype(dtype) if dtype != A.vals.dtype else A)
    bd = dev(b)
    xd = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    if kw.get("use_x0"):
        xd.copy_(dev(kw.pop("x0")))
    st, info = M.cg(bd, xd, **kw)
    torch.cuda.synchronize()
    x = host(xd)
    M.close()
    return st, info, x


@pytest.mark.parametrize("variant", [None, (1, 1), (2, 8), (3, 4), (4, 1), (7, 1)])
def test_small_spd_converges_like_the_oracle(variant):
    A = inputs.spd_random(3000, 12, 20.0, 4)
    b = inputs.uniform(5, A.n)
    torch = torch_cuda()
    M = L.CsrMatrix.from_csr(A)
    if variant:
        M.set_variant(*variant)
    bd, xd = dev(b), torch.zeros(A.n, dtype=torch.float64, device="cuda")
    st, info = M.cg(bd, xd, rtol=1e-10, max_iter=500)
    torch.cuda.synchronize()
    x = host(xd)
    M.close()
    xr, itr, str_ = oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=500, rtol=1e-10)
    assert st == L.LILAC_OK and info.status == L.LILAC_OK
    assert abs(info.iters - itr) <= 1
    assert true_rel_residual(A, b, x) <= 1e-10
    assert info.true_rel_res <= 1e-10
    assert np.linalg.norm(x - xr) <= 1e-9 * np.linalg.norm(xr)


def test_sell_split_epilogue_cg_matches_single_pass():
    """SELL with the p.q reduction in a row-order pass (many short sorted
    rows) converges like the oracle and, run twice, bitwise alike."""
    A = inputs.spd_random(70000, 10, 20.0, 6)
    b = inputs.uniform(7, A.n)
    torch = torch_cuda()
    M = L.CsrMatrix.from_csr(A)
    M.set_variant(L.LILAC_VARIANT_SELL, 1)
    info = M.info()
    assert info["active_variant"] == L.LILAC_VARIANT_SELL and info["spmv_kernels"] == 2
    xs = []
    for _ in range(2):
        bd, xd = dev(b), torch.zeros(A.n, dtype=torch.float64, device="cuda")
        st, inf = M.cg(bd, xd, rtol=1e-10, max_iter=500)
        torch.cuda.synchronize()
        assert st == L.LILAC_OK
        xs.append(host(xd))
    M.close()
    np.testing.assert_array_equal(xs[0], xs[1])
    _, itr, _ = oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=500, rtol=1e-10)
    assert abs(inf.iters - itr) <= 1
    assert true_rel_residual(A, b, xs[0]) <= 1e-10


@pytest.mark.parametrize("variant", [5, 7])
def test_slab_and_sell_cg_converge_and_repeat_bitwise(variant):
    """SLAB (the last CTA of each row group combines the slabs; its p.q sums
    go to the group's slot) and SELL: CG as the oracle, bitwise run to run."""
    A = inputs.spd_random(20000, 30, 20.0, 8)
    b = inputs.uniform(9, A.n)
    torch = torch_cuda()
    M = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
    M.set_variant(variant, 4)
    assert M.info()["active_variant"] == variant
    xs = []
    for _ in range(2):
        bd, xd = dev(b), torch.zeros(A.n, dtype=torch.float64, device="cuda")
        st, inf = M.cg(bd, xd, rtol=1e-10, max_iter=500)
        torch.cuda.synchronize()
        assert st == L.LILAC_OK
        xs.append(host(xd))
    M.close()
    np.testing.assert_array_equal(xs[0], xs[1])
    xr, itr, _ = oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=500, rtol=1e-10)
    assert abs(inf.iters - itr) <= 1
    assert true_rel_residual(A, b, xs[0]) <= 1e-10
    assert np.linalg.norm(xs[0] - xr) <= 1e-9 * np.linalg.norm(xr)


def test_laplacian_converges_and_eigenmode_in_one_step():
    A = inputs.laplacian2d(40)
    b = np.ones(A.n)
    st, info, x = _solve(A, b, rtol=1e-10, max_iter=2000)
    _, itr, _ = oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=2000, rtol=1e-10)
    assert st == L.LILAC_OK and abs(info.iters - itr) <= 2
    assert true_rel_residual(A, b, x) <= 1e-10
    m = 40
    a = np.arange(1, m + 1)
    v = np.outer(np.sin(3 * np.pi * a / (m + 1)), np.sin(5 * np.pi * a / (m + 1))).ravel()
    lam = 4 - 2 * np.cos(3 * np.pi / (m + 1)) - 2 * np.cos(5 * np.pi / (m + 1))
    st, info, x = _solve(A, v, rtol=1e-10, max_iter=10)
    assert info.iters == 1
    np.testing.assert_allclose(x, v / lam, rtol=0, atol=1e-12 * np.abs(v / lam).max())


def test_fixed_iterations_graph_equals_eager_bitwise():
    """Same handle (same kernel choice): the captured graph and eager launches
    give bitwise-identical iterates (every reduction order is fixed)."""
    torch = torch_cuda()
    A = inputs.spd_random(5000, 20, 20.0, 2)
    b = np.ones(A.n)
    M = L.CsrMatrix.from_csr(A)
    bd = dev(b)
    xs = []
    for use_graph in (True, False, True):
        xd = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        st, info = M.cg(bd, xd, rtol=0.0, max_iter=40, use_graph=use_graph)
        assert st == L.LILAC_OK and info.iters == 40
        xs.append(host(xd))
    M.close()
    np.testing.assert_array_equal(xs[0], xs[1])
    np.testing.assert_array_equal(xs[0], xs[2])
    assert true_rel_residual(A, b, xs[0]) <= 1e-10


def test_breakdown_zero_rhs_not_converged_and_x0():
    # indefinite: p.Ap = 0 at the first step
    A = inputs.CSR(2, 2, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32),
                   np.array([1.0, -1.0]))
    st, info, _ = _solve(A, np.array([1.0, 1.0]), rtol=1e-12, max_iter=5)
    assert st == L.LILAC_ERR_BREAKDOWN and info.status == L.LILAC_ERR_BREAKDOWN
    B = inputs.laplacian2d(10)
    st, info, x = _solve(B, np.zeros(B.n), rtol=1e-10, max_iter=10)
    assert st == L.LILAC_OK and info.iters == 0 and not np.any(x)
    st, info, _ = _solve(B, np.ones(B.n), rtol=1e-14, max_iter=3)
    assert st == L.LILAC_ERR_NOT_CONVERGED and info.iters == 3
    # restart from the oracle's iterate after 20 steps
    xr, _, _ = oracle.cg(B.row_ptr, B.col_ind, B.vals, np.ones(B.n), max_iter=20, rtol=0.0)
    st, info, x = _solve(B, np.ones(B.n), rtol=1e-10, max_iter=500, use_x0=True, x0=xr)
    assert st == L.LILAC_OK
    assert true_rel_residual(B, np.ones(B.n), x) <= 1e-10


def test_host_buffers_match_device_buffers():
    torch = torch_cuda()
    A = inputs.spd_random(4000, 15, 20.0, 9)
    b = inputs.uniform(10, A.n)
    M = L.CsrMatrix.from_csr(A)
    xdev = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    st, info = M.cg(dev(b), xdev, rtol=1e-10, max_iter=300)
    xd = host(xdev)
    xh = np.zeros(A.n)
    st2, info2 = M.cg(b, xh, rtol=1e-10, max_iter=300)
    M.close()
    assert st2 == L.LILAC_OK and info2.iters == info.iters
    np.testing.assert_array_equal(xh, xd)


@pytest.mark.slow
def test_full_spd_75k_75_iterations():
    """The benchmark workload: random SPD n=75,000 (~181 nnz/row), b = 1, 75 iterations."""
    A, b = inputs.workload_spd_cg()
    st, info, x = _solve(A, b, rtol=0.0, max_iter=75)
    assert st == L.LILAC_OK and info.iters == 75
    assert true_rel_residual(A, b, x) <= 1e-10
    xr, itr, _ = oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=75, rtol=0.0)
    assert np.linalg.norm(x - xr) <= 1e-10 * np.linalg.norm(xr)
