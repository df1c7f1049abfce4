"""GPU BFS (lilac_bfs through the C ABI) against the oracle's queue BFS.

The handle holds the transposed adjacency (row v = in-neighbours of v); the
oracle walks out-neighbour lists, so it gets the plain transpose of the same
graph.  BFS levels are unique: the comparison is bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_2001_07938_gb300 import inputs
from paper_2001_07938_gb300 import lilac as L
from lilac_testutil import dev, host, torch_cuda

pytestmark = pytest.mark.gpu


def _transpose(A):
    """Plain CSR transpose (row j of the result lists the rows i with A_ij)."""
    n = A.n
    rows = np.repeat(np.arange(n, dtype=np.int32), np.diff(A.row_ptr))
    order = np.argsort(A.col_ind, kind="stable")
    col = rows[order]
    rp = np.zeros(A.ncols + 1, np.int64)
    np.cumsum(np.bincount(A.col_ind, minlength=A.ncols), out=rp[1:])
    return rp.astype(np.int32), col.astype(np.int32)


def _gpu_levels(M, source, on_device=True):
    torch = torch_cuda()
    if on_device:
        lv = torch.full((M.rows,), -7, dtype=torch.int32, device="cuda")
        depth = M.bfs(source, lv)
        torch.cuda.synchronize()
        return host(lv), depth
    lv = np.full(M.rows, -7, np.int32)
    depth = M.bfs(source, lv)
    return lv, depth


def test_rmat_graph_levels_bit_exact():
    AT = inputs.rmat_transposed(12, 16, 0.57, 0.19, 0.19, seed=4, permute=True)
    rp_out, col_out = _transpose(AT)
    M = L.CsrMatrix.from_csr(AT, flags=L.LILAC_CREATE_NO_TUNE)
    outdeg = np.diff(rp_out)
    for src in (0, int(np.argmax(outdeg)), int(np.argmin(outdeg)), AT.n - 1):
        ref = oracle.bfs_levels(rp_out, col_out, src)
        lv, depth = _gpu_levels(M, src)
        assert np.array_equal(lv, ref), src
        assert depth == int(ref.max()) + 1
        lh, dh = _gpu_levels(M, src, on_device=False)
        assert np.array_equal(lh, ref) and dh == depth
    M.close()


def test_directed_path_deeper_than_a_graph_chunk():
    n = 100
    # edges i -> i+1; transposed: row v lists v - 1
    rp = np.concatenate([[0], np.arange(n)]).astype(np.int32)
    col = np.arange(n - 1, dtype=np.int32)
    AT = inputs.CSR(n, n, rp, col, np.ones(n - 1))
    M = L.CsrMatrix.from_csr(AT, flags=L.LILAC_CREATE_NO_TUNE)
    lv, depth = _gpu_levels(M, 0)
    assert lv.tolist() == list(range(n)) and depth == n
    lv, depth = _gpu_levels(M, 50)
    assert lv.tolist() == [-1] * 50 + list(range(50)) and depth == 50
    M.close()


def test_edgeless_graph_and_errors():
    n = 10
    AT = inputs.CSR(n, n, np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    M = L.CsrMatrix(AT.row_ptr, AT.col_ind, AT.vals, ncols=n, flags=L.LILAC_CREATE_NO_TUNE)
    lv, depth = _gpu_levels(M, 3)
    assert lv.tolist() == [-1, -1, -1, 0, -1, -1, -1, -1, -1, -1] and depth == 1
    with pytest.raises(L.LilacError):
        M.bfs(n, np.zeros(n, np.int32))
    with pytest.raises(L.LilacError):
        M.bfs(-1, np.zeros(n, np.int32))
    M.close()
    R = L.CsrMatrix(np.array([0, 1, 2], np.int32), np.array([0, 2], np.int32), np.ones(2),
                    flags=L.LILAC_CREATE_NO_TUNE)
    with pytest.raises(L.LilacError):
        R.bfs(0, np.zeros(2, np.int32))  # 2 x 3: not square
    R.close()


@pytest.mark.slow
def test_full_rmat22_levels_bit_exact():
    AT = inputs.workload_rmat_pagerank()
    rp_out, col_out = _transpose(AT)
    M = L.CsrMatrix.from_csr(AT)
    src = int(np.argmax(np.diff(rp_out)))
    ref = oracle.bfs_levels(rp_out, col_out, src)
    lv, depth = _gpu_levels(M, src)
    assert np.array_equal(lv, ref)
    assert depth == int(ref.max()) + 1
    M.close()
