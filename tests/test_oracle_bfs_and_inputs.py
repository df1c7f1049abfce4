"""Pins of the oracle's BFS levels and of the shared input generators."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

import oracle
from paper_2001_07938_gb300 import inputs


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bfs_levels_vs_scipy_shortest_path(seed):
    A = inputs.random_csr(300, 300, 4, 0.3, seed)
    lev = oracle.bfs_levels(A.row_ptr, A.col_ind, 0)
    G = sp.csr_matrix((np.ones(A.nnz), A.col_ind, A.row_ptr), shape=(300, 300))
    d = shortest_path(G, unweighted=True, indices=0, directed=True)
    ref = np.where(np.isinf(d), -1, d).astype(np.int64)
    np.testing.assert_array_equal(lev, ref)


def test_splitmix64_known_answers():
    # Published outputs of SplitMix64 started from state 0.
    assert inputs.splitmix64_at(0, 0) == 0xE220A8397B1DCDAF
    assert inputs.splitmix64_at(0, 1) == 0x6E789E6AA1B965F4
    assert inputs.splitmix64_at(0, 2) == 0x06C45D188009454F


def test_uniform_range_and_determinism():
    x = inputs.uniform(0, 4096)
    assert np.all(x >= -1.0) and np.all(x < 1.0)
    np.testing.assert_array_equal(x, inputs.uniform(0, 4096))
    assert x[0] == 2.0 * ((0xE220A8397B1DCDAF >> 11) * 2.0 ** -53) - 1.0


def test_spd_random_structure():
    A = inputs.spd_random(500, 10, 20.0, 1)
    rp, ci, v = A.row_ptr, A.col_ind, A.vals
    D = sp.csr_matrix((v, ci, rp), shape=(500, 500)).toarray()
    np.testing.assert_array_equal(D, D.T)
    off = D - np.diag(np.diag(D))
    np.testing.assert_allclose(np.diag(D), off.sum(1) + 20.0, rtol=1e-14)
    assert np.all(np.linalg.eigvalsh(D) > 0)
    for i in range(500):
        assert np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0)


def test_banded_structure_and_fp32_exact():
    A = inputs.banded_spd(100, 5, 1.0, 2, fp32_exact=True)
    D = sp.csr_matrix((A.vals, A.col_ind, A.row_ptr), shape=(100, 100)).toarray()
    np.testing.assert_array_equal(D, D.T)
    off = D - np.diag(np.diag(D))
    assert np.all(off[np.abs(np.subtract.outer(np.arange(100), np.arange(100))) > 5] == 0)
    offv = off[off != 0]
    np.testing.assert_array_equal(offv.astype(np.float32).astype(np.float64), offv)


def test_all_cores_oracle_is_bitwise_the_sequential_one():
    """The OpenMP build (timed by the benchmark on all host cores) shares only
    the rows of an SpMV among threads, each row still summed alone in
    ascending order: SpMV, CG and PageRank results are bitwise those of the
    sequential build."""
    import pytest
    if oracle.build_parallel() is None:
        pytest.skip("no OpenMP in the host compiler")
    A = inputs.spd_random(3000, 20, 20.0, 3)
    x = inputs.uniform(4, A.n)
    np.testing.assert_array_equal(oracle.spmv(A.row_ptr, A.col_ind, A.vals, x),
                                  oracle.spmv(A.row_ptr, A.col_ind, A.vals, x, parallel=True))
    b = inputs.uniform(5, A.n)
    xs, its, _ = oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=30)
    xp, itp, _ = oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=30, parallel=True)
    assert its == itp
    np.testing.assert_array_equal(xs, xp)
    G = inputs.rmat_transposed(12, 8, seed=2)
    ps, ls = oracle.pagerank(G.row_ptr, G.col_ind, G.vals, iters=8)
    pp, lp = oracle.pagerank(G.row_ptr, G.col_ind, G.vals, iters=8, parallel=True)
    np.testing.assert_array_equal(ps, pp)
    np.testing.assert_array_equal(ls, lp)
    assert oracle.threads(False) == 1 and oracle.threads(True) >= 1
