"""Pins of the oracle's CSR SpMV, dot product, ncols invariant and JDS path.

Each test checks the oracle against something other than itself: the
paper's printed worked example, a dense product computed by numpy / scipy,
closed-form Laplacian eigenpairs, or exact integer arithmetic.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2001_07938_gb300 import inputs
from conftest import load_golden


def _dense(n, ncols, rp, ci, v):
    D = np.zeros((n, ncols))
    for i in range(n):
        for j in range(rp[i], rp[i + 1]):
            D[i, ci[j]] += v[j]
    return D


def test_paper_csr_example_by_hand():
    g = load_golden("csr_example_5x5.txt")
    rp, ci, v = g["row_ptr"], g["col_ind"], g["val"]
    assert len(rp) - 1 == 5
    assert oracle.csr_ncols(ci) == 5
    assert list(np.diff(rp)) == [2, 2, 3, 1, 2]
    y = oracle.spmv(rp, ci, v, g["x"])
    assert list(y) == [float(t) for t in g["y"]]  # exact integers


def test_paper_csr_example_vs_dense():
    g = load_golden("csr_example_5x5.txt")
    rp, ci, v = g["row_ptr"], g["col_ind"], g["val"]
    D = _dense(5, 5, rp, ci, v)
    x = inputs.uniform(11, 5)
    np.testing.assert_allclose(oracle.spmv(rp, ci, v, x), D @ x, rtol=0, atol=1e-14)


def test_paper_jds_example_matches_csr_example():
    """CSR -> JDS of the printed CSR example reproduces the printed JDS arrays."""
    c = load_golden("csr_example_5x5.txt")
    j = load_golden("jds_example_5x5.txt")
    J = oracle.csr_to_jds(c["row_ptr"], c["col_ind"], c["val"])
    assert list(J["perm"]) == j["perm"]
    assert list(J["nzcnt"]) == j["nzcnt"]
    assert list(J["jd_ptr"]) == j["jd_ptr"]
    assert list(J["col_ind"]) == j["col_ind"]
    assert list(J["val"]) == [float(t) for t in j["val"]]


def test_paper_jds_example_spmv_vs_dense():
    c = load_golden("csr_example_5x5.txt")
    j = load_golden("jds_example_5x5.txt")
    D = _dense(5, 5, c["row_ptr"], c["col_ind"], c["val"])
    # build the dense matrix from the printed JDS arrays directly
    DJ = np.zeros((5, 5))
    slot_row = {s: r for r, s in enumerate(j["perm"])}
    for k in range(len(j["jd_ptr"]) - 1):
        for s in range(j["jd_ptr"][k + 1] - j["jd_ptr"][k]):
            DJ[slot_row[s], j["col_ind"][j["jd_ptr"][k] + s]] += j["val"][j["jd_ptr"][k] + s]
    np.testing.assert_array_equal(D, DJ)
    x = inputs.uniform(5, 5)
    y = oracle.jds_spmv(j["perm"], j["jd_ptr"], j["col_ind"], j["val"], x)
    np.testing.assert_allclose(y, D @ x, rtol=0, atol=1e-14)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
@pytest.mark.parametrize("n,ncols,max_len", [(1, 1, 3), (7, 5, 4), (64, 40, 12), (50, 200, 30)])
def test_random_csr_vs_scipy_and_dense(seed, n, ncols, max_len):
    A = inputs.random_csr(n, ncols, max_len, 0.2, seed)
    x = inputs.uniform(100 + seed, ncols)
    y = oracle.spmv(A.row_ptr, A.col_ind, A.vals, x)
    bound = 1e-12 * oracle.spmv_abs_bound(A.row_ptr, A.col_ind, A.vals, x)
    S = sp.csr_matrix((A.vals, A.col_ind, A.row_ptr), shape=(n, ncols))  # sums duplicates
    assert np.all(np.abs(y - S @ x) <= bound + 1e-300)
    D = _dense(n, ncols, A.row_ptr, A.col_ind, A.vals)
    assert np.all(np.abs(y - D @ x) <= bound + 1e-300)


def test_empty_rows_give_zero_and_empty_matrix():
    rp = np.array([0, 0, 2, 2, 3], np.int32)
    ci = np.array([3, 1, 0], np.int32)
    v = np.array([2.0, -1.0, 5.0])
    y = oracle.spmv(rp, ci, v, np.array([1.0, 2.0, 3.0, 4.0]))
    assert list(y) == [0.0, 8.0 - 2.0, 0.0, 5.0]
    y0 = oracle.spmv(np.zeros(4, np.int32), np.zeros(0, np.int32), np.zeros(0), np.ones(3))
    assert list(y0) == [0.0, 0.0, 0.0]
    assert oracle.csr_ncols(np.zeros(0, np.int32)) == 0


@pytest.mark.parametrize("m", [1, 5, 16, 64])
@pytest.mark.parametrize("jk", [(1, 1), (2, 3), (5, 4)])
def test_laplacian2d_eigenpair(m, jk):
    """A v = lambda v for v_(a,b) = sin(j pi (a+1)/(m+1)) sin(k pi (b+1)/(m+1)),
    lambda = 4 - 2cos(j pi/(m+1)) - 2cos(k pi/(m+1))."""
    j, k = jk
    if j > m or k > m:
        pytest.skip("mode index beyond grid")
    A = inputs.laplacian2d(m)
    a = np.arange(1, m + 1)
    v = np.outer(np.sin(j * np.pi * a / (m + 1)), np.sin(k * np.pi * a / (m + 1))).ravel()
    lam = 4 - 2 * math.cos(j * math.pi / (m + 1)) - 2 * math.cos(k * math.pi / (m + 1))
    y = oracle.spmv(A.row_ptr, A.col_ind, A.vals, v)
    bound = 1e-12 * oracle.spmv_abs_bound(A.row_ptr, A.col_ind, A.vals, v) + 8 * abs(lam) * 2.3e-16
    assert np.all(np.abs(y - lam * v) <= bound)


@pytest.mark.parametrize("m", [2, 7, 12])
def test_laplacian3d_eigenpair(m):
    j, k, l = 1, min(2, m), min(3, m)
    A = inputs.laplacian3d(m)
    a = np.arange(1, m + 1)
    s = lambda q: np.sin(q * np.pi * a / (m + 1))
    v = np.einsum("i,j,k->ijk", s(j), s(k), s(l)).ravel()
    lam = 6 - 2 * sum(math.cos(q * math.pi / (m + 1)) for q in (j, k, l))
    y = oracle.spmv(A.row_ptr, A.col_ind, A.vals, v)
    bound = 1e-12 * oracle.spmv_abs_bound(A.row_ptr, A.col_ind, A.vals, v) + 8 * abs(lam) * 2.3e-16
    assert np.all(np.abs(y - lam * v) <= bound)


def test_row_sums_exact_for_integers():
    A = inputs.random_csr(300, 120, 25, 0.1, 7)
    vals = np.round(A.vals * 50)  # integer-valued
    y = oracle.spmv(A.row_ptr, A.col_ind, vals, np.ones(120))
    rs = np.array([vals[A.row_ptr[i]:A.row_ptr[i + 1]].sum() for i in range(300)])
    np.testing.assert_array_equal(y, rs)


def test_dot_against_exact_sum():
    a = inputs.uniform(1, 10_000)
    b = inputs.uniform(2, 10_000)
    exact = math.fsum(float(p) for p in (a * b))  # products are exact? no: bound below
    got = oracle.dot(a, b)
    # |fl(sum) - sum| <= n eps sum|a_i b_i| (products rounded too)
    assert abs(got - exact) <= 10_000 * 1.2e-16 * float(np.sum(np.abs(a * b)))
    ai = np.round(a * 1000)
    bi = np.round(b * 1000)
    assert oracle.dot(ai, bi) == float(sum(int(p) * int(q) for p, q in zip(ai, bi)))


def test_laplacian_nnz_closed_forms():
    for m in (1, 2, 3, 64):
        assert inputs.laplacian2d(m).nnz == 5 * m * m - 4 * m
    for m in (1, 2, 5, 16):
        assert inputs.laplacian3d(m).nnz == 7 * m ** 3 - 6 * m * m


@pytest.mark.parametrize("seed", [0, 1])
def test_jds_roundtrip_random(seed):
    A = inputs.random_csr(80, 60, 9, 0.2, seed)
    J = oracle.csr_to_jds(A.row_ptr, A.col_ind, A.vals)
    # nzcnt non-increasing; perm is a permutation
    assert np.all(np.diff(J["nzcnt"]) <= 0)
    assert sorted(J["perm"]) == list(range(80))
    x = inputs.uniform(9, 60)
    y = oracle.jds_spmv(J["perm"], J["jd_ptr"], J["col_ind"], J["val"], x)
    S = sp.csr_matrix((A.vals, A.col_ind, A.row_ptr), shape=(80, 60))
    bound = 1e-12 * oracle.spmv_abs_bound(A.row_ptr, A.col_ind, A.vals, x)
    assert np.all(np.abs(y - S @ x) <= bound + 1e-300)
