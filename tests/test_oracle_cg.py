"""Pins of the oracle's conjugate gradient (Hestenes-Stiefel, the NAS CG solver).

Against: finite termination in exact arithmetic (n steps; #distinct
eigenvalues steps for a diagonal matrix; one step for an eigenvector
right-hand side), a dense Cholesky solve (numpy/LAPACK), and the breakdown
condition on an indefinite matrix.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2001_07938_gb300 import inputs


def _csr_from_dense(D):
    n = D.shape[0]
    rp = [0]
    ci, v = [], []
    for i in range(n):
        for j in range(D.shape[1]):
            if D[i, j] != 0.0:
                ci.append(j)
                v.append(D[i, j])
        rp.append(len(ci))
    return np.array(rp, np.int32), np.array(ci, np.int32), np.array(v)


def _spd_dense(n, seed, cond=50.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, cond, n)
    return (Q * ev) @ Q.T


@pytest.mark.parametrize("n", [2, 8, 20, 32])
def test_finite_termination_within_n_steps(n):
    D = _spd_dense(n, n, cond=5.0)
    rp, ci, v = _csr_from_dense(D)
    b = inputs.uniform(3, n)
    x, it, st = oracle.cg(rp, ci, v, b, max_iter=n, rtol=1e-12)
    assert st == oracle.CG_CONVERGED and it <= n
    assert np.linalg.norm(b - D @ x) <= 1e-11 * np.linalg.norm(b)


def test_diagonal_converges_in_distinct_eigenvalue_steps():
    d = np.array([1.0, 3.0, 3.0, 7.0, 1.0, 7.0, 3.0, 1.0])  # 3 distinct values
    n = d.size
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    x, it, st, hist = oracle.cg(rp, ci, d, np.ones(n), max_iter=10, rtol=1e-14, want_hist=True)
    assert st == oracle.CG_CONVERGED
    assert it == 3
    np.testing.assert_allclose(x, 1.0 / d, rtol=1e-14)


@pytest.mark.parametrize("m,jk", [(8, (1, 1)), (16, (3, 2)), (31, (7, 11))])
def test_laplacian_eigenmode_rhs_one_step(m, jk):
    j, k = jk
    A = inputs.laplacian2d(m)
    a = np.arange(1, m + 1)
    v = np.outer(np.sin(j * np.pi * a / (m + 1)), np.sin(k * np.pi * a / (m + 1))).ravel()
    lam = 4 - 2 * math.cos(j * math.pi / (m + 1)) - 2 * math.cos(k * math.pi / (m + 1))
    x, it, st = oracle.cg(A.row_ptr, A.col_ind, A.vals, v, max_iter=5, rtol=1e-12)
    assert it == 1 and st == oracle.CG_CONVERGED
    np.testing.assert_allclose(x, v / lam, rtol=0, atol=1e-13 * np.max(np.abs(v / lam)))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_against_dense_cholesky(seed):
    n = 200
    A = inputs.banded_spd(n, 6, 1.0, seed)
    D = np.zeros((n, n))
    for i in range(n):
        D[i, A.col_ind[A.row_ptr[i]:A.row_ptr[i + 1]]] = A.vals[A.row_ptr[i]:A.row_ptr[i + 1]]
    b = inputs.uniform(seed + 40, n)
    L = np.linalg.cholesky(D)
    xs = np.linalg.solve(L.T, np.linalg.solve(L, b))
    x, it, st = oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=1000, rtol=1e-13)
    assert st == oracle.CG_CONVERGED
    assert np.linalg.norm(x - xs) <= 1e-11 * np.linalg.norm(xs)


def test_exact_iteration_count_and_x0():
    A = inputs.laplacian2d(20)
    b = np.ones(A.n)
    x, it, st = oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=17, rtol=0.0)
    assert it == 17 and st == oracle.CG_MAXITER
    # restarting from that iterate continues to decrease the true residual
    r0 = np.linalg.norm(b - oracle.spmv(A.row_ptr, A.col_ind, A.vals, x))
    x2, it2, _ = oracle.cg(A.row_ptr, A.col_ind, A.vals, b, x0=x, max_iter=40, rtol=0.0)
    r2 = np.linalg.norm(b - oracle.spmv(A.row_ptr, A.col_ind, A.vals, x2))
    assert r2 < r0


def test_zero_rhs_and_breakdown():
    A = inputs.laplacian2d(4)
    x, it, st = oracle.cg(A.row_ptr, A.col_ind, A.vals, np.zeros(A.n), max_iter=10, rtol=1e-10)
    assert it == 0 and st == oracle.CG_CONVERGED and not np.any(x)
    # indefinite: diag(1, -1) with b = (1, 1) gives p.Ap = 0 at the first step
    rp = np.array([0, 1, 2], np.int32)
    ci = np.array([0, 1], np.int32)
    x, it, st = oracle.cg(rp, ci, np.array([1.0, -1.0]), np.array([1.0, 1.0]), max_iter=5,
                          rtol=1e-12)
    assert st == oracle.CG_BREAKDOWN and it == 0


def test_cg_history_matches_true_residual_small():
    """On a well-conditioned problem the recursive residual tracks b - A x."""
    A = inputs.spd_random(400, 12, 20.0, 3)
    b = np.ones(A.n)
    x, it, st, hist = oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=30, rtol=0.0,
                                want_hist=True)
    r = b - oracle.spmv(A.row_ptr, A.col_ind, A.vals, x)
    assert abs(math.sqrt(hist[-1]) - np.linalg.norm(r)) <= 1e-10 * np.linalg.norm(b)
    assert math.sqrt(hist[-1]) <= 1e-10 * np.linalg.norm(b)
