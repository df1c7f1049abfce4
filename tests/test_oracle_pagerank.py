"""Pins of the oracle's PageRank power iteration (GAP PageRank, Section 5).

Against: mass conservation (sum x = 1), the uniform fixed point of a directed
cycle and of an edgeless graph, the closed-form fixed point
x* = (1-d)/N (I - d M)^-1 1 solved densely, and the L1 contraction by d.
"""
import numpy as np
import pytest

import oracle
from paper_2001_07938_gb300 import inputs


def _transposed_csr(N, edges):
    """Transposed link matrix (row = destination) with 1/outdeg values from an edge list."""
    edges = sorted(set((s, t) for s, t in edges if s != t), key=lambda e: (e[1], e[0]))
    outdeg = np.zeros(N, np.int64)
    for s, _ in edges:
        outdeg[s] += 1
    rp = np.zeros(N + 1, np.int32)
    for _, t in edges:
        rp[t + 1] += 1
    rp = np.cumsum(rp).astype(np.int32)
    ci = np.array([s for s, _ in edges], np.int32)
    v = np.array([1.0 / outdeg[s] for s, _ in edges])
    return rp, ci, v, outdeg


def _closed_form(N, rp, ci, v, outdeg, d):
    M = np.zeros((N, N))
    for i in range(N):
        for j in range(rp[i], rp[i + 1]):
            M[i, ci[j]] += v[j]
    M[:, outdeg == 0] = 1.0 / N
    return np.linalg.solve(np.eye(N) - d * M, np.full(N, (1 - d) / N))


def test_mass_conserved_every_iteration():
    A = inputs.rmat_transposed(10, 8, seed=3)
    od = A.extra["outdeg"]
    assert np.any(od == 0)  # has dangling vertices
    v64 = 1.0 / od[A.col_ind]  # FP64 1/outdeg: columns of non-dangling vertices sum to 1
    for t in range(1, 8):
        x, l1 = oracle.pagerank(A.row_ptr, A.col_ind, v64, iters=t)
        assert abs(x.sum() - 1.0) <= 1e-12
    # with the FP32-rounded values the mass drifts only by the value rounding
    x, _ = oracle.pagerank(A.row_ptr, A.col_ind, A.vals, iters=7)
    assert abs(x.sum() - 1.0) <= 7 * 6e-8


@pytest.mark.parametrize("N", [1, 2, 7, 100])
def test_cycle_is_uniform(N):
    if N == 1:
        rp, ci, v = np.array([0, 0], np.int32), np.zeros(0, np.int32), np.zeros(0)
    else:
        rp, ci, v, _ = _transposed_csr(N, [(i, (i + 1) % N) for i in range(N)])
    x, l1 = oracle.pagerank(rp, ci, v, iters=20)
    np.testing.assert_allclose(x, 1.0 / N, rtol=1e-15, atol=0)
    assert np.all(l1 <= 1e-15)


def test_edgeless_graph_is_uniform():
    N = 9
    x0 = inputs.uniform(4, N, 0.0, 1.0)
    x0 /= x0.sum()
    x, l1 = oracle.pagerank(np.zeros(N + 1, np.int32), np.zeros(0, np.int32), np.zeros(0),
                            iters=1, x0=x0)
    np.testing.assert_allclose(x, 1.0 / N, rtol=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("d", [0.85, 0.5])
def test_fixed_point_closed_form(seed, d):
    N = 40
    rng = np.random.default_rng(seed)
    edges = [(int(s), int(t)) for s, t in rng.integers(0, N, size=(120, 2))]
    edges = [e for e in edges if e[0] % 7 != 3]  # make some vertices dangling
    rp, ci, v, od = _transposed_csr(N, edges)
    assert np.any(od == 0)
    xs = _closed_form(N, rp, ci, v, od, d)
    x, l1 = oracle.pagerank(rp, ci, v, iters=300, damping=d)
    np.testing.assert_allclose(x, xs, rtol=1e-12, atol=1e-15)


def test_l1_contracts_by_damping():
    A = inputs.rmat_transposed(9, 8, seed=5)
    v64 = 1.0 / A.extra["outdeg"][A.col_ind]
    x, l1 = oracle.pagerank(A.row_ptr, A.col_ind, v64, iters=30, damping=0.85)
    assert np.all(l1[1:] <= 0.85 * l1[:-1] * (1 + 1e-9) + 1e-17)
    assert l1[0] > 0


def test_generator_transposed_structure():
    A = inputs.rmat_transposed(8, 8, seed=1)
    od = A.extra["outdeg"]
    rp, ci, v = A.row_ptr, A.col_ind, A.vals
    # sorted unique sources per row, no self-loops, values 1/outdeg in FP32
    for i in range(A.n):
        row = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0)
        assert not np.any(row == i)
    np.testing.assert_array_equal(np.bincount(ci, minlength=A.n), od)
    np.testing.assert_array_equal(v, (1.0 / od[ci]).astype(np.float32))
