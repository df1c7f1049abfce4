"""The request server: every request of a mixed SpMV / CG stream (CG in FP64
or in FP32 with FP64 reliable updates; SpMV of one vector batched, of 2..32
through the multi-vector kernel) completes with the oracle's result (SpMV
tolerance; CG true residual <= 1e-10), with arrival <= admission <= finish,
a request's result is bitwise the same alone and in the mix, the matrices
may be tuned at upload, and a small device-memory budget forces
evictions and waiting without changing results."""
import numpy as np
import pytest

import oracle
from paper_2001_07938_gb300 import inputs
from paper_2001_07938_gb300 import lilac as L
from lilac_testutil import spmv_tolerance, torch_cuda, true_rel_residual

pytestmark = pytest.mark.gpu


def _pool():
    return [inputs.laplacian2d(20), inputs.laplacian2d(37), inputs.banded_spd(3000, 8, 1.0, 1),
            inputs.banded_spd(12000, 30, 1.0, 2), inputs.spd_random(5000, 12, 20.0, 3),
            inputs.laplacian3d(12)]


def _requests(pool, n, seed):
    """(kind, matrix index, input, vectors, tag, precision) for a seeded mix of
    SpMV and CG requests; half of the CG requests run in mixed precision."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(n):
        mi = int(rng.integers(len(pool)))
        A = pool[mi]
        if rng.random() < 0.5:
            k = int(rng.integers(1, 4))
            x = inputs.uniform(1000 + t, k * A.ncols)
            out.append(("spmv", mi, x, k, t, 0))
        else:
            b = inputs.uniform(2000 + t, A.n)
            out.append(("cg", mi, b, 1, t, 2 if rng.random() < 0.5 else 0))
    return out


def _serve(pool, reqs, budget=None, burst=7, tune=0):
    torch_cuda()
    S = L.Server(hbm_budget_bytes=budget, iters_per_round=8, tune=tune)
    ids = [S.add_matrix(A) for A in pool]
    outs, results = {}, {}
    i, steps = 0, 0
    while i < len(reqs) or len(results) < len(reqs):
        steps += 1
        assert steps < 20000, ("no progress", S.stats())
        for kind, mi, inp, k, tag, prec in reqs[i:i + burst]:
            A = pool[mi]
            if kind == "spmv":
                out = np.full(k * A.n, np.nan)
                S.submit(L.LILAC_REQ_SPMV, ids[mi], inp, out, tag, nvec=k)
            else:
                out = np.full(A.n, np.nan)
                S.submit(L.LILAC_REQ_CG, ids[mi], inp, out, tag, max_iter=5000, rtol=1e-10,
                         precision=prec)
            outs[tag] = out
        i += burst
        S.step()
        for c in S.poll():
            results[c["tag"]] = c
    stats = S.stats()
    S.close()
    return outs, results, stats


def _check(pool, reqs, outs, results):
    for kind, mi, inp, k, tag, prec in reqs:
        A, out, c = pool[mi], outs[tag], results[tag]
        assert c["status"] == L.LILAC_OK, (tag, c)
        assert c["arrival"] <= c["admitted"] <= c["finish"] and c["rounds"] >= 1
        if kind == "spmv":
            for j in range(k):
                x = inp[j * A.ncols:(j + 1) * A.ncols]
                y = out[j * A.n:(j + 1) * A.n]
                ref = oracle.spmv(A.row_ptr, A.col_ind, A.vals, x)
                assert np.all(np.abs(y - ref) <= spmv_tolerance(A, x, False)), tag
        else:
            assert true_rel_residual(A, inp, out) <= 1e-10, (tag, prec)
            if prec == 2:  # reported: the last FP64 residual b - A x
                assert c["rel_res"] <= 1e-10


@pytest.mark.parametrize("tune", [0, 1])
def test_mixed_stream_matches_oracle(tune):
    pool = _pool()
    reqs = _requests(pool, 60, seed=0)
    outs, results, stats = _serve(pool, reqs, tune=tune)
    assert stats["completed"] == 60 and stats["submitted"] == 60
    _check(pool, reqs, outs, results)


def test_same_result_alone_and_in_the_mix(tune=0):
    """(Untuned: the timed tuner may pick another kernel in another run.)"""
    pool = _pool()
    reqs = _requests(pool, 40, seed=1)
    outs_mix, _, _ = _serve(pool, reqs, tune=tune)
    cgs = [r for r in reqs if r[0] == "cg"]
    spmvs = [r for r in reqs if r[0] == "spmv"]
    probes = ([r for r in cgs if r[5] == 0][:2] + [r for r in cgs if r[5] == 2][:2] +
              [r for r in spmvs if r[3] == 1][:2] + [r for r in spmvs if r[3] > 1][:2])
    assert len(probes) == 8
    for probe in probes:
        outs_alone, _, _ = _serve(pool, [probe], tune=tune)
        np.testing.assert_array_equal(outs_alone[probe[4]], outs_mix[probe[4]])


def test_small_budget_evicts_and_waits_but_results_hold():
    pool = _pool()
    reqs = _requests(pool, 40, seed=2)
    budget = 13 << 20  # the largest matrix fits, the whole pool (~18 MB) does not
    outs, results, stats = _serve(pool, reqs, budget=budget, burst=40)
    _check(pool, reqs, outs, results)
    assert stats["evictions"] > 0 and stats["uploads"] > len(pool)


def test_invalid_requests_are_rejected():
    torch_cuda()
    S = L.Server()
    A = inputs.laplacian2d(8)
    mid = S.add_matrix(A)
    x = np.zeros(A.n)
    with pytest.raises(L.LilacError):
        S.submit(L.LILAC_REQ_SPMV, mid + 5, x, x, 0)
    with pytest.raises(L.LilacError):
        S.submit(L.LILAC_REQ_SPMV, mid, x, x, 0, nvec=0)
    with pytest.raises(L.LilacError):
        S.submit(L.LILAC_REQ_CG, mid, x, x, 0, precision=1)
    big = L.Server(hbm_budget_bytes=1 << 10)
    bid = big.add_matrix(A)
    with pytest.raises(L.LilacError) as e:
        big.submit(L.LILAC_REQ_CG, bid, x, x, 0)
    assert e.value.status == L.LILAC_ERR_BUDGET
    S.close()
    big.close()


def test_request_that_can_never_fit_completes_with_budget_error():
    """A matrix that fits the budget with a request whose workspace never can
    (a 32-vector SpMV: 4 MB of vectors against a 3 MB budget) completes with
    LILAC_ERR_BUDGET instead of waiting forever; the server then serves a
    single-vector request on the same matrix."""
    torch_cuda()
    A = inputs.laplacian2d(50)
    S = L.Server(hbm_budget_bytes=3 << 20)
    mid = S.add_matrix(A)
    X = inputs.uniform(5, 32 * A.ncols)
    Y = np.full(32 * A.n, np.nan)
    S.submit(L.LILAC_REQ_SPMV, mid, X, Y, 7, nvec=32)
    done = []
    for _ in range(100):
        S.step()
        done += S.poll()
        if done:
            break
    assert [c["tag"] for c in done] == [7] and done[0]["status"] == L.LILAC_ERR_BUDGET
    x = inputs.uniform(6, A.ncols)
    y = np.full(A.n, np.nan)
    S.submit(L.LILAC_REQ_SPMV, mid, x, y, 8)
    done = []
    for _ in range(100):
        S.step()
        done += S.poll()
        if done:
            break
    assert [c["tag"] for c in done] == [8] and done[0]["status"] == L.LILAC_OK
    ref = oracle.spmv(A.row_ptr, A.col_ind, A.vals, x)
    assert np.all(np.abs(y - ref) <= spmv_tolerance(A, x, False))
    S.close()
