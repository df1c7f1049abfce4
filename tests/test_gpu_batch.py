"""Batched execution (lilac_batch_spmv / lilac_batch_cg) against the FP64
oracle, and the alone-versus-in-a-mix property: a problem's result is bitwise
the same whatever else runs in the batch (its reductions follow its own tile
order only)."""
import numpy as np
import pytest

import oracle
from paper_2001_07938_gb300 import inputs
from paper_2001_07938_gb300 import lilac as L
from lilac_testutil import assert_spmv_close, dev, host, torch_cuda, true_rel_residual

pytestmark = pytest.mark.gpu


def _mats():
    return [inputs.laplacian2d(30), inputs.powerlaw_csr(3000, 4000, 30000, power=8, seed=2),
            inputs.random_csr(2500, 1800, 25, 0.2, 4), inputs.spd_random(6000, 15, 20.0, 3),
            inputs.banded_spd(9000, 20, 1.0, 5)]


def test_batched_spmv_matches_oracle_including_shared_matrix():
    torch = torch_cuda()
    As = _mats()
    Ms = [L.CsrMatrix.from_csr(A) for A in As]
    # the power-law matrix twice with different x: split rows must not share scratch
    mats, xs_np = [], []
    for i, (A, M) in enumerate(zip(As, Ms)):
        mats.append((A, M))
        xs_np.append(inputs.uniform(30 + i, A.ncols))
    mats.append((As[1], Ms[1]))
    xs_np.append(inputs.uniform(99, As[1].ncols))
    xs = [dev(x) for x in xs_np]
    ys = [torch.full((A.n,), float("nan"), dtype=torch.float64, device="cuda") for A, _ in mats]
    B = L.Batch()
    B.spmv([M for _, M in mats], xs, ys)
    torch.cuda.synchronize()
    for (A, _), x, y in zip(mats, xs_np, ys):
        assert_spmv_close(A, x, host(y), False, A.name)
    B.close()
    for M in Ms:
        M.close()


def test_batched_cg_converges_and_matches_oracle_iterations():
    torch = torch_cuda()
    As = [inputs.laplacian2d(24), inputs.spd_random(6000, 15, 20.0, 3), inputs.banded_spd(9000, 20, 1.0, 5)]
    Ms = [L.CsrMatrix.from_csr(A) for A in As]
    bs_np = [inputs.uniform(50 + i, A.n) for i, A in enumerate(As)]
    bs_np.append(inputs.uniform(77, As[1].n))  # second system on the same matrix
    mats = Ms + [Ms[1]]
    Asx = As + [As[1]]
    xs = [torch.zeros(A.n, dtype=torch.float64, device="cuda") for A in Asx]
    B = L.Batch()
    st, infos = B.cg(mats, [dev(b) for b in bs_np], xs, max_iter=3000, rtol=1e-10)
    torch.cuda.synchronize()
    assert st == L.LILAC_OK
    for A, b, x, info in zip(Asx, bs_np, xs, infos):
        assert info.status == L.LILAC_OK
        assert true_rel_residual(A, b, host(x)) <= 1e-10
        _, itr, _ = oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=3000, rtol=1e-10)
        assert abs(info.iters - itr) <= 2
    B.close()
    for M in Ms:
        M.close()


def test_result_is_bitwise_the_same_alone_and_in_a_mix():
    torch = torch_cuda()
    As = [inputs.spd_random(6000, 15, 20.0, 3), inputs.laplacian2d(40), inputs.banded_spd(5000, 9, 1.0, 1)]
    Ms = [L.CsrMatrix.from_csr(A) for A in As]
    b0 = dev(inputs.uniform(5, As[0].n))
    B = L.Batch()
    x_alone = torch.zeros(As[0].n, dtype=torch.float64, device="cuda")
    B.cg([Ms[0]], [b0], [x_alone], max_iter=500, rtol=1e-10)
    xs = [torch.zeros(A.n, dtype=torch.float64, device="cuda") for A in As]
    bs = [b0] + [dev(inputs.uniform(6 + i, A.n)) for i, A in enumerate(As[1:])]
    B.cg(list(reversed(Ms)), list(reversed(bs)), list(reversed(xs)), max_iter=500, rtol=1e-10)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(xs[0]), host(x_alone))
    # SpMV too
    y_alone = torch.empty(As[0].n, dtype=torch.float64, device="cuda")
    B.spmv([Ms[0]], [b0], [y_alone])
    ys = [torch.empty(A.n, dtype=torch.float64, device="cuda") for A in As]
    B.spmv(Ms[::-1], [dev(inputs.uniform(1, As[2].ncols)), dev(inputs.uniform(2, As[1].ncols)), b0],
           ys[::-1])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(ys[0]), host(y_alone))
    B.close()
    for M in Ms:
        M.close()


def test_batch_rejects_fp32_handles():
    A = inputs.laplacian2d(10).astype(np.float32)
    M = L.CsrMatrix.from_csr(A)
    B = L.Batch()
    torch = torch_cuda()
    x = torch.zeros(A.n, dtype=torch.float32, device="cuda")
    with pytest.raises(L.LilacError) as e:
        B.spmv([M], [x], [x])
    assert e.value.status == L.LILAC_ERR_DTYPE
    B.close()
    M.close()


def test_batched_mixed_precision_cg_reaches_fp64_tolerance_alone_and_in_a_mix():
    """Precision 2 (FP32 values and vectors, FP64 reliable updates) in the
    batched engine: each system's FP64 true residual <= 1e-10 (values FP32-exact
    or not), and a system's result is bitwise the same alone and in a mix."""
    torch = torch_cuda()
    As = [inputs.laplacian3d(20), inputs.banded_spd(5000, 12, 1.0, seed=3, fp32_exact=False),
          inputs.spd_random(6000, 15, 20.0, 3)]
    Ms = [L.CsrMatrix.from_csr(A) for A in As]
    bs = [dev(inputs.uniform(60 + i, A.n)) for i, A in enumerate(As)]
    xs = [torch.zeros(A.n, dtype=torch.float64, device="cuda") for A in As]
    B = L.Batch()
    st, infos = B.cg(Ms, bs, xs, max_iter=5000, rtol=1e-10, precision=2)
    torch.cuda.synchronize()
    assert st == L.LILAC_OK
    for A, b, x, info in zip(As, bs, xs, infos):
        assert info.status == L.LILAC_OK and info.refinements >= 1
        assert true_rel_residual(A, host(b), host(x)) <= 1e-10
        assert info.rel_res <= 1e-10
    x_alone = torch.zeros(As[1].n, dtype=torch.float64, device="cuda")
    B.cg([Ms[1]], [bs[1]], [x_alone], max_iter=5000, rtol=1e-10, precision=2)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(x_alone), host(xs[1]))
    B.close()
    for M in Ms:
        M.close()
