"""Batched execution (lilac_batch_spmv / lilac_batch_cg) against the FP64
oracle, and the alone-versus-in-a-mix property: a problem's result is bitwise
the same whatever else runs in the batch (its reductions follow its own item
order only).  Problems run in the layout their handle's tuned kernel asks for
(sliced ELL chunk groups for SELL and SLAB, STAGED tiles otherwise), with
FP64 and FP32 handles in the same batch."""
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


# (matrix, variant forced on an untuned handle): sliced ELL layouts (SELL,
# SLAB) and STAGED tiles (STAGED, VECTOR, MERGE) in one batch
_LAYOUT_MIX = [
    (lambda: inputs.spd_random(6000, 15, 20.0, 3), L.LILAC_VARIANT_SELL),
    (lambda: inputs.spd_random(30000, 40, 20.0, 4), L.LILAC_VARIANT_SLAB),
    (lambda: inputs.powerlaw_csr(3000, 3000, 30000, power=8, seed=2), L.LILAC_VARIANT_SELL),
    (lambda: inputs.banded_spd(9000, 20, 1.0, 5), L.LILAC_VARIANT_STAGED),
    (lambda: inputs.laplacian2d(40), L.LILAC_VARIANT_VECTOR),
    (lambda: inputs.random_csr(2500, 2500, 25, 0.2, 4), L.LILAC_VARIANT_MERGE),
]


def _layout_handles(dtype=np.float64):
    As, Ms = [], []
    for make, variant in _LAYOUT_MIX:
        A = make().astype(dtype)
        M = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
        M.set_variant(variant, 4)
        As.append(A)
        Ms.append(M)
    return As, Ms


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_batched_spmv_runs_each_problem_in_its_tuned_layout(dtype):
    """SELL- and SLAB-tuned handles run as sliced ELL chunk groups (the SLAB
    handle gets its sliced ELL copy on first batched use), the others as
    STAGED tiles; FP64 or FP32 handles; every y within the oracle's bound and
    bitwise the same alone and in the mix."""
    torch = torch_cuda()
    fp32 = dtype == np.float32
    tdt = torch.float32 if fp32 else torch.float64
    As, Ms = _layout_handles(dtype)
    assert Ms[1].info()["sell_padded_nnz"] == 0  # SLAB: no sliced ELL copy yet
    xs_np = [inputs.uniform(70 + i, A.ncols, dtype=dtype) for i, A in enumerate(As)]
    xs = [dev(x) for x in xs_np]
    ys = [torch.full((A.n,), float("nan"), dtype=tdt, device="cuda") for A in As]
    B = L.Batch()
    B.spmv(Ms, xs, ys)
    torch.cuda.synchronize()
    assert Ms[1].info()["sell_padded_nnz"] > 0  # built for the batch
    for A, x, y in zip(As, xs_np, ys):
        assert_spmv_close(A, x.astype(np.float64), host(y), fp32, A.name)
    for i in range(len(As)):
        y1 = torch.empty(As[i].n, dtype=tdt, device="cuda")
        B.spmv([Ms[i]], [xs[i]], [y1])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(host(y1), host(ys[i]))
    B.close()
    for M in Ms:
        M.close()


def test_batched_cg_in_mixed_layouts_and_precisions():
    """FP64 CG over handles of every layout, and precision-2 CG over FP32
    handles (their own values are the FP32 values; the FP64 residual promotes
    them): each within 1e-10 of its own system, bitwise the same alone and in
    the mix.  FP32 handles refuse FP64 CG."""
    torch = torch_cuda()
    spd = [0, 1, 3, 4]  # the SPD matrices of the mix
    As, Ms = _layout_handles(np.float64)
    As = [As[i] for i in spd]
    for i in set(range(len(Ms))) - set(spd):
        Ms[i].close()
    Ms = [Ms[i] for i in spd]
    bs = [dev(inputs.uniform(80 + i, A.n)) for i, A in enumerate(As)]
    xs = [torch.zeros(A.n, dtype=torch.float64, device="cuda") for A in As]
    B = L.Batch()
    st, infos = B.cg(Ms, bs, xs, max_iter=3000, rtol=1e-10)
    torch.cuda.synchronize()
    assert st == L.LILAC_OK
    for A, b, x, info in zip(As, bs, xs, infos):
        assert info.status == L.LILAC_OK
        assert true_rel_residual(A, host(b), host(x)) <= 1e-10
    for i in (0, 1, 3):
        x1 = torch.zeros(As[i].n, dtype=torch.float64, device="cuda")
        B.cg([Ms[i]], [bs[i]], [x1], max_iter=3000, rtol=1e-10)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(host(x1), host(xs[i]))
    # FP32 handles: precision 2, values FP32-exact (Laplacian) or rounded
    A32 = [inputs.laplacian3d(16).astype(np.float32),
           inputs.banded_spd(4000, 10, 1.0, seed=6, fp32_exact=False).astype(np.float32)]
    M32 = [L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE) for A in A32]
    M32[0].set_variant(L.LILAC_VARIANT_SELL, 4)
    b32 = [dev(inputs.uniform(90 + i, A.n)) for i, A in enumerate(A32)]
    x32 = [torch.zeros(A.n, dtype=torch.float64, device="cuda") for A in A32]
    st, infos = B.cg(M32 + [Ms[0]], b32 + [bs[0]],
                     x32 + [torch.zeros(As[0].n, dtype=torch.float64, device="cuda")],
                     max_iter=5000, rtol=1e-10, precision=2)
    torch.cuda.synchronize()
    assert st == L.LILAC_OK
    for A, b, x, info in zip(A32, b32, x32, infos):
        assert info.status == L.LILAC_OK and info.refinements >= 1
        # the system of the FP32 values, in FP64 arithmetic
        assert true_rel_residual(A.astype(np.float64), host(b), host(x)) <= 1e-10
    x1 = torch.zeros(A32[0].n, dtype=torch.float64, device="cuda")
    B.cg([M32[0]], [b32[0]], [x1], max_iter=5000, rtol=1e-10, precision=2)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(x1), host(x32[0]))
    with pytest.raises(L.LilacError) as e:
        B.cg([M32[0]], [b32[0]], [x1], max_iter=10, rtol=1e-10, precision=0)
    assert e.value.status == L.LILAC_ERR_DTYPE
    B.close()
    for M in Ms + M32:
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
