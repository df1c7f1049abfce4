"""Mixed-precision CG on the GPU: FP32 inner CG with FP64 iterative
refinement (precision 1), and FP32 CG with FP64 reliable updates (precision
2: x accumulated in FP64, the residual replaced by the FP64 b - A x).

Accepted when the FP64 true residual ||b - A x|| / ||b||, computed by the
oracle's SpMV with the handle's own values, is <= 1e-10.  The 3D Laplacian's
values (6, -1) are exact in FP32, so the FP32 matrix is A itself; for a
matrix whose values are not FP32-exact the refinement still converges to the
FP64 system because the residual uses the FP64 values.
"""
import numpy as np
import pytest

import oracle
from paper_2001_07938_gb300 import inputs
from paper_2001_07938_gb300 import lilac as L
from lilac_testutil import dev, host, torch_cuda, true_rel_residual

pytestmark = pytest.mark.gpu


def _mixed(A, b, precision=1, variant=None, **kw):
    torch = torch_cuda()
    M = L.CsrMatrix.from_csr(A)
    if variant:
        M.set_variant(*variant)
    xd = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    st, info = M.cg(dev(b), xd, precision=precision, **kw)
    torch.cuda.synchronize()
    M.close()
    return st, info, host(xd)


def test_poisson3d_fp32_values_reach_1e10():
    A, b = inputs.workload_poisson3d_ir(24)
    st, info, x = _mixed(A, b, rtol=1e-10, max_iter=20)
    assert st == L.LILAC_OK and info.status == L.LILAC_OK
    assert info.refinements >= 2  # one FP32 solve alone cannot reach 1e-10
    A64 = A.astype(np.float64)
    assert true_rel_residual(A64, b, x) <= 1e-10
    # one FP32 solve alone, asked for 1e-12, stalls far above 1e-10
    st1, info1, x1 = _mixed(A, b, rtol=1e-10, max_iter=1, inner_rtol=1e-12, inner_max_iter=3000)
    assert st1 == L.LILAC_ERR_NOT_CONVERGED and info1.refinements == 1
    assert true_rel_residual(A64, b, x1) > 1e-9


def test_fp64_values_not_fp32_exact():
    A = inputs.banded_spd(5000, 12, 1.0, seed=3, fp32_exact=False)
    b = inputs.uniform(4, A.n)
    st, info, x = _mixed(A, b, rtol=1e-10, max_iter=30)
    assert st == L.LILAC_OK
    assert true_rel_residual(A, b, x) <= 1e-10
    xr, _, _ = oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=5000, rtol=1e-12)
    assert np.linalg.norm(x - xr) <= 1e-8 * np.linalg.norm(xr)


@pytest.mark.parametrize("precision", [1, 2])
def test_copy_variant_on_fp64_values_with_fp32_inner_solve(precision):
    """FP64 handle pinned to SELL: the FP64 residual runs on the SELL copy, the
    FP32 inner SpMV (a derived FP32 value array) falls back to STAGED."""
    A = inputs.banded_spd(6000, 16, 1.0, seed=5, fp32_exact=False)
    b = inputs.uniform(6, A.n)
    st, info, x = _mixed(A, b, precision=precision, variant=(7, 4), rtol=1e-10, max_iter=3000)
    assert st == L.LILAC_OK
    assert true_rel_residual(A, b, x) <= 1e-10


@pytest.mark.slow
def test_full_poisson3d_192():
    """3D Poisson 192^3 (n = 7,077,888), FP32 values, b uniform in [-1, 1] seed 1."""
    A, b = inputs.workload_poisson3d_ir()
    st, info, x = _mixed(A, b, rtol=1e-10, max_iter=20, inner_max_iter=4000)
    assert st == L.LILAC_OK
    assert true_rel_residual(A.astype(np.float64), b, x) <= 1e-10


def test_reliable_updates_reach_1e10_in_about_fp64_iterations():
    """Precision 2 keeps the Krylov direction across residual replacements, so
    it needs about as many iterations as FP64 CG (restarted refinement needs
    many more), and reaches the FP64 tolerance."""
    A, b = inputs.workload_poisson3d_ir(40)
    st, info, x = _mixed(A, b, precision=2, rtol=1e-10, max_iter=5000)
    assert st == L.LILAC_OK and info.status == L.LILAC_OK
    A64 = A.astype(np.float64)
    assert true_rel_residual(A64, b, x) <= 1e-10
    assert info.rel_res <= 1e-10 and info.refinements >= 5
    _, k64, _ = oracle.cg(A64.row_ptr, A64.col_ind, A64.vals, b, max_iter=5000, rtol=1e-10)
    assert info.iters <= int(1.25 * k64) + 5, (info.iters, k64)
    # a replacement every iteration (delta close to 1) is still correct
    st1, info1, x1 = _mixed(A, b, precision=2, rtol=1e-10, max_iter=5000, ru_delta=0.99)
    assert st1 == L.LILAC_OK and true_rel_residual(A64, b, x1) <= 1e-10


def test_reliable_updates_fp64_values_and_x0():
    A = inputs.banded_spd(5000, 12, 1.0, seed=3, fp32_exact=False)
    b = inputs.uniform(4, A.n)
    torch = torch_cuda()
    M = L.CsrMatrix.from_csr(A)
    x0 = inputs.uniform(5, A.n)
    xd = dev(x0.copy())
    st, info = M.cg(dev(b), xd, precision=2, rtol=1e-10, max_iter=3000, use_x0=True)
    torch.cuda.synchronize()
    x = host(xd)
    assert st == L.LILAC_OK
    assert true_rel_residual(A, b, x) <= 1e-10
    xr, _, _ = oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=5000, rtol=1e-12)
    assert np.linalg.norm(x - xr) <= 1e-8 * np.linalg.norm(xr)
    # iteration cap: NOT_CONVERGED with the FP64 residual reported
    xd.copy_(torch.zeros_like(xd))
    st2, info2 = M.cg(dev(b), xd, precision=2, rtol=1e-10, max_iter=3)
    assert st2 == L.LILAC_ERR_NOT_CONVERGED and info2.iters == 3
    assert info2.rel_res > 1e-10
    M.close()
