"""Failure paths, exercised without faulting the GPU: an injected allocation
failure, and bounded device waits made to expire by host-set test hooks (the
STAGED kernel's first bulk copy left unissued; a CTA that skips the fused CG
step's grid barrier); the handle reports the timeout, stays sticky, and works
again after lilac_csr_reset_error."""
import numpy as np
import pytest

from paper_2001_07938_gb300 import inputs
from paper_2001_07938_gb300 import lilac as L
from lilac_testutil import assert_spmv_close, dev, host, torch_cuda, true_rel_residual

pytestmark = pytest.mark.gpu


def test_injected_allocation_failure_is_oom_and_leaves_no_state():
    torch_cuda()
    A = inputs.laplacian2d(32)
    L.lilac_debug_inject(None, L.LILAC_INJECT_ALLOC_FAIL, 1)
    with pytest.raises(L.LilacError) as e:
        L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
    assert e.value.status == L.LILAC_ERR_OOM
    # a later allocation in the middle of create
    L.lilac_debug_inject(None, L.LILAC_INJECT_ALLOC_FAIL, 3)
    with pytest.raises(L.LilacError) as e:
        L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
    assert e.value.status == L.LILAC_ERR_OOM
    L.lilac_debug_inject(None, L.LILAC_INJECT_ALLOC_FAIL, 0)
    M = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
    x = inputs.uniform(1, A.ncols)
    y = np.zeros(A.n)
    M.spmv(x, y)
    assert_spmv_close(A, x, y, False, "after injected OOM")
    M.close()


def test_bounded_wait_timeout_is_reported_sticky_and_reset():
    torch_cuda()
    A = inputs.laplacian2d(200)
    M = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
    M.set_variant(L.LILAC_VARIANT_STAGED, 1)
    x = inputs.uniform(2, A.ncols)
    y = np.zeros(A.n)
    M.spmv(x, y)
    assert_spmv_close(A, x, y, False, "before")
    L.lilac_debug_inject(M.handle, L.LILAC_INJECT_SKIP_COPY)
    with pytest.raises(L.LilacError) as e:
        M.spmv(x, y)  # CTA 0 waits ~2 s for a copy that was never issued
    assert e.value.status == L.LILAC_ERR_TIMEOUT
    with pytest.raises(L.LilacError) as e:
        M.spmv(x, y)  # sticky until reset
    assert e.value.status == L.LILAC_ERR_TIMEOUT
    L.lilac_csr_reset_error(M.handle)
    y[:] = 0.0
    M.spmv(x, y)
    assert_spmv_close(A, x, y, False, "after reset")
    M.close()


@pytest.mark.parametrize("variant,width,precision", [
    (L.LILAC_VARIANT_SLAB, 4, 0),   # cg_step_slabs_kernel
    (L.LILAC_VARIANT_SELL, 1, 0),   # cg_step_kernel, FP64
    (L.LILAC_VARIANT_SELL, 1, 2),   # cg_step_kernel, FP32 with FP64 reliable updates
])
def test_cg_step_barrier_timeout_is_reported_sticky_and_reset(variant, width, precision):
    """CG runs each step's update and direction in one launch with a bounded
    grid barrier.  With CTA 0 kept from arriving, the other CTAs give up after
    ~2 s and the solve reports LILAC_ERR_TIMEOUT (sticky); after the reset the
    same solve converges."""
    torch = torch_cuda()
    A = inputs.spd_random(30000, 40, 20.0, 4)
    b = inputs.uniform(3, A.n)
    M = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
    M.set_variant(variant, width)
    assert M.info()["active_variant"] == variant
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    L.lilac_debug_inject(M.handle, L.LILAC_INJECT_SKIP_BARRIER)
    with pytest.raises(L.LilacError) as e:
        M.cg(dev(b), x, rtol=1e-10, max_iter=300, precision=precision)
    assert e.value.status == L.LILAC_ERR_TIMEOUT
    with pytest.raises(L.LilacError) as e:
        M.cg(dev(b), x, rtol=1e-10, max_iter=300, precision=precision)
    assert e.value.status == L.LILAC_ERR_TIMEOUT
    L.lilac_csr_reset_error(M.handle)
    x.zero_()
    st, info = M.cg(dev(b), x, rtol=1e-10, max_iter=300, precision=precision)
    torch.cuda.synchronize()
    assert st == L.LILAC_OK
    assert true_rel_residual(A, b, host(x)) <= 1e-10
    M.close()
