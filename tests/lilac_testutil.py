"""Helpers shared by the GPU parity tests: device tensors, tolerances, and
calls through the C ABI (via the thin binding)."""
import numpy as np

import oracle

U64 = 2.0 ** -53  # unit roundoff, binary64
U32 = 2.0 ** -24  # unit roundoff, binary32


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def dev(a):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def row_lengths(A):
    return np.diff(A.row_ptr).astype(np.float64)


def spmv_tolerance(A, x, fp32: bool):
    """Componentwise bound on |y - y_ref| for y = A x.

    FP64: 1e-12 (|A||x|)_i, the stated SpMV tolerance, widened to
    (k_i + 2) u64 (|A||x|)_i for rows long enough (k_i > ~9000) that the
    worst-case summation error of any order can exceed it.  FP32 (values and
    x given in FP32, FP32 accumulation in any order): (k_i + 2) u32 (|A||x|)_i,
    the worst-case bound of a length-k_i sum of rounded products.
    """
    ax = oracle.spmv_abs_bound(A.row_ptr, A.col_ind, A.vals, x)
    k = row_lengths(A)
    if fp32:
        return (k + 2.0) * U32 * ax * 1.0001 + 1e-37
    return np.maximum(1e-12, (k + 2.0) * U64) * ax + 1e-300


def assert_spmv_close(A, x, y, fp32: bool, what=""):
    ref = oracle.spmv(A.row_ptr, A.col_ind, A.vals, x)
    tol = spmv_tolerance(A, x, fp32)
    err = np.abs(np.asarray(y, np.float64) - ref)
    bad = np.nonzero(err > tol)[0]
    assert bad.size == 0, (f"{what}: {bad.size} rows out of tolerance, first {bad[:5]}, "
                           f"err {err[bad[:5]]}, tol {tol[bad[:5]]}")
    return ref


def true_rel_residual(A, b, x):
    r = np.asarray(b, np.float64) - oracle.spmv(A.row_ptr, A.col_ind, A.vals, x)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


# (variant, lanes per row); for SLAB and SELL the width is the STAGED width
# they fall back to where their copy is not built
ALL_VARIANTS = ([(1, 1)] + [(2, w) for w in (2, 4, 8, 16, 32)] + [(3, w) for w in (1, 2, 4, 8, 16, 32)]
                + [(4, 1)] + [(5, 1), (5, 4)] + [(6, 1)] + [(7, 1), (7, 8)] + [(8, 1)])
