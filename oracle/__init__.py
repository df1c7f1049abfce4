"""CPU ORACLE -- test infrastructure only.

Plain sequential FP64 implementations (``lilac_oracle.c``) of what the CUDA
library computes: CSR SpMV, dot product, conjugate gradient, PageRank power
iteration, CSR->JDS conversion with JDS SpMV, and BFS levels.  Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the library
(``paper_2001_07938_gb300``) and never imports it.

FP32 inputs are promoted to FP64 before the C code sees them, so every oracle
result is an FP64 computation of the given (possibly FP32-rounded) matrix.

Each function below says which part of the paper it follows; the C file
holds the definitions themselves.  Every function is pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_*.py`` against values fixed by
the paper (its CSR and JDS worked example) or by mathematics (dense brute
force, Laplacian eigenpairs, CG finite termination, a dense Cholesky solve,
PageRank invariants and its closed-form fixed point).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD_DIR, "liblilac_oracle.so")
_SO_OMP = os.path.join(_BUILD_DIR, "liblilac_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

CG_CONVERGED, CG_MAXITER, CG_BREAKDOWN = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2, sequential: the paper's CPU baseline is
    sequential code built at -O2, Section 6)."""
    src = os.path.join(_HERE, "lilac_oracle.c")
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def build_parallel(force: bool = False):
    """The same source built with OpenMP (the SpMV row loop shared among the
    host's cores, static schedule; results bitwise those of the sequential
    build).  None when the compiler has no OpenMP."""
    src = os.path.join(_HERE, "lilac_oracle.c")
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_SO_OMP) or os.path.getmtime(_SO_OMP) < os.path.getmtime(src):
        tmp = _SO_OMP + f".tmp{os.getpid()}"
        p = subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", src, "-o",
                            tmp, "-lm"], capture_output=True)
        if p.returncode != 0:
            return None
        os.replace(tmp, _SO_OMP)
    return _SO_OMP


def threads(parallel: bool = True) -> int:
    """Threads an oracle SpMV uses in the given build."""
    return int(_load(parallel).oracle_threads())


def _load(parallel: bool = False):
    global _lib, _lib_omp
    with _lock:
        if parallel and _lib_omp is None:
            path = build_parallel()
            if path is None:
                raise RuntimeError("the C compiler has no OpenMP: no all-cores oracle")
            _lib_omp = _declare(ctypes.CDLL(path))
        if parallel:
            return _lib_omp
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _declare(lib):
    c = ctypes
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    lib.oracle_spmv.restype = None
    lib.oracle_spmv.argtypes = [c.c_int32, i32p, i32p, f64p, f64p, f64p]
    lib.oracle_dot.restype = c.c_double
    lib.oracle_dot.argtypes = [c.c_int64, f64p, f64p]
    lib.oracle_csr_ncols.restype = c.c_int32
    lib.oracle_csr_ncols.argtypes = [c.c_int64, i32p]
    lib.oracle_cg.restype = c.c_int
    lib.oracle_cg.argtypes = [c.c_int32, i32p, i32p, f64p, f64p, f64p, c.c_int32,
                              c.c_double, c.POINTER(c.c_int32), c.c_void_p]
    lib.oracle_pagerank.restype = None
    lib.oracle_pagerank.argtypes = [c.c_int32, i32p, i32p, f64p, c.c_void_p, c.c_int32,
                                    c.c_double, f64p, c.c_void_p]
    lib.oracle_csr_to_jds.restype = c.c_int32
    lib.oracle_csr_to_jds.argtypes = [c.c_int32, i32p, i32p, f64p, i32p, i32p, i32p,
                                      i32p, f64p]
    lib.oracle_jds_spmv.restype = None
    lib.oracle_jds_spmv.argtypes = [c.c_int32, c.c_int32, i32p, i32p, i32p, f64p, f64p,
                                    f64p]
    lib.oracle_bfs_levels.restype = c.c_int32
    lib.oracle_bfs_levels.argtypes = [c.c_int32, i32p, i32p, c.c_int32, i32p]
    lib.oracle_threads.restype = c.c_int32
    lib.oracle_threads.argtypes = []
    return lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def spmv(row_ptr, col_ind, vals, x, parallel: bool = False) -> np.ndarray:
    """y = A x, CSR (Section 3.2), FP64, ascending-j accumulation."""
    rp = _i32(row_ptr)
    n = rp.size - 1
    y = np.empty(n, np.float64)
    _load(parallel).oracle_spmv(n, rp, _i32(col_ind), _f64(vals), _f64(x), y)
    return y


def spmv_abs_bound(row_ptr, col_ind, vals, x) -> np.ndarray:
    """(|A| |x|)_i, the scale of the componentwise SpMV error bound."""
    return spmv(row_ptr, col_ind, np.abs(_f64(vals)), np.abs(_f64(x)))


def dot(a, b) -> float:
    """sum_i a_i b_i in ascending i (Section 4.1, dotproduct)."""
    a = _f64(a)
    return float(_load().oracle_dot(a.size, a, _f64(b)))


def csr_ncols(col_ind) -> int:
    """max(col_ind) + 1, the cached 'Maximum' invariant of Section 3.3."""
    ci = _i32(col_ind)
    return int(_load().oracle_csr_ncols(ci.size, ci))


def cg(row_ptr, col_ind, vals, b, x0=None, max_iter=1000, rtol=0.0, want_hist=False,
       parallel: bool = False):
    """Hestenes-Stiefel CG (the NAS CG solver, Section 2).  Returns (x, iters, status[, rr_hist])."""
    rp = _i32(row_ptr)
    n = rp.size - 1
    x = np.zeros(n, np.float64) if x0 is None else _f64(x0).copy()
    it = ctypes.c_int32(0)
    hist = np.zeros(max_iter + 1, np.float64) if want_hist else None
    st = _load(parallel).oracle_cg(n, rp, _i32(col_ind), _f64(vals), _f64(b), x, int(max_iter),
                           float(rtol), ctypes.byref(it),
                           None if hist is None else hist.ctypes.data_as(ctypes.c_void_p))
    if want_hist:
        return x, it.value, st, hist[: it.value + 1]
    return x, it.value, st


def pagerank(row_ptr, col_ind, vals, iters=20, damping=0.85, x0=None, parallel: bool = False):
    """PageRank power iteration on the transposed link matrix (Section 5). Returns (x, l1[iters])."""
    rp = _i32(row_ptr)
    n = rp.size - 1
    x = np.empty(n, np.float64)
    l1 = np.empty(max(iters, 1), np.float64)
    x0a = None if x0 is None else _f64(x0)
    _load(parallel).oracle_pagerank(n, rp, _i32(col_ind), _f64(vals),
                            None if x0a is None else x0a.ctypes.data_as(ctypes.c_void_p),
                            int(iters), float(damping), x, l1.ctypes.data_as(ctypes.c_void_p))
    return x, l1[:iters]


def csr_to_jds(row_ptr, col_ind, vals):
    """CSR -> JDS (Section 3.2). Returns dict(perm, nzcnt, jd_ptr, col_ind, val)."""
    rp = _i32(row_ptr)
    n = rp.size - 1
    nnz = int(rp[-1])
    maxlen = int(np.max(np.diff(rp))) if n > 0 else 0
    perm = np.empty(max(n, 1), np.int32)
    nzcnt = np.empty(max(n, 1), np.int32)
    jd_ptr = np.empty(maxlen + 1, np.int32)
    jc = np.empty(max(nnz, 1), np.int32)
    jv = np.empty(max(nnz, 1), np.float64)
    nd = _load().oracle_csr_to_jds(n, rp, _i32(col_ind), _f64(vals), perm, nzcnt, jd_ptr, jc, jv)
    return {"perm": perm[:n], "nzcnt": nzcnt[:n], "jd_ptr": jd_ptr[: nd + 1],
            "col_ind": jc[:nnz], "val": jv[:nnz], "ndiag": int(nd)}


def jds_spmv(perm, jd_ptr, jd_col, jd_val, x) -> np.ndarray:
    """y = A x with A in JDS (Section 3.2)."""
    perm = _i32(perm)
    n = perm.size
    jd_ptr = _i32(jd_ptr)
    y = np.empty(max(n, 1), np.float64)
    _load().oracle_jds_spmv(n, jd_ptr.size - 1, perm if n else np.zeros(1, np.int32), jd_ptr,
                            _i32(jd_col) if len(jd_col) else np.zeros(1, np.int32),
                            _f64(jd_val) if len(jd_val) else np.zeros(1),
                            _f64(x) if len(x) else np.zeros(1), y)
    return y[:n]


def bfs_levels(row_ptr, col_ind, src: int) -> np.ndarray:
    """BFS levels from src (-1 unreachable), queue-based (GAP BFS, Section 5)."""
    rp = _i32(row_ptr)
    n = rp.size - 1
    lev = np.empty(max(n, 1), np.int32)
    ci = _i32(col_ind) if len(col_ind) else np.zeros(1, np.int32)
    _load().oracle_bfs_levels(n, rp, ci, int(src), lev)
    return lev[:n]
