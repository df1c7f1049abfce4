"""Thin ctypes binding of liblilac.so (include/lilac.h).

The functions keep the C names and arguments; they only marshal arguments
(pointers of numpy arrays or torch tensors, the current CUDA stream) and
turn a non-OK status into ``LilacError``.  All computation happens in the
CUDA library.  There is no CPU fallback: if the library is missing, loading
fails with an error that says how to build it.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

LILAC_OK = 0
LILAC_ERR_INVALID_ARG = 1
LILAC_ERR_INVALID_CSR = 2
LILAC_ERR_OOM = 3
LILAC_ERR_BUDGET = 4
LILAC_ERR_CUDA = 5
LILAC_ERR_BREAKDOWN = 6
LILAC_ERR_NOT_CONVERGED = 7
LILAC_ERR_TIMEOUT = 8
LILAC_ERR_DTYPE = 9
LILAC_ERR_UNSUPPORTED = 10

LILAC_F64, LILAC_F32 = 0, 1
LILAC_MEM_HOST, LILAC_MEM_DEVICE = 0, 1
LILAC_VARIANT_AUTO, LILAC_VARIANT_SCALAR, LILAC_VARIANT_VECTOR, LILAC_VARIANT_STAGED, \
    LILAC_VARIANT_MERGE, LILAC_VARIANT_SLAB, LILAC_VARIANT_JDS, LILAC_VARIANT_SELL, \
    LILAC_VARIANT_HUB = 0, 1, 2, 3, 4, 5, 6, 7, 8
LILAC_CREATE_NO_TUNE = 0x1

VARIANT_NAMES = {1: "scalar", 2: "vector", 3: "staged", 4: "merge", 5: "slab", 6: "jds",
                 7: "sell", 8: "hub"}

# every symbol include/lilac.h declares (checked by the tests)
EXPORTS = (
    "lilac_csr_create", "lilac_csr_update_values", "lilac_csr_destroy", "lilac_csr_info",
    "lilac_csr_set_variant", "lilac_spmv", "lilac_cg_opts_default", "lilac_cg",
    "lilac_pagerank", "lilac_csr_reset_error", "lilac_status_string", "lilac_last_error",
    "lilac_version", "lilac_spmv_noalloc", "lilac_csr_profile", "lilac_batch_create",
    "lilac_batch_destroy", "lilac_batch_spmv", "lilac_batch_cg", "lilac_server_opts_default",
    "lilac_server_create", "lilac_server_destroy", "lilac_server_add_matrix",
    "lilac_server_submit", "lilac_server_step", "lilac_server_poll", "lilac_server_stats",
    "lilac_server_now", "lilac_csr_jds", "lilac_bfs", "lilac_spmv_host",
    "lilac_host_cache_stats", "lilac_host_cache_clear", "lilac_spmm", "lilac_debug_inject",
    "lilac_csr_tune_table",
)

LILAC_INJECT_ALLOC_FAIL, LILAC_INJECT_SKIP_COPY, LILAC_INJECT_SKIP_BARRIER = 1, 2, 3

LILAC_LAYOUT_ROWS, LILAC_LAYOUT_VECTORS = 0, 1

LILAC_HOST_CACHED, LILAC_HOST_NAIVE = 0, 1

LILAC_REQ_SPMV, LILAC_REQ_CG = 0, 1


class lilac_csr_info_t(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("ncols", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("dtype", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("vector_width", ctypes.c_int32), ("max_row_len", ctypes.c_int32),
                ("empty_rows", ctypes.c_int32), ("num_tiles", ctypes.c_int32),
                ("num_long_rows", ctypes.c_int32), ("sm_count", ctypes.c_int32),
                ("mean_row_len", ctypes.c_double), ("std_row_len", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("h2d_bytes", ctypes.c_int64),
                ("active_variant", ctypes.c_int32), ("sell_split_rows", ctypes.c_int32),
                ("sell_padded_nnz", ctypes.c_int64), ("spmv_kernels", ctypes.c_int32)]


class lilac_cg_opts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("rtol", ctypes.c_double),
                ("precision", ctypes.c_int32), ("inner_rtol", ctypes.c_double),
                ("inner_max_iter", ctypes.c_int32), ("use_x0", ctypes.c_int32),
                ("true_residual", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("ru_delta", ctypes.c_double)]


class lilac_cg_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("status", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("rel_res", ctypes.c_double), ("true_rel_res", ctypes.c_double),
                ("spmv_ms", ctypes.c_double), ("spmv_launches", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int32)]


class lilac_server_opts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_active", ctypes.c_int32),
                ("iters_per_round", ctypes.c_int32), ("tune", ctypes.c_int32)]


class lilac_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("matrix", ctypes.c_int32), ("nvec", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("rtol", ctypes.c_double),
                ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("tag", ctypes.c_int64),
                ("precision", ctypes.c_int32), ("pad", ctypes.c_int32)]


class lilac_completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_int64), ("status", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("rel_res", ctypes.c_double), ("arrival", ctypes.c_double),
                ("finish", ctypes.c_double), ("admitted", ctypes.c_double),
                ("rounds", ctypes.c_int32), ("pad", ctypes.c_int32)]


class lilac_server_stats_t(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("submitted", "completed", "rounds", "uploads",
                                              "upload_bytes", "evictions", "budget_waits",
                                              "resident_bytes", "pool_bytes")] + \
               [("queued", ctypes.c_int32), ("active", ctypes.c_int32)]


class lilac_host_stats_t(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_int64), ("uploads", ctypes.c_int64),
                ("value_updates", ctypes.c_int64), ("structure_changes", ctypes.c_int64),
                ("hits", ctypes.c_int64), ("hashed_bytes", ctypes.c_int64),
                ("resident", ctypes.c_int32), ("pad", ctypes.c_int32)]


class LilacError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib().lilac_status_string(status).decode()
        detail = _lib().lilac_last_error().decode()
        super().__init__(f"{where}: {msg} ({status})" + (f": {detail}" if detail else ""))


_LIB = None


def library_path() -> str:
    return _build.LIB


def _lib():
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build it with `python -m paper_2001_07938_gb300.build` "
                "(the library is CUDA-only; there is no CPU path)")
        lib = ctypes.CDLL(path)
        c = ctypes
        vp, i32, i64, u32, dbl = c.c_void_p, c.c_int32, c.c_int64, c.c_uint32, c.c_double
        st = c.c_int
        lib.lilac_csr_create.argtypes = [i32, i32, i64, vp, vp, vp, c.c_int, c.c_int, u32, vp,
                                         c.POINTER(vp)]
        lib.lilac_csr_update_values.argtypes = [vp, vp, c.c_int, vp]
        lib.lilac_csr_destroy.argtypes = [vp]
        lib.lilac_csr_info.argtypes = [vp, c.POINTER(lilac_csr_info_t)]
        lib.lilac_csr_set_variant.argtypes = [vp, i32, i32]
        lib.lilac_csr_tune_table.argtypes = [vp, i32, vp, vp, vp, c.POINTER(i32)]
        lib.lilac_csr_jds.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.lilac_bfs.argtypes = [vp, i32, vp, c.c_int, c.POINTER(i32), vp]
        lib.lilac_spmv_host.argtypes = [i32, i32, i64, vp, vp, vp, c.c_int, vp, vp, c.c_uint64,
                                        u32, vp]
        lib.lilac_host_cache_stats.argtypes = [c.POINTER(lilac_host_stats_t)]
        lib.lilac_host_cache_clear.argtypes = []
        lib.lilac_spmm.argtypes = [vp, vp, vp, i32, i32, c.c_int, vp]
        lib.lilac_debug_inject.argtypes = [vp, i32, i64]
        lib.lilac_spmv.argtypes = [vp, vp, vp, c.c_int, vp]
        lib.lilac_cg_opts_default.argtypes = [c.POINTER(lilac_cg_opts)]
        lib.lilac_cg_opts_default.restype = None
        lib.lilac_cg.argtypes = [vp, vp, vp, c.c_int, c.POINTER(lilac_cg_opts),
                                 c.POINTER(lilac_cg_info), vp]
        lib.lilac_pagerank.argtypes = [vp, vp, i32, i32, dbl, vp, c.c_int, vp]
        lib.lilac_csr_reset_error.argtypes = [vp]
        lib.lilac_spmv_noalloc.argtypes = [i32, i32, i64, vp, vp, vp, c.c_int, vp, vp, vp]
        lib.lilac_csr_profile.argtypes = [vp, i32, c.POINTER(dbl), c.POINTER(i64)]
        lib.lilac_batch_create.argtypes = [c.POINTER(vp)]
        lib.lilac_batch_destroy.argtypes = [vp]
        lib.lilac_batch_spmv.argtypes = [vp, i32, c.POINTER(vp), c.POINTER(vp), c.POINTER(vp), vp]
        lib.lilac_batch_cg.argtypes = [vp, i32, c.POINTER(vp), c.POINTER(vp), c.POINTER(vp), i32,
                                       dbl, i32, c.POINTER(lilac_cg_info), vp]
        lib.lilac_server_opts_default.argtypes = [c.POINTER(lilac_server_opts)]
        lib.lilac_server_opts_default.restype = None
        lib.lilac_server_create.argtypes = [c.POINTER(lilac_server_opts), vp, c.POINTER(vp)]
        lib.lilac_server_destroy.argtypes = [vp]
        lib.lilac_server_add_matrix.argtypes = [vp, i32, i32, i64, vp, vp, vp, c.POINTER(i32)]
        lib.lilac_server_submit.argtypes = [vp, c.POINTER(lilac_request)]
        lib.lilac_server_step.argtypes = [vp, c.POINTER(i32)]
        lib.lilac_server_poll.argtypes = [vp, c.POINTER(lilac_completion), i32, c.POINTER(i32)]
        lib.lilac_server_stats.argtypes = [vp, c.POINTER(lilac_server_stats_t)]
        lib.lilac_server_now.argtypes = []
        lib.lilac_server_now.restype = dbl
        lib.lilac_status_string.argtypes = [c.c_int]
        lib.lilac_status_string.restype = c.c_char_p
        lib.lilac_last_error.argtypes = []
        lib.lilac_last_error.restype = c.c_char_p
        lib.lilac_version.argtypes = []
        lib.lilac_version.restype = i32
        for name in ("lilac_csr_create", "lilac_csr_update_values", "lilac_csr_destroy",
                     "lilac_csr_info", "lilac_csr_set_variant", "lilac_spmv", "lilac_cg",
                     "lilac_pagerank", "lilac_csr_reset_error", "lilac_spmv_noalloc",
                     "lilac_csr_profile", "lilac_batch_create", "lilac_batch_destroy",
                     "lilac_batch_spmv", "lilac_batch_cg", "lilac_server_create",
                     "lilac_server_destroy", "lilac_server_add_matrix", "lilac_server_submit",
                     "lilac_server_step", "lilac_server_poll", "lilac_server_stats",
                     "lilac_csr_jds", "lilac_bfs", "lilac_spmv_host", "lilac_host_cache_stats",
                     "lilac_host_cache_clear", "lilac_spmm", "lilac_debug_inject",
                     "lilac_csr_tune_table"):
            getattr(lib, name).restype = st
        _LIB = lib
    return _LIB


def load():
    """Load the library (raises if it was not built)."""
    return _lib()


def _check(status: int, where: str, ok=(LILAC_OK,)):
    if status not in ok:
        raise LilacError(status, where)
    return status


# --- argument marshalling ----------------------------------------------------

def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr_where(a):
    """(pointer, LILAC_MEM_*) of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None, LILAC_MEM_DEVICE
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), (LILAC_MEM_DEVICE if a.is_cuda else LILAC_MEM_HOST)
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, LILAC_MEM_HOST
    raise TypeError(f"unsupported array type {type(a)}")


def current_stream():
    """cudaStream_t of torch's current stream (0 without torch/CUDA)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


def _dtype_code(dt) -> int:
    name = str(dt)
    if name.endswith("float64") or name == "double":
        return LILAC_F64
    if name.endswith("float32") or name == "float":
        return LILAC_F32
    raise ValueError(f"values must be float64 or float32, got {dt}")


# --- the C entry points, same names -----------------------------------------

def lilac_csr_create(rows, ncols, nnz, row_ptr, col_ind, vals, dtype, where, flags=0, stream=None):
    h = ctypes.c_void_p()
    _check(_lib().lilac_csr_create(rows, ncols, nnz, row_ptr, col_ind, vals, dtype, where, flags,
                                   stream if stream is not None else current_stream(),
                                   ctypes.byref(h)), "lilac_csr_create")
    return h


def lilac_csr_update_values(A, vals, where, stream=None):
    _check(_lib().lilac_csr_update_values(A, vals, where,
                                          stream if stream is not None else current_stream()),
           "lilac_csr_update_values")


def lilac_csr_destroy(A):
    _check(_lib().lilac_csr_destroy(A), "lilac_csr_destroy")


def lilac_csr_info(A) -> dict:
    info = lilac_csr_info_t()
    _check(_lib().lilac_csr_info(A, ctypes.byref(info)), "lilac_csr_info")
    return {f: getattr(info, f) for f, _ in lilac_csr_info_t._fields_}


def lilac_csr_set_variant(A, variant, vector_width=0):
    _check(_lib().lilac_csr_set_variant(A, variant, vector_width), "lilac_csr_set_variant")


def lilac_csr_tune_table(A):
    """The autotuner's trial: a list of {variant, width, ms} per candidate."""
    n = ctypes.c_int32(0)
    _check(_lib().lilac_csr_tune_table(A, 0, None, None, None, ctypes.byref(n)),
           "lilac_csr_tune_table")
    m = n.value
    v = (ctypes.c_int32 * max(1, m))()
    w = (ctypes.c_int32 * max(1, m))()
    t = (ctypes.c_float * max(1, m))()
    _check(_lib().lilac_csr_tune_table(A, m, v, w, t, ctypes.byref(n)), "lilac_csr_tune_table")
    return [{"variant": int(v[i]), "width": int(w[i]), "ms": float(t[i])} for i in range(m)]


def lilac_csr_jds(A, perm, jd_ptr, col_ind, vals, nzcnt):
    """Copy the handle's JDS form into host numpy arrays (None entries skipped)."""
    p = [a.ctypes.data if a is not None else None for a in (perm, jd_ptr, col_ind, vals, nzcnt)]
    _check(_lib().lilac_csr_jds(A, *p), "lilac_csr_jds")


def lilac_spmv_host(rows, ncols, nnz, row_ptr, col_ind, vals, dtype, x, y, version=0,
                    mode=LILAC_HOST_CACHED, stream=None):
    """y = A x on host arrays with library-side marshaling (pointers as ints)."""
    _check(_lib().lilac_spmv_host(rows, ncols, nnz, row_ptr, col_ind, vals, dtype, x, y, version,
                                  mode, stream if stream is not None else current_stream()),
           "lilac_spmv_host")


def lilac_host_cache_stats() -> dict:
    st = lilac_host_stats_t()
    _check(_lib().lilac_host_cache_stats(ctypes.byref(st)), "lilac_host_cache_stats")
    return {f: getattr(st, f) for f, _ in lilac_host_stats_t._fields_ if f != "pad"}


def lilac_host_cache_clear():
    _check(_lib().lilac_host_cache_clear(), "lilac_host_cache_clear")


def spmv_host(A, x, y, version=0, naive=False):
    """Host-convention SpMV of a CSR record (numpy row_ptr/col_ind/vals, x, y)."""
    lilac_spmv_host(A.n, A.ncols, A.nnz, A.row_ptr.ctypes.data, A.col_ind.ctypes.data,
                    A.vals.ctypes.data, _dtype_code(A.vals.dtype), x.ctypes.data, y.ctypes.data,
                    version, LILAC_HOST_NAIVE if naive else LILAC_HOST_CACHED)
    return y


def lilac_debug_inject(A, what, arg=0):
    _check(_lib().lilac_debug_inject(A, what, arg), "lilac_debug_inject")


def lilac_spmm(A, X, Y, k, layout, where, stream=None):
    _check(_lib().lilac_spmm(A, X, Y, k, layout, where,
                             stream if stream is not None else current_stream()), "lilac_spmm")


def lilac_bfs(A, source, level, where, stream=None):
    """BFS levels from `source` on a transposed adjacency handle; returns the depth."""
    d = ctypes.c_int32()
    _check(_lib().lilac_bfs(A, source, level, where, ctypes.byref(d),
                            stream if stream is not None else current_stream()), "lilac_bfs")
    return d.value


def lilac_spmv(A, x, y, where, stream=None):
    _check(_lib().lilac_spmv(A, x, y, where, stream if stream is not None else current_stream()),
           "lilac_spmv")


def lilac_cg_opts_default() -> lilac_cg_opts:
    o = lilac_cg_opts()
    _lib().lilac_cg_opts_default(ctypes.byref(o))
    return o


def lilac_cg(A, b, x, where, opts=None, want_info=True, stream=None, raise_on=None):
    info = lilac_cg_info()
    st = _lib().lilac_cg(A, b, x, where, ctypes.byref(opts) if opts is not None else None,
                         ctypes.byref(info) if want_info else None,
                         stream if stream is not None else current_stream())
    ok = (LILAC_OK, LILAC_ERR_NOT_CONVERGED, LILAC_ERR_BREAKDOWN) if raise_on is None else raise_on
    _check(st, "lilac_cg", ok)
    return st, info


def lilac_pagerank(A, x, init_uniform, iters, damping, l1_per_iter, where, stream=None):
    _check(_lib().lilac_pagerank(A, x, init_uniform, iters, damping, l1_per_iter, where,
                                 stream if stream is not None else current_stream()),
           "lilac_pagerank")


class Batch:
    """Owns a lilac_batch context (batched SpMV / CG over FP64 or FP32 handles)."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(_lib().lilac_batch_create(ctypes.byref(h)), "lilac_batch_create")
        self.handle = h

    @staticmethod
    def _ptrs(seq):
        arr = (ctypes.c_void_p * max(1, len(seq)))()
        for i, a in enumerate(seq):
            arr[i] = a if isinstance(a, int) else _ptr_where(a)[0]
        return arr

    def spmv(self, mats, xs, ys, stream=None):
        n = len(mats)
        hs = self._ptrs([m.handle.value for m in mats])
        _check(_lib().lilac_batch_spmv(self.handle, n, hs, self._ptrs(xs), self._ptrs(ys),
                                       stream if stream is not None else current_stream()),
               "lilac_batch_spmv")

    def cg(self, mats, bs, xs, max_iter=1000, rtol=1e-10, precision=0, stream=None):
        n = len(mats)
        infos = (lilac_cg_info * max(1, n))()
        st = _lib().lilac_batch_cg(self.handle, n, self._ptrs([m.handle.value for m in mats]),
                                   self._ptrs(bs), self._ptrs(xs), max_iter, rtol, precision, infos,
                                   stream if stream is not None else current_stream())
        _check(st, "lilac_batch_cg", (LILAC_OK, LILAC_ERR_NOT_CONVERGED, LILAC_ERR_BREAKDOWN))
        return st, [infos[i] for i in range(n)]

    def close(self):
        if getattr(self, "handle", None):
            _lib().lilac_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owns a lilac_server (continuous batching of SpMV / CG requests)."""

    def __init__(self, hbm_budget_bytes=None, max_active=None, iters_per_round=None, tune=None,
                 stream=None):
        o = lilac_server_opts()
        _lib().lilac_server_opts_default(ctypes.byref(o))
        if hbm_budget_bytes is not None:
            o.hbm_budget_bytes = int(hbm_budget_bytes)
        if max_active is not None:
            o.max_active = int(max_active)
        if iters_per_round is not None:
            o.iters_per_round = int(iters_per_round)
        if tune is not None:
            o.tune = int(tune)
        h = ctypes.c_void_p()
        _check(_lib().lilac_server_create(ctypes.byref(o), stream if stream is not None
                                          else current_stream(), ctypes.byref(h)),
               "lilac_server_create")
        self.handle = h
        self._keep = {}  # host arrays the server reads later

    def add_matrix(self, A):
        rp = np.ascontiguousarray(A.row_ptr, np.int32)
        ci = np.ascontiguousarray(A.col_ind, np.int32)
        v = np.ascontiguousarray(A.vals, np.float64)
        mid = ctypes.c_int32()
        _check(_lib().lilac_server_add_matrix(self.handle, A.n, A.ncols, A.nnz, rp.ctypes.data,
                                              ci.ctypes.data, v.ctypes.data, ctypes.byref(mid)),
               "lilac_server_add_matrix")
        self._keep[("m", mid.value)] = (rp, ci, v)
        return mid.value

    def submit(self, kind, matrix, inp, out, tag, nvec=1, max_iter=1000, rtol=1e-10, precision=0):
        r = lilac_request(kind, matrix, nvec, max_iter, rtol, inp.ctypes.data, out.ctypes.data, tag,
                          precision, 0)
        _check(_lib().lilac_server_submit(self.handle, ctypes.byref(r)), "lilac_server_submit")
        self._keep[("r", tag)] = (inp, out)

    def step(self):
        n = ctypes.c_int32()
        _check(_lib().lilac_server_step(self.handle, ctypes.byref(n)), "lilac_server_step")
        return n.value

    def poll(self, max_n=4096):
        buf = (lilac_completion * max_n)()
        n = ctypes.c_int32()
        _check(_lib().lilac_server_poll(self.handle, buf, max_n, ctypes.byref(n)), "lilac_server_poll")
        out = []
        for i in range(n.value):
            c = buf[i]
            out.append({"tag": c.tag, "status": c.status, "iters": c.iters, "rel_res": c.rel_res,
                        "arrival": c.arrival, "finish": c.finish, "admitted": c.admitted,
                        "rounds": c.rounds})
            self._keep.pop(("r", c.tag), None)
        return out

    def stats(self):
        st = lilac_server_stats_t()
        _check(_lib().lilac_server_stats(self.handle, ctypes.byref(st)), "lilac_server_stats")
        return {f: getattr(st, f) for f, _ in lilac_server_stats_t._fields_}

    @staticmethod
    def now():
        return float(_lib().lilac_server_now())

    def close(self):
        if getattr(self, "handle", None):
            _lib().lilac_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lilac_csr_profile(A, enable):
    """Start (enable=True) or stop SpMV launch timing; returns (ms, launches) so far."""
    ms, n = ctypes.c_double(0.0), ctypes.c_int64(0)
    _check(_lib().lilac_csr_profile(A, int(enable), ctypes.byref(ms), ctypes.byref(n)),
           "lilac_csr_profile")
    return ms.value, n.value


def lilac_spmv_noalloc(rows, ncols, nnz, row_ptr, col_ind, vals, dtype, x, y, stream=None):
    """y = A x on caller-held device CSR arrays, with no device allocation."""
    _check(_lib().lilac_spmv_noalloc(rows, ncols, nnz, row_ptr, col_ind, vals, dtype, x, y,
                                     stream if stream is not None else current_stream()),
           "lilac_spmv_noalloc")


def lilac_csr_reset_error(A):
    _check(_lib().lilac_csr_reset_error(A), "lilac_csr_reset_error")


def lilac_status_string(s: int) -> str:
    return _lib().lilac_status_string(s).decode()


def lilac_last_error() -> str:
    return _lib().lilac_last_error().decode()


def lilac_version() -> int:
    return int(_lib().lilac_version())


# --- a small object wrapper ----------------------------------------------------

class CsrMatrix:
    """Owns one lilac_csr handle.  Arrays may be numpy (host) or torch (host/device)."""

    def __init__(self, row_ptr, col_ind, vals, ncols: int = -1, flags: int = 0, stream=None):
        rp, where = _ptr_where(row_ptr)
        ci, w2 = _ptr_where(col_ind)
        va, w3 = _ptr_where(vals)
        if len(col_ind) and len({where, w2, w3}) != 1:
            raise ValueError("row_ptr, col_ind and vals must all be on the host or all on the device")
        rows = len(row_ptr) - 1
        nnz = len(col_ind)
        self.dtype = _dtype_code(vals.dtype)
        self.handle = lilac_csr_create(rows, ncols, nnz, rp, ci if nnz else None,
                                       va if nnz else None, self.dtype, where, flags, stream)
        self.rows = rows

    @classmethod
    def from_csr(cls, A, flags: int = 0, dtype=None):
        """From a host CSR record with row_ptr / col_ind / vals / ncols fields."""
        vals = A.vals if dtype is None else np.ascontiguousarray(A.vals.astype(dtype))
        return cls(np.ascontiguousarray(A.row_ptr, np.int32),
                   np.ascontiguousarray(A.col_ind, np.int32), vals, A.ncols, flags)

    def info(self) -> dict:
        return lilac_csr_info(self.handle)

    def set_variant(self, variant: int, width: int = 0):
        lilac_csr_set_variant(self.handle, variant, width)

    def tune_table(self) -> list:
        return lilac_csr_tune_table(self.handle)

    def spmm(self, X, Y, k, layout=LILAC_LAYOUT_ROWS, stream=None):
        """Y = A X for k vectors (numpy host or torch arrays, flat or 2D)."""
        px, wx = _ptr_where(X)
        py, wy = _ptr_where(Y)
        if wx != wy:
            raise ValueError("X and Y must both be host or both device")
        lilac_spmm(self.handle, px, py, int(k), layout, wx, stream)
        return Y

    def bfs(self, source, level, stream=None):
        """Levels from `source` into `level` (int32, host numpy or device torch); returns depth."""
        p, w = _ptr_where(level)
        return lilac_bfs(self.handle, int(source), p, w, stream)

    def jds(self):
        """The handle's JDS form: (perm, jd_ptr, col_ind, vals, nzcnt) as numpy arrays."""
        inf = self.info()
        n, nnz = inf["rows"], inf["nnz"]
        vals = np.empty(nnz, np.float64 if inf["dtype"] == LILAC_F64 else np.float32)
        out = (np.empty(n, np.int32), np.empty(inf["max_row_len"] + 1, np.int32),
               np.empty(nnz, np.int32), vals, np.empty(n, np.int32))
        lilac_csr_jds(self.handle, *out)
        return out

    def spmv(self, x, y, stream=None):
        px, wx = _ptr_where(x)
        py, wy = _ptr_where(y)
        if wx != wy:
            raise ValueError("x and y must both be host or both device")
        lilac_spmv(self.handle, px, py, wx, stream)
        return y

    def cg(self, b, x, *, max_iter=1000, rtol=1e-10, precision=0, inner_rtol=1e-5,
           inner_max_iter=1000, use_x0=False, true_residual=True, use_graph=True,
           check_every=32, want_info=True, profile=False, ru_delta=0.1, stream=None):
        o = lilac_cg_opts_default()
        o.profile = int(profile)
        o.ru_delta = ru_delta
        o.max_iter, o.rtol, o.precision = max_iter, rtol, precision
        o.inner_rtol, o.inner_max_iter = inner_rtol, inner_max_iter
        o.use_x0, o.true_residual, o.use_graph = int(use_x0), int(true_residual), int(use_graph)
        o.check_every = check_every
        pb, wb = _ptr_where(b)
        px, wx = _ptr_where(x)
        if wb != wx:
            raise ValueError("b and x must both be host or both device")
        st, info = lilac_cg(self.handle, pb, px, wb, o, want_info, stream)
        return st, info

    def pagerank(self, x, iters=20, damping=0.85, init_uniform=True, want_l1=True, stream=None):
        px, wx = _ptr_where(x)
        l1 = np.zeros(max(iters, 1), np.float64) if want_l1 else None
        lilac_pagerank(self.handle, px, int(init_uniform), iters, damping,
                       l1.ctypes.data if l1 is not None else None, wx, stream)
        return l1[:iters] if l1 is not None else None

    def close(self):
        if getattr(self, "handle", None):
            lilac_csr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
