"""Seeded synthetic inputs for the SpMV / CG / PageRank workloads.

This module is shared by the CUDA library's tests and benchmark and by the
CPU oracle's tests.  It only builds inputs (CSR structure, values, vectors);
it contains none of the arithmetic that the library or the oracle computes.
The generators are plain C (``gen.c``), compiled on first use with gcc, so
that multi-million-row matrices are built in seconds on any host.

Random numbers come from a counter-based SplitMix64 (Steele, Lea & Flood,
OOPSLA 2014); the exact draw order of each generator is documented in
``gen.c``.

The workload recipes (sizes, value distributions, seeds) stand in for the
paper's inputs (University of Florida matrices and the NAS CG inputs,
Section 5), which are not available here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD_DIR, "libinputs.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into a shared library next to it; returns its path."""
    src = os.path.join(_HERE, "gen.c")
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", src, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
            c = ctypes
            lib.gen_splitmix64_at.restype = c.c_uint64
            lib.gen_splitmix64_at.argtypes = [c.c_uint64, c.c_uint64]
            lib.gen_uniform_f64.restype = None
            lib.gen_uniform_f64.argtypes = [c.c_uint64, c.c_int64, c.c_double, c.c_double, f64p]
            lib.gen_uniform_f32.restype = None
            lib.gen_uniform_f32.argtypes = [c.c_uint64, c.c_int64, c.c_double, c.c_double, f32p]
            for name in ("gen_laplacian2d", "gen_laplacian3d"):
                fn = getattr(lib, name)
                fn.restype = c.c_int64
                fn.argtypes = [c.c_int32, i32p, i32p, c.c_void_p, c.c_void_p]
            lib.gen_spd_random.restype = c.c_int64
            lib.gen_spd_random.argtypes = [c.c_int32, c.c_int32, c.c_double, c.c_uint64,
                                           i32p, i32p, f64p, c.c_void_p]
            lib.gen_banded_spd.restype = c.c_int64
            lib.gen_banded_spd.argtypes = [c.c_int32, c.c_int32, c.c_double, c.c_uint64, c.c_int,
                                           i32p, i32p, f64p, c.c_void_p]
            lib.gen_rmat_transposed.restype = c.c_int64
            lib.gen_rmat_transposed.argtypes = [c.c_int32, c.c_int32, c.c_double, c.c_double,
                                                c.c_double, c.c_uint64, c.c_int,
                                                i32p, i32p, f32p, i32p]
            lib.gen_random_csr.restype = c.c_int64
            lib.gen_random_csr.argtypes = [c.c_int32, c.c_int32, c.c_int32, c.c_double,
                                           c.c_uint64, i32p, i32p, f64p]
            lib.gen_powerlaw_csr.restype = c.c_int64
            lib.gen_powerlaw_csr.argtypes = [c.c_int32, c.c_int32, c.c_int32, c.c_int32,
                                             c.c_uint64, i32p, i32p, f64p]
            _lib = lib
    return _lib


@dataclass
class CSR:
    """A CSR matrix on the host: int32 row_ptr[n+1] / col_ind[nnz], vals[nnz]."""
    n: int
    ncols: int
    row_ptr: np.ndarray
    col_ind: np.ndarray
    vals: np.ndarray
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def astype(self, dtype) -> "CSR":
        return CSR(self.n, self.ncols, self.row_ptr, self.col_ind,
                   np.ascontiguousarray(self.vals.astype(dtype)), self.name, dict(self.extra))


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def splitmix64_at(key: int, k: int) -> int:
    """Draw k of the SplitMix64 stream with key `key` (for tests of the generator)."""
    return int(_load().gen_splitmix64_at(ctypes.c_uint64(key & (2**64 - 1)), ctypes.c_uint64(k)))


def uniform(seed: int, n: int, lo: float = -1.0, hi: float = 1.0, dtype=np.float64) -> np.ndarray:
    """x_i = lo + (hi - lo) * u_i, u_i = draw i of stream `seed`."""
    lib = _load()
    if dtype == np.float32:
        out = np.empty(n, np.float32)
        lib.gen_uniform_f32(seed, n, lo, hi, out)
    else:
        out = np.empty(n, np.float64)
        lib.gen_uniform_f64(seed, n, lo, hi, out)
    return out


def laplacian2d(m: int, dtype=np.float64) -> CSR:
    """2D 5-point Laplacian, m x m grid, Dirichlet: n = m^2, nnz = 5m^2 - 4m."""
    lib = _load()
    n = m * m
    rp = np.empty(n + 1, np.int32)
    nnz_bound = 5 * n
    ci = np.empty(nnz_bound, np.int32)
    v64 = np.empty(nnz_bound, np.float64) if dtype == np.float64 else None
    v32 = np.empty(nnz_bound, np.float32) if dtype == np.float32 else None
    nnz = lib.gen_laplacian2d(m, rp, ci, _ptr(v64), _ptr(v32))
    vals = (v64 if v64 is not None else v32)[:nnz].copy()
    return CSR(n, n, rp, ci[:nnz].copy(), vals, f"laplacian2d_m{m}", {"m": m})


def laplacian3d(m: int, dtype=np.float64) -> CSR:
    """3D 7-point Laplacian, m^3 grid, Dirichlet: n = m^3, nnz = 7m^3 - 6m^2."""
    lib = _load()
    n = m ** 3
    rp = np.empty(n + 1, np.int32)
    nnz_bound = 7 * n
    ci = np.empty(nnz_bound, np.int32)
    v64 = np.empty(nnz_bound, np.float64) if dtype == np.float64 else None
    v32 = np.empty(nnz_bound, np.float32) if dtype == np.float32 else None
    nnz = lib.gen_laplacian3d(m, rp, ci, _ptr(v64), _ptr(v32))
    vals = (v64 if v64 is not None else v32)[:nnz]
    ci = ci[:nnz]
    return CSR(n, n, rp, ci, vals, f"laplacian3d_m{m}", {"m": m})


def spd_random(n: int, k: int = 90, shift: float = 20.0, seed: int = 0) -> CSR:
    """Random SPD matrix (k random columns per row, symmetrised, diagonal = row sum + shift)."""
    lib = _load()
    bound = n * (2 * k + 1)
    rp = np.empty(n + 1, np.int32)
    ci = np.empty(bound, np.int32)
    v = np.empty(bound, np.float64)
    nnz = lib.gen_spd_random(n, k, shift, seed, rp, ci, v, None)
    if nnz < 0:
        raise ValueError("gen_spd_random: bad size")
    return CSR(n, n, rp, ci[:nnz].copy(), v[:nnz].copy(), f"spd_random_n{n}_k{k}",
               {"k": k, "shift": shift, "seed": seed})


def banded_spd(n: int, w: int, shift: float = 1.0, seed: int = 0, fp32_exact: bool = True) -> CSR:
    """Symmetric full-band SPD matrix, half-bandwidth w, diagonal = row sum + shift."""
    lib = _load()
    bound = n * (2 * w + 1)
    rp = np.empty(n + 1, np.int32)
    ci = np.empty(bound, np.int32)
    v = np.empty(bound, np.float64)
    nnz = lib.gen_banded_spd(n, w, shift, seed, 1 if fp32_exact else 0, rp, ci, v, None)
    if nnz < 0:
        raise ValueError("gen_banded_spd: bad size")
    return CSR(n, n, rp, ci[:nnz].copy(), v[:nnz].copy(), f"banded_n{n}_w{w}",
               {"w": w, "shift": shift, "seed": seed, "fp32_exact": fp32_exact})


def rmat_transposed(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
                    c: float = 0.19, seed: int = 0, permute: bool = True) -> CSR:
    """Transposed R-MAT adjacency (row = destination), FP32 values 1/outdeg(source).

    extra["outdeg"] holds the out-degrees; vertices with outdeg 0 are dangling.
    """
    lib = _load()
    N = 1 << scale
    M = edge_factor * N
    rp = np.empty(N + 1, np.int32)
    ci = np.empty(M, np.int32)
    v = np.empty(M, np.float32)
    od = np.empty(N, np.int32)
    nnz = lib.gen_rmat_transposed(scale, edge_factor, a, b, c, seed, 1 if permute else 0,
                                  rp, ci, v, od)
    if nnz < 0:
        raise ValueError("gen_rmat_transposed: bad size")
    if nnz < M // 2:
        ci = ci[:nnz].copy()
        v = v[:nnz].copy()
    else:
        ci = ci[:nnz]
        v = v[:nnz]
    return CSR(N, N, rp, ci, v, f"rmat_s{scale}_ef{edge_factor}",
               {"outdeg": od, "scale": scale, "edge_factor": edge_factor, "seed": seed,
                "permute": permute})


def random_csr(n: int, ncols: int, max_len: int, empty_frac: float = 0.1, seed: int = 0) -> CSR:
    """Small random CSR with empty rows, unsorted and duplicate columns (edge cases)."""
    lib = _load()
    bound = max(1, n * max_len)
    rp = np.empty(n + 1, np.int32)
    ci = np.empty(bound, np.int32)
    v = np.empty(bound, np.float64)
    nnz = lib.gen_random_csr(n, ncols, max_len, empty_frac, seed, rp, ci, v)
    return CSR(n, ncols, rp, ci[:nnz].copy(), v[:nnz].copy(), f"random_n{n}", {"seed": seed})


def powerlaw_csr(n: int, ncols: int, max_len: int, power: int = 6, seed: int = 0) -> CSR:
    """Rows of length floor(max_len * u^power): a few very long rows, many short ones."""
    lib = _load()
    # expected nnz = max_len/(power+1) per row; bound generously by drawing sizes first
    bound = max(1, int(n * max_len / (power + 1) * 1.5) + 4 * max_len)
    while True:
        rp = np.empty(n + 1, np.int32)
        ci = np.empty(bound, np.int32)
        v = np.empty(bound, np.float64)
        # the C generator writes at most sum(len) entries; probe the lengths first
        lens_probe = _powerlaw_total(n, max_len, power, seed)
        if lens_probe <= bound:
            break
        bound = lens_probe
    nnz = lib.gen_powerlaw_csr(n, ncols, max_len, power, seed, rp, ci, v)
    return CSR(n, ncols, rp, ci[:nnz].copy(), v[:nnz].copy(), f"powerlaw_n{n}", {"seed": seed})


def _powerlaw_total(n: int, max_len: int, power: int, seed: int) -> int:
    # Replays the length draws of gen_powerlaw_csr (one draw per row, then
    # 2 draws per entry) to size the output buffers exactly.
    total = 0
    draw = 0
    for _ in range(n):
        z = splitmix64_at(seed, draw)
        draw += 1
        u = (z >> 11) * (1.0 / 9007199254740992.0)
        f = 1.0
        for _q in range(power):
            f *= u
        ln = int(max_len * f)
        total += ln
        draw += 2 * ln
    return total


# --- the workloads -----------------------------------------------------------

def workload_laplacian2d_spmv(m: int = 64):
    """2D 5-point Laplacian on an m x m grid (FP64), x uniform in [-1, 1] from seed 0."""
    A = laplacian2d(m)
    x = uniform(0, A.ncols)
    return A, x


def workload_spd_cg(n: int = 75_000, k: int = 90, seed: int = 0):
    """Random SPD (k random columns per row, ~2k+1 nnz/row after symmetrising), b = ones."""
    A = spd_random(n, k, 20.0, seed)
    b = np.ones(n, np.float64)
    return A, b


def workload_rmat_pagerank(scale: int = 22, edge_factor: int = 16, seed: int = 0,
                           permute: bool = True):
    """R-MAT graph, transposed CSR with FP32 values 1/outdeg (dangling vertices have none)."""
    return rmat_transposed(scale, edge_factor, 0.57, 0.19, 0.19, seed, permute)


def workload_poisson3d_ir(m: int = 192, seed: int = 1):
    """3D 7-point Poisson on an m^3 grid, FP32 values (exact), b uniform in [-1, 1]."""
    A = laplacian3d(m, np.float32)
    b = uniform(seed, A.n)
    return A, b
