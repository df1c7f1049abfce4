#!/usr/bin/env python
"""Benchmark of the GB300 SpMV / CG / PageRank library (one JSON line on stdout).

Default workload (cg75k): unpreconditioned FP64 CG, 75 iterations, on a
random SPD CSR matrix with n = 75,000 and ~181 nonzeros per row at uniformly
random columns (values U[0,1), symmetrised, diagonal = row sum + 20),
b = ones, int32 indices.  One step = one full solve through lilac_cg (device
buffers, resident matrix); the metric is solves/s, and the roofline object
reports the fused SpMV kernel (q = A p with p.q) against the measured HBM
copy bandwidth.

Other workloads (--workload):
  spmv2d      2D Laplacian 64x64 (n = 4,096, nnz = 20,224) FP64, one step = 1000
              lilac_spmv calls on the resident matrix; metric SpMV GB/s
  pagerank22  R-MAT scale 22 (4,194,304 vertices, ~65M edges) FP32 PageRank,
              20 iterations per step; metric SpMV GB/s of the fused iterations
  ir192       3D Poisson 192^3 (n = 7,077,888), FP32 inner CG + FP64 refinement
              to 1e-10; metric solves/s, with plain FP64 CG timed beside it

--impl reference times the CPU oracle (sequential FP64 C, the paper's
baseline kind: sequential code at -O2) on the same workload on the host
cores, one bounded sample per step, rank 0 only.

Multi-GPU: replicas only (each rank runs its own copy; no collective on the
data path); value = work of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SpMV GB/s (% of HBM peak); CG solves/s + p50/p99, served vs plain"
L2_BYTES = 129 * 2 ** 20


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# FP64 rate of the GB300: 152 SMs x 2 FP64 FMA per clock (ncu's own peak:
# 304 DFMA per cycle per GPU) x 2 FLOP x 2.07 GHz = 1.2586 TFLOP/s.  A loop of
# independent DFMAs measured 1.20 TFLOP/s on this machine.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

# --variant: the kernel to use instead of the tuner's choice (the matrix is
# then created without the timed tuning, so that a run under a profiler uses
# the same kernel as the plain run)
FORCED_VARIANT = None
VARIANT_CODES = {"scalar": 1, "vector": 2, "staged": 3, "merge": 4, "slab": 5, "jds": 6, "sell": 7,
                 "hub": 8}


def _kernel_src_hash():
    h = hashlib.sha256()
    for f in ("spmv_kernels.cuh", "ops.cuh", "lilac_device.cuh", "launch.cuh", "lilac_sell.cu",
              "lilac_hub.cu"):
        with open(os.path.join(ROOT, "paper_2001_07938_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel_key: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the kernel source as it is now (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel_key)
    if not e or e.get("src_hash") != _kernel_src_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def _spmv_bytes(n, ncols, nnz, vb):
    """Roofline bytes of one SpMV: nnz*(vb+4) + (n+1)*4 + ncols*vb + n*vb."""
    return nnz * (vb + 4) + (n + 1) * 4 + ncols * vb + n * vb


def _kernel_name(M):
    info = M.info()
    w = info["vector_width"]
    return {1: "spmv_rows_kernel (scalar)", 2: f"spmv_rows_kernel (vector, {w} lanes/row)",
            3: f"spmv_staged_kernel ({w} lanes/row)", 4: "spmv_merge_kernel",
            5: "spmv_slab_kernel (sliced ELL over x slabs in shared memory, slabs combined per row group)",
            6: "spmv_jds_kernel", 7: "spmv_sell_kernel (sliced ELL, one lane per row)",
            8: "hub_pieces_kernel + spmv_sell_kernel (hub columns' x in shared memory, "
               "cold columns as sliced ELL adding the slab sums)"
            }.get(info["variant"], "spmv")


# --- workloads ------------------------------------------------------------------

class Workload:
    """A benchmark workload: setup / step / check / roofline_sample /
    e2e_setup / e2e_step / cpu_sample / config; `work_per_step` units of
    `unit` x seconds per step."""
    flush_l2 = False
    work_per_step = 1.0
    traffic_key = None  # the profiles/traffic.json entry of the dominant kernel

    def __init__(self, L, torch):
        self.L, self.torch = L, torch

    def extra(self):
        """Further measurements of the workload for its JSON object."""
        return {}

    def _matrix(self, A):
        L = self.L
        if FORCED_VARIANT is None:
            return L.CsrMatrix.from_csr(A)
        M = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
        M.set_variant(*FORCED_VARIANT)
        return M

    def roofline_alu(self):
        """(FLOP per SpMV launch, what) when the SpMV is bound by FP64
        arithmetic rather than HBM, else None."""
        return None

    def _profiled(self, k, nbytes, what):
        """Average SpMV launch duration over k steps (lilac_csr_profile:
        CUDA event pairs on the launching stream, inside the captured graphs)."""
        L = self.L
        L.lilac_csr_profile(self.M.handle, True)
        for _ in range(k):
            self.step()
        ms, n = L.lilac_csr_profile(self.M.handle, False)
        return ms / n, n, nbytes, _kernel_name(self.M) + what


class CG75k(Workload):
    name = "cg_spd_n75000_75it"
    traffic_key = "cg75k"
    unit = "solves/s"
    dtype = "f64"
    iters = 75

    def __init__(self, L, torch):
        super().__init__(L, torch)
        from paper_2001_07938_gb300 import inputs
        self.A, self.b = inputs.workload_spd_cg()

    def roofline_alu(self):
        # one FP64 FMA per nonzero: ncu shows the FP64 pipe, not DRAM, nearest
        # its limit for this matrix (random columns, FP64 values)
        return 2.0 * self.A.nnz, "FP64 FMA per nonzero"

    def config(self):
        A = self.A
        mat = A.nnz * 12 + (A.n + 1) * 4
        return {"workload": self.name, "matrix": "random SPD, ~181 nnz/row, uniform columns",
                "n": A.n, "nnz": A.nnz, "iterations": self.iters, "precision": "fp64",
                "index": "int32", "rhs": "ones",
                "l2": f"inputs larger than L2: matrix {mat / 1e6:.0f} MB > "
                      f"{L2_BYTES / 1e6:.0f} MB L2, no flush"}

    def setup(self):
        torch, L = self.torch, self.L
        self.M = self._matrix(self.A)
        self.bd = torch.from_numpy(self.b).cuda()
        self.xd = torch.zeros(self.A.n, dtype=torch.float64, device="cuda")
        self.opts = L.lilac_cg_opts_default()
        self.opts.max_iter, self.opts.rtol, self.opts.true_residual = self.iters, 0.0, 0
        # kernels per solve, as the library counts them for the chosen variant
        _, info = L.lilac_cg(self.M.handle, self.bd.data_ptr(), self.xd.data_ptr(),
                             L.LILAC_MEM_DEVICE, self.opts, want_info=True)
        self.launches_per_step = info.kernel_launches

    def step(self):
        L = self.L
        L.lilac_cg(self.M.handle, self.bd.data_ptr(), self.xd.data_ptr(), L.LILAC_MEM_DEVICE,
                   self.opts, want_info=False)

    def check(self):
        st, info = self.M.cg(self.bd, self.xd, max_iter=self.iters, rtol=0.0, true_residual=True)
        return {"iters": info.iters, "true_rel_res": info.true_rel_res}

    def roofline_sample(self, k):
        A = self.A
        ms, n, nbytes, name = self._profiled(k, _spmv_bytes(A.n, A.ncols, A.nnz, 8),
                                             " with the CG epilogue (q = A p, p.q fused)")
        if self.M.info()["variant"] == VARIANT_CODES["slab"]:
            # FP64 CG on a SLAB handle runs the SLAB CG form
            name = ("spmv_slab_cg_kernel (sliced ELL over x slabs in shared memory; q left as slab "
                    "partials and p.q as per-CTA sums for the fused CG step)")
        return ms, n, nbytes, name

    def e2e_setup(self):
        torch = self.torch
        self.bh = torch.from_numpy(self.b).pin_memory()
        self.xh = torch.zeros(self.A.n, dtype=torch.float64).pin_memory()
        self.e2e_bytes = (self.A.n * 8, self.A.n * 8)

    def e2e_step(self):
        L = self.L
        L.lilac_cg(self.M.handle, self.bh.data_ptr(), self.xh.data_ptr(), L.LILAC_MEM_HOST,
                   self.opts, want_info=False)

    def cpu_sample(self, budget_s, parallel=False):
        """Oracle CG on the same system; a full 75-iteration solve if it fits
        the budget, else the first k iterations scaled to a solve."""
        import oracle
        A, b = self.A, self.b
        t0 = time.perf_counter()
        oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=2, rtol=0.0, parallel=parallel)
        t_it = (time.perf_counter() - t0) / 2
        k = int(max(1, min(self.iters, budget_s / max(t_it, 1e-9))))
        t0 = time.perf_counter()
        oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=k, rtol=0.0, parallel=parallel)
        t = time.perf_counter() - t0
        solve_s = t * self.iters / k
        sample = (f"one full {self.iters}-iteration oracle CG solve" if k == self.iters else
                  f"first {k} of {self.iters} oracle CG iterations, scaled to a solve")
        return 1.0 / solve_s, sample

    def close(self):
        self.M.close()


class SpMV2D(Workload):
    name = "spmv_laplacian2d_m64_1000calls"
    traffic_key = "spmv2d"
    unit = "GB/s"
    dtype = "f64"
    flush_l2 = True
    calls = 1000

    def __init__(self, L, torch):
        super().__init__(L, torch)
        from paper_2001_07938_gb300 import inputs
        self.A, self.x = inputs.workload_laplacian2d_spmv(64)
        self.work_per_step = self.calls * self.spmv_bytes() / 1e9

    def spmv_bytes(self):
        A = self.A
        return _spmv_bytes(A.n, A.ncols, A.nnz, 8)

    def config(self):
        A = self.A
        return {"workload": self.name, "matrix": "2D 5-point Laplacian, 64x64 grid",
                "n": A.n, "nnz": A.nnz, "calls_per_step": self.calls, "precision": "fp64",
                "index": "int32", "x": "uniform [-1,1], seed 0",
                "l2": "L2 flushed (256 MB write) between steps; within a step the 325 KB "
                      "matrix stays L2-resident, which is the workload (1000 repeated calls)"}

    def setup(self):
        torch, L = self.torch, self.L
        self.M = self._matrix(self.A)
        self.xd = torch.from_numpy(self.x).cuda()
        self.yd = torch.empty(self.A.n, dtype=torch.float64, device="cuda")
        self.launches_per_step = self.calls
        self.px, self.py = self.xd.data_ptr(), self.yd.data_ptr()
        self.stream = torch.cuda.current_stream().cuda_stream

    def step(self):
        L, h = self.L, self.M.handle
        st = self.stream
        for _ in range(self.calls):
            L.lilac_spmv(h, self.px, self.py, L.LILAC_MEM_DEVICE, st)

    def check(self):
        return {"calls_per_step": self.calls, "us_per_call_note": "ms_per_step / 1000 calls"}

    def roofline_sample(self, k):
        torch = self.torch
        stream = torch.cuda.current_stream()
        n = 50 * k
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * n)]
        L, h = self.L, self.M.handle
        for i in range(n):
            evs[2 * i].record(stream)
            L.lilac_spmv(h, self.px, self.py, L.LILAC_MEM_DEVICE)
            evs[2 * i + 1].record(stream)
        torch.cuda.synchronize()
        ms = sum(evs[2 * i].elapsed_time(evs[2 * i + 1]) for i in range(n))
        return ms / n, n, self.spmv_bytes(), _kernel_name(self.M)

    def extra(self):
        """The same 1000 calls captured once into one CUDA graph and replayed:
        the launch cost of the API calls removed (L2 flushed before each
        replay, as between the API steps)."""
        torch, L, h = self.torch, self.L, self.M.handle
        flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                L.lilac_spmv(h, self.px, self.py, L.LILAC_MEM_DEVICE, side.cuda_stream)
        torch.cuda.current_stream().wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            cs = torch.cuda.current_stream().cuda_stream
            for _ in range(self.calls):
                L.lilac_spmv(h, self.px, self.py, L.LILAC_MEM_DEVICE, cs)
        stream = torch.cuda.current_stream()
        for _ in range(3):
            g.replay()
        reps = 10
        ms = []
        for k in range(reps):
            flush.fill_(k & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.replay()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        del g
        t = sum(ms) / reps
        return {"graph_1000_calls": {"us_per_call": 1000.0 * t / self.calls,
                                     "gbs": self.calls * self.spmv_bytes() / (t / 1000.0) / 1e9,
                                     "replays": reps,
                                     "note": "1000 lilac_spmv calls captured in one CUDA graph"},
                "api_1000_calls": {"us_per_call": None}}

    def e2e_setup(self):
        torch = self.torch
        self.xh = torch.from_numpy(self.x).pin_memory()
        self.yh = torch.empty(self.A.n, dtype=torch.float64).pin_memory()
        self.e2e_bytes = (self.calls * self.A.ncols * 8, self.calls * self.A.n * 8)

    def e2e_step(self):
        L, h = self.L, self.M.handle
        px, py = self.xh.data_ptr(), self.yh.data_ptr()
        for _ in range(self.calls):
            L.lilac_spmv(h, px, py, L.LILAC_MEM_HOST)

    def cpu_sample(self, budget_s, parallel=False):
        import oracle
        A, x = self.A, self.x
        t0 = time.perf_counter()
        n = 0
        while time.perf_counter() - t0 < min(budget_s, 2.0) or n == 0:
            oracle.spmv(A.row_ptr, A.col_ind, A.vals, x, parallel=parallel)
            n += 1
        t = (time.perf_counter() - t0) / n
        return self.spmv_bytes() / t / 1e9, f"{n} oracle SpMV calls on the same matrix"

    def close(self):
        self.M.close()


class PageRank22(Workload):
    name = "pagerank_rmat22_20it"
    traffic_key = "pagerank22"
    unit = "GB/s"
    dtype = "f32"
    iters = 20
    scale = 22  # --rmat-scale: smaller graphs of the same recipe for profiling
    permute = True  # --rmat-unpermuted: the graph without the random vertex relabelling

    def __init__(self, L, torch, permute=None):
        super().__init__(L, torch)
        from paper_2001_07938_gb300 import inputs
        if permute is not None:
            self.permute = permute
        self.name = f"pagerank_rmat{self.scale}{'' if self.permute else '_unpermuted'}_20it"
        if not self.permute:
            self.traffic_key = "pagerank22_unpermuted"
        self.A = inputs.workload_rmat_pagerank(scale=self.scale, permute=self.permute)
        self.work_per_step = self.iters * self.iter_bytes() / 1e9

    def iter_bytes(self):
        """Per iteration: SpMV roofline bytes (FP32) + the dangling bitmap."""
        A = self.A
        return _spmv_bytes(A.n, A.ncols, A.nnz, 4) + A.n // 8

    def config(self):
        A = self.A
        return {"workload": self.name,
                "matrix": ("R-MAT a=.57 b=c=.19, " +
                           ("relabelled (seeded random permutation)" if self.permute else
                            "unpermuted (R-MAT vertex ids)") +
                           ", no self-loops/duplicates, transposed"),
                "n": A.n, "nnz": A.nnz, "iterations": self.iters, "damping": 0.85,
                "precision": "fp32 (D, L1 in fp64)", "index": "int32",
                "l2": f"inputs larger than L2: matrix {A.nnz * 8 / 1e6:.0f} MB, no flush"}

    def setup(self):
        torch, L = self.torch, self.L
        self.M = self._matrix(self.A)
        self.xd = torch.empty(self.A.n, dtype=torch.float32, device="cuda")
        self.launches_per_step = 1 + self.iters * self.M.info()["spmv_kernels"]

    def step(self):
        L = self.L
        L.lilac_pagerank(self.M.handle, self.xd.data_ptr(), 1, self.iters, 0.85, None,
                         L.LILAC_MEM_DEVICE)

    def check(self):
        l1 = self.M.pagerank(self.xd, iters=self.iters)
        return {"l1_last": float(l1[-1]), "sum_x": float(self.xd.double().sum().item())}

    def roofline_sample(self, k):
        return self._profiled(k, self.iter_bytes(),
                              " with the PageRank epilogue (teleport, L1, dangling sum)")

    def e2e_setup(self):
        self.xh = self.torch.empty(self.A.n, dtype=self.torch.float32).pin_memory()
        self.e2e_bytes = (0, self.A.n * 4)  # starts from 1/N on the device; result copied back

    def e2e_step(self):
        L = self.L
        L.lilac_pagerank(self.M.handle, self.xh.data_ptr(), 1, self.iters, 0.85, None,
                         L.LILAC_MEM_HOST)

    def cpu_sample(self, budget_s, parallel=False):
        import oracle
        A = self.A
        t0 = time.perf_counter()
        oracle.pagerank(A.row_ptr, A.col_ind, A.vals, iters=1, parallel=parallel)
        t1 = time.perf_counter() - t0
        k = int(max(1, min(self.iters, budget_s / max(t1, 1e-9))))
        if k > 1:
            t0 = time.perf_counter()
            oracle.pagerank(A.row_ptr, A.col_ind, A.vals, iters=k, parallel=parallel)
            t1 = (time.perf_counter() - t0) / k
        return self.iter_bytes() / t1 / 1e9, f"{k} oracle PageRank iterations"

    def close(self):
        self.M.close()


class IR192(Workload):
    name = "cg_mixed_poisson3d_m192_to_1e-10"
    traffic_key = "ir192"
    unit = "solves/s"
    dtype = "f32 inner / f64 refinement"
    precision = 2  # --ir-precision: 2 reliable updates, 1 restarted refinement

    def __init__(self, L, torch):
        super().__init__(L, torch)
        from paper_2001_07938_gb300 import inputs
        self.A, self.b = inputs.workload_poisson3d_ir()
        self.fp64_iters = None

    def config(self):
        A = self.A
        return {"workload": self.name, "matrix": "3D 7-point Poisson, 192^3 grid, FP32 values",
                "n": A.n, "nnz": A.nnz, "rtol": 1e-10, "b": "uniform [-1,1], seed 1",
                "index": "int32",
                "mixed_precision": ("FP32 CG with FP64 reliable updates (residual replacement)"
                                    if self.precision == 2 else
                                    "FP32 inner CG restarted by FP64 iterative refinement"),
                "l2": f"inputs larger than L2 ({A.nnz * 8 / 1e6:.0f} MB matrix), no flush"}

    def setup(self):
        torch, L = self.torch, self.L
        self.M = self._matrix(self.A)
        self.bd = torch.from_numpy(self.b).cuda()
        self.xd = torch.zeros(self.A.n, dtype=torch.float64, device="cuda")
        self.opts = self._opts(self.precision)
        st, info = L.lilac_cg(self.M.handle, self.bd.data_ptr(), self.xd.data_ptr(),
                              L.LILAC_MEM_DEVICE, self.opts, want_info=True)
        self.launches_per_step = info.kernel_launches

    def _opts(self, precision):
        o = self.L.lilac_cg_opts_default()
        o.precision, o.rtol = precision, 1e-10
        if precision == 1:
            o.max_iter, o.inner_max_iter, o.inner_rtol = 30, 4000, 1e-5
        else:
            o.max_iter, o.ru_delta = 20000, 0.1
        return o

    def step(self):
        L = self.L
        L.lilac_cg(self.M.handle, self.bd.data_ptr(), self.xd.data_ptr(), L.LILAC_MEM_DEVICE,
                   self.opts, want_info=False)

    def check(self):
        L, torch = self.L, self.torch
        st, info = L.lilac_cg(self.M.handle, self.bd.data_ptr(), self.xd.data_ptr(),
                              L.LILAC_MEM_DEVICE, self.opts, want_info=True)
        res = {"status": L.lilac_status_string(st), "inner_iters": info.iters,
               "refinements": info.refinements, "true_rel_res": info.true_rel_res}
        # the other mixed-precision form on the same handle, timed once
        other = 1 if self.precision == 2 else 2
        oo = self._opts(other)
        L.lilac_cg(self.M.handle, self.bd.data_ptr(), self.xd.data_ptr(), L.LILAC_MEM_DEVICE, oo,
                   want_info=False)  # warm-up (graph capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st2, i2 = L.lilac_cg(self.M.handle, self.bd.data_ptr(), self.xd.data_ptr(),
                             L.LILAC_MEM_DEVICE, oo, want_info=True)
        torch.cuda.synchronize()
        res[f"precision_{other}"] = {"solves_per_s": 1.0 / (time.perf_counter() - t0),
                                     "status": L.lilac_status_string(st2), "iters": i2.iters,
                                     "refinements": i2.refinements,
                                     "true_rel_res": i2.true_rel_res}
        # plain FP64 CG on the same system: the comparator
        M64 = L.CsrMatrix.from_csr(self.A.astype(np.float64))
        x64 = torch.zeros(self.A.n, dtype=torch.float64, device="cuda")
        M64.cg(self.bd, x64, max_iter=4000, rtol=1e-10)  # warm-up (graph capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st64, i64 = M64.cg(self.bd, x64, max_iter=4000, rtol=1e-10)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        M64.close()
        self.fp64_iters = i64.iters
        res["plain_fp64"] = {"solves_per_s": 1.0 / t64, "iters": i64.iters,
                             "true_rel_res": i64.true_rel_res}
        return res

    def roofline_sample(self, k):
        A = self.A
        return self._profiled(k, _spmv_bytes(A.n, A.ncols, A.nnz, 4),
                              " with the FP32 CG epilogue (q = A p, p.q fused)")

    def e2e_setup(self):
        torch = self.torch
        self.bh = torch.from_numpy(self.b).pin_memory()
        self.xh = torch.zeros(self.A.n, dtype=torch.float64).pin_memory()
        self.e2e_bytes = (self.A.n * 8, self.A.n * 8)

    def e2e_step(self):
        L = self.L
        L.lilac_cg(self.M.handle, self.bh.data_ptr(), self.xh.data_ptr(), L.LILAC_MEM_HOST,
                   self.opts, want_info=False)

    def cpu_sample(self, budget_s, parallel=False):
        """Oracle FP64 CG: k iterations timed, scaled to the FP64 CG iteration
        count to 1e-10 (a full oracle solve takes far longer than a step)."""
        import oracle
        A, b = self.A, self.b
        t0 = time.perf_counter()
        oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=2, rtol=0.0, parallel=parallel)
        t_it = (time.perf_counter() - t0) / 2
        k = int(max(1, min(200, budget_s / max(t_it, 1e-9))))
        t0 = time.perf_counter()
        oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=k, rtol=0.0, parallel=parallel)
        t_it = (time.perf_counter() - t0) / k
        n_it = self.fp64_iters or 1400
        return 1.0 / (t_it * n_it), (f"{k} oracle FP64 CG iterations, scaled to {n_it} "
                                     "iterations (the FP64 CG iteration count to 1e-10)")

    def close(self):
        self.M.close()


class SpMM8(Workload):
    """Y = A X for 8 vectors at once (row-major X), the random SPD n=75,000
    FP64 matrix: each nonzero is streamed once for all 8 vectors."""
    name = "spmm_spd_n75000_k8"
    traffic_key = "spmm8"
    unit = "GB/s"
    dtype = "f64"
    k = 8

    def __init__(self, L, torch):
        super().__init__(L, torch)
        from paper_2001_07938_gb300 import inputs
        self.A, _ = inputs.workload_spd_cg()
        A = self.A
        self.nbytes = A.nnz * 12 + (A.n + 1) * 4 + self.k * (A.ncols + A.n) * 8
        self.work_per_step = self.nbytes / 1e9

    def config(self):
        A = self.A
        return {"workload": self.name, "matrix": "random SPD, ~181 nnz/row, uniform columns",
                "n": A.n, "nnz": A.nnz, "vectors": self.k, "layout": "row-major X, Y",
                "index": "int32",
                "l2": f"inputs larger than L2: matrix {A.nnz * 12 / 1e6:.0f} MB, no flush"}

    def setup(self):
        torch, L = self.torch, self.L
        self.M = self._matrix(self.A)
        self.X = torch.rand(self.A.ncols, self.k, dtype=torch.float64, device="cuda")
        self.Y = torch.empty(self.A.n, self.k, dtype=torch.float64, device="cuda")
        self.launches_per_step = 1

    def step(self):
        self.M.spmm(self.X, self.Y, self.k)

    def check(self):
        torch = self.torch
        y1 = torch.empty(self.A.n, dtype=torch.float64, device="cuda")
        x1 = self.X[:, 3].contiguous()
        self.M.spmv(x1, y1)
        self.step()
        torch.cuda.synchronize()
        d = float((self.Y[:, 3] - y1).abs().max() / y1.abs().max())
        # the same 8 products through 8 single-vector SpMVs, for the ratio
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        xs = [self.X[:, j].contiguous() for j in range(self.k)]
        e0.record()
        for _ in range(5):
            for j in range(self.k):
                self.M.spmv(xs[j], y1)
        e1.record()
        torch.cuda.synchronize()
        return {"max_rel_diff_vs_spmv_column": d,
                "k_single_spmv_ms": e0.elapsed_time(e1) / 5}

    def roofline_alu(self):
        # one FP64 FMA per nonzero and vector: the FP64 pipe, not DRAM, bounds it
        return 2.0 * self.A.nnz * self.k, f"FP64 FMA per nonzero and vector ({self.k} vectors)"

    def roofline_sample(self, k):
        torch = self.torch
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            self.step()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k, k, self.nbytes, "spmm_rows_kernel<8> (warp per row)"

    def e2e_setup(self):
        torch = self.torch
        self.Xh = self.X.cpu().pin_memory()
        self.Yh = torch.empty(self.A.n, self.k, dtype=torch.float64).pin_memory()
        self.e2e_bytes = (self.A.ncols * self.k * 8, self.A.n * self.k * 8)

    def e2e_step(self):
        self.M.spmm(self.Xh, self.Yh, self.k)

    def cpu_sample(self, budget_s, parallel=False):
        import oracle
        A = self.A
        x = np.random.default_rng(0).random(A.ncols)
        t0 = time.perf_counter()
        oracle.spmv(A.row_ptr, A.col_ind, A.vals, x)
        t1 = time.perf_counter() - t0
        # k oracle SpMVs per SpMM
        return self.nbytes / (self.k * t1) / 1e9, f"one oracle SpMV timed, x{self.k} for the {self.k} vectors"

    def close(self):
        self.M.close()


class BFS22(Workload):
    """BFS levels on the R-MAT scale-22 graph (transposed adjacency handle), from
    the vertex of largest out-degree; GTEPS = edges of the reached component /
    time (the GAP convention)."""
    name = "bfs_rmat22"
    traffic_key = "bfs22"
    unit = "GTEPS"
    dtype = "int32"

    def __init__(self, L, torch):
        super().__init__(L, torch)
        from paper_2001_07938_gb300 import inputs
        self.A = inputs.workload_rmat_pagerank()
        outdeg = np.bincount(self.A.col_ind, minlength=self.A.n)
        self.src = int(np.argmax(outdeg))
        self.edges = None
        self.depth = None

    def config(self):
        A = self.A
        return {"workload": self.name, "matrix": "R-MAT scale 22 (as pagerank22), transposed",
                "n": A.n, "nnz": A.nnz, "source": self.src, "index": "int32",
                "l2": f"inputs larger than L2: {A.nnz * 8 / 1e6:.0f} MB of indices, no flush"}

    def setup(self):
        torch, L = self.torch, self.L
        self.M = self._matrix(self.A)
        self.lv = torch.empty(self.A.n, dtype=torch.int32, device="cuda")
        self.depth = self.M.bfs(self.src, self.lv)
        torch.cuda.synchronize()
        reached = self.lv.cpu().numpy() >= 0
        self.edges = int(np.diff(self.A.row_ptr)[reached].sum())
        self.work_per_step = self.edges / 1e9
        self.launches_per_step = 1 + 8 * ((self.depth + 8) // 8)

    def step(self):
        self.M.bfs(self.src, self.lv)

    def check(self):
        lv = self.lv.cpu().numpy()
        return {"depth": self.depth, "reached": int((lv >= 0).sum()), "edges": self.edges}

    def roofline_sample(self, k):
        """Whole BFS timed with events; bytes = the lower bound of its launches:
        each of depth + 1 level launches streams the row index of every nonzero
        and reads a level per row, and every column index is read at least once."""
        torch = self.torch
        A = self.A
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            self.step()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        nbytes = (self.depth + 1) * (A.nnz * 4 + A.n * 4) + A.nnz * 4
        return ms, k, nbytes, "bfs_pull_kernel x (depth + 1), whole BFS (lower-bound bytes)"

    def e2e_setup(self):
        self.lh = self.torch.empty(self.A.n, dtype=self.torch.int32).pin_memory()
        self.e2e_bytes = (0, self.A.n * 4)

    def e2e_step(self):
        self.L.lilac_bfs(self.M.handle, self.src, self.lh.data_ptr(), self.L.LILAC_MEM_HOST)

    def close(self):
        self.M.close()

    def cpu_sample(self, budget_s, parallel=False):
        import oracle
        A = self.A
        rows = np.repeat(np.arange(A.n, dtype=np.int32), np.diff(A.row_ptr))
        order = np.argsort(A.col_ind, kind="stable")
        rp = np.zeros(A.n + 1, np.int64)
        np.cumsum(np.bincount(A.col_ind, minlength=A.n), out=rp[1:])
        t0 = time.perf_counter()
        lev = oracle.bfs_levels(rp.astype(np.int32), rows[order], self.src)
        t = time.perf_counter() - t0
        if self.edges is None:  # reference arm: no GPU run to take it from
            self.edges = int(np.diff(A.row_ptr)[lev >= 0].sum())
            self.work_per_step = self.edges / 1e9
        return self.edges / t / 1e9, "one full oracle BFS (queue, out-edge lists) from the same source"


WORKLOADS = {"cg75k": CG75k, "spmv2d": SpMV2D, "pagerank22": PageRank22, "ir192": IR192,
             "bfs22": BFS22, "spmm8": SpMM8}


# --- served request stream ------------------------------------------------------

def served_stream(n_req=2000, n_mats=32, n_lo=1e3, n_hi=2e5, kmax=8, seed=0):
    """Seeded request stream: a pool of 2D/3D Laplacians and banded SPD matrices
    (half-bandwidth 8..64) with n log-uniform in [n_lo, n_hi]; requests pick a
    matrix with Zipf(1.1) popularity; half are SpMV batches of k uniform in
    [1, kmax] vectors, half CG solves to 1e-10, of which half ask for FP32
    values with FP64 refinement (precision 2).  Requests are (kind, matrix, k,
    precision); their vectors come from per-matrix blocks (served_inputs)."""
    from paper_2001_07938_gb300 import inputs
    rng = np.random.default_rng(seed)
    pool = []
    for i in range(n_mats):
        n = float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        kind = i % 3
        if kind == 0:
            pool.append(inputs.laplacian2d(max(4, int(round(n ** 0.5)))))
        elif kind == 1:
            pool.append(inputs.laplacian3d(max(3, int(round(n ** (1 / 3))))))
        else:
            pool.append(inputs.banded_spd(int(n), int(rng.integers(8, 65)), 1.0, seed=100 + i))
    w = 1.0 / np.arange(1, n_mats + 1) ** 1.1
    w /= w.sum()
    reqs = []
    for t in range(n_req):
        mi = int(rng.choice(n_mats, p=w))
        if rng.random() < 0.5:
            reqs.append(("spmv", mi, int(rng.integers(1, kmax + 1)), 0))
        else:
            reqs.append(("cg", mi, 1, 2 if rng.random() < 0.5 else 0))
    return pool, reqs


def _pinned(n):
    """An FP64 host array in page-locked memory (a numpy view of a pinned
    tensor, which the view keeps alive)."""
    import torch
    return torch.empty(max(1, n), dtype=torch.float64, pin_memory=True).numpy()[:n]


def served_inputs(pool, reqs, kmax, alloc=np.empty):
    """Per used matrix: kmax SpMV input vectors (one block, a request of k
    vectors takes the first k) and one right-hand side, uniform in [-1, 1]:
    the requests' inputs without a copy per request."""
    from paper_2001_07938_gb300 import inputs
    spmv_m = {r[1] for r in reqs if r[0] == "spmv"}
    cg_m = {r[1] for r in reqs if r[0] == "cg"}
    X, B = {}, {}
    for mi in sorted(spmv_m):
        X[mi] = alloc(kmax * pool[mi].ncols)
        X[mi][:] = inputs.uniform(10_000 + mi, kmax * pool[mi].ncols)
    for mi in sorted(cg_m):
        B[mi] = alloc(pool[mi].n)
        B[mi][:] = inputs.uniform(20_000 + mi, pool[mi].n)
    return X, B


class _BufPool:
    """Reusable host output buffers by length, page-locked like the inputs."""

    def __init__(self, alloc=np.empty):
        self.free = {}
        self.alloc = alloc

    def get(self, n):
        lst = self.free.get(n)
        return lst.pop() if lst else self.alloc(n)

    def put(self, a):
        self.free.setdefault(a.size, []).append(a)


def run_served(args):
    """The served stream against the plain system (one request at a time,
    lilac_spmv per vector / FP64 lilac_cg, matrices resident), both with the
    same tuning policy.  The server is created once; a first pass at
    saturation uploads the pool (as the plain system's handles are created
    before it is timed), then one saturated pass and one Poisson pass per load
    point are timed.  Plain latencies under the same arrivals follow exactly
    from its measured service times (FIFO, one server).  Every result is
    compared with the plain system's at 16 sampled positions."""
    import torch
    from paper_2001_07938_gb300 import build as lbuild
    from paper_2001_07938_gb300 import lilac as L
    torch.cuda.set_device(0)
    lbuild.build()
    L.load()
    t_begin = time.perf_counter()

    def note(msg):
        print(f"[served] {msg} at {time.perf_counter() - t_begin:.1f} s", file=sys.stderr, flush=True)

    pool, reqs = served_stream(n_req=args.served_requests, n_mats=args.served_mats,
                               n_hi=args.served_nmax, kmax=args.served_kmax)
    X, B = served_inputs(pool, reqs, args.served_kmax, alloc=_pinned)
    note(f"stream of {len(reqs)} requests over {len(pool)} matrices built")
    N = len(reqs)
    n_cg = sum(1 for r in reqs if r[0] == "cg")
    n_mixed = sum(1 for r in reqs if r[0] == "cg" and r[3] == 2)
    pool_bytes = sum(A.nnz * 12 + (A.n + 1) * 4 for A in pool)
    req_bytes = sum(8 * r[2] * (pool[r[1]].ncols + pool[r[1]].n) for r in reqs)
    bufs = _BufPool(alloc=_pinned)

    def inp_of(r):
        kind, mi, k, _ = r
        return X[mi][:k * pool[mi].ncols] if kind == "spmv" else B[mi]

    def out_len(r):
        return r[2] * pool[r[1]].n

    rs = np.random.default_rng(7)
    samples = [rs.integers(0, out_len(r), 16) for r in reqs]
    ref = [None] * N  # (values at the samples, max |plain result|)

    flags = 0 if args.served_tune else L.LILAC_CREATE_NO_TUNE
    Ms = [L.CsrMatrix.from_csr(A, flags=flags) for A in pool]

    def plain_one(r, out):
        kind, mi, k, _ = r  # plain: every solve in FP64
        A, M, inp = pool[mi], Ms[mi], inp_of(r)
        if kind == "spmv":
            for j in range(k):
                M.spmv(inp[j * A.ncols:(j + 1) * A.ncols], out[j * A.n:(j + 1) * A.n])
        else:
            out[:] = 0.0
            M.cg(inp, out, max_iter=20000, rtol=1e-10, true_residual=False)

    for r in reqs[:20]:  # warm-up (graph capture per matrix)
        o = bufs.get(out_len(r))
        plain_one(r, o)
        bufs.put(o)
    service = []
    t_all = time.perf_counter()
    for t, r in enumerate(reqs):
        t0 = time.perf_counter()
        o = bufs.get(out_len(r))
        plain_one(r, o)
        service.append(time.perf_counter() - t0)
        ref[t] = (o[samples[t]].copy(), float(np.max(np.abs(o))))
        bufs.put(o)
    plain_makespan = time.perf_counter() - t_all
    for M in Ms:
        M.close()
    cap = N / plain_makespan
    note(f"plain done: {plain_makespan:.1f} s")

    def serve(S, ids, timed_arrivals, max_inflight=512, max_inflight_bytes=8 << 30):
        """One pass of the stream; saturated (timed_arrivals None) keeps up to
        max_inflight requests submitted and not yet completed."""
        outs = {}
        lat, wait, svc, rounds = [0.0] * N, [0.0] * N, [0.0] * N, [0] * N
        worst = 0.0
        got, i, inflight_bytes = 0, 0, 0
        t0 = L.Server.now()
        st0 = S.stats()
        last_progress = L.Server.now()
        while got < N:
            now = L.Server.now() - t0
            if L.Server.now() - last_progress > 300.0:
                raise RuntimeError(f"served stream stalled: {S.stats()}")
            while i < N and (timed_arrivals[i] <= now if timed_arrivals is not None else
                             (i - got < max_inflight and inflight_bytes < max_inflight_bytes)):
                kind, mi, k, prec = reqs[i]
                out = bufs.get(out_len(reqs[i]))
                outs[i] = out
                inflight_bytes += out.nbytes
                if kind == "spmv":
                    S.submit(L.LILAC_REQ_SPMV, ids[mi], inp_of(reqs[i]), out, i, nvec=k)
                else:
                    S.submit(L.LILAC_REQ_CG, ids[mi], inp_of(reqs[i]), out, i, max_iter=20000,
                             rtol=1e-10, precision=prec)
                i += 1
            pending = S.step()
            for c in S.poll():
                # latency from the scheduled arrival when arrivals are timed
                tag = c["tag"]
                if c["status"] != L.LILAC_OK:
                    raise RuntimeError(f"request {tag} failed: {c}")
                a = c["arrival"] if timed_arrivals is None else t0 + timed_arrivals[tag]
                lat[tag] = c["finish"] - a
                wait[tag] = c["admitted"] - a
                svc[tag] = c["finish"] - c["admitted"]
                rounds[tag] = c["rounds"]
                out = outs.pop(tag)
                vals, mx = ref[tag]
                worst = max(worst, float(np.max(np.abs(out[samples[tag]] - vals))) / max(mx, 1e-300))
                inflight_bytes -= out.nbytes
                bufs.put(out)
                got += 1
                last_progress = L.Server.now()
            if pending == 0 and i < N and timed_arrivals is not None:
                time.sleep(max(0.0, min(0.01, timed_arrivals[i] - (L.Server.now() - t0))))
        makespan = L.Server.now() - t0
        st1 = S.stats()
        delta = {k: st1[k] - st0[k] for k in ("rounds", "uploads", "evictions", "budget_waits")}
        return lat, wait, svc, rounds, makespan, delta, worst

    def pct(v, q):
        return 1000.0 * float(np.percentile(v, q))

    def breakdown(lat, wait, svc, rounds):
        """Mean queue wait / service / rounds of the requests at or above the
        99th latency percentile, by kind."""
        p99 = np.percentile(lat, 99)
        top = [t for t in range(N) if lat[t] >= p99]
        kinds = {}
        for name in ("spmv", "cg"):
            ts = [t for t in top if reqs[t][0] == name]
            if ts:
                kinds[name] = {"count": len(ts),
                               "queue_wait_ms": 1000 * float(np.mean([wait[t] for t in ts])),
                               "service_ms": 1000 * float(np.mean([svc[t] for t in ts])),
                               "rounds": float(np.mean([rounds[t] for t in ts])),
                               "n": float(np.mean([pool[reqs[t][1]].n for t in ts]))}
        return kinds

    def timed_pass(S, ids, load):
        lam = load * cap
        arrivals = np.cumsum(np.random.default_rng(1).exponential(1.0 / lam, N))
        lat, wait, svc, rounds, mk, delta, worst = serve(S, ids, arrivals)
        return {"load": load, "arrival_rate_per_s": lam,
                "served": {"latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99)},
                           "queue_wait_ms": {"p50": pct(wait, 50), "p99": pct(wait, 99)},
                           "p99_breakdown": breakdown(lat, wait, svc, rounds),
                           "makespan_s": mk, "max_rel_diff_vs_plain": worst, **delta}}, arrivals

    def plain_latency(arrivals):
        fin, lat_plain = 0.0, []
        for a, sv in zip(arrivals, service):  # FIFO single server, exact from service times
            fin = max(fin, a) + sv
            lat_plain.append(fin - a)
        return {"latency_ms": {"p50": pct(lat_plain, 50), "p99": pct(lat_plain, 99)}}

    S = L.Server(hbm_budget_bytes=int(args.served_budget_gb * 2 ** 30),
                 iters_per_round=args.served_round, tune=args.served_tune)
    ids = [S.add_matrix(A) for A in pool]
    serve(S, ids, None)  # warm-up: uploads, graph capture, pool blocks
    note("warm-up pass done")
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    _, _, _, _, served_makespan, sat_delta, diff = serve(S, ids, None)
    note("saturated pass done")
    value = N / served_makespan
    loads = []
    for load in [float(v) for v in args.served_loads.split(",")]:
        entry, arrivals = timed_pass(S, ids, load)
        entry["plain"] = plain_latency(arrivals)
        loads.append(entry)
        note(f"load {load} done")
    st = S.stats()
    S.close()
    bound = None
    if args.served_bind_gb > 0:
        # the same stream under a device-memory budget below the pool's
        # footprint: uploads, evictions and waits inside the timed passes
        S = L.Server(hbm_budget_bytes=int(args.served_bind_gb * 2 ** 30),
                     iters_per_round=args.served_round, tune=args.served_tune)
        ids = [S.add_matrix(A) for A in pool]
        entry, arrivals = timed_pass(S, ids, 0.8)  # from cold: uploads inside the pass
        entry["plain"] = plain_latency(arrivals)
        bound = {"hbm_budget_gb": args.served_bind_gb, "load_0.8": entry}
        S.close()
        note("budget-bound passes done")
    clk = clocks.stop()
    line = {"metric": METRIC, "value": value, "unit": "requests/s", "n_gpus": 1,
            "steps": 1, "warmup": 1, "ms_per_step": served_makespan * 1000,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "served_stream", "requests": N, "cg_requests": n_cg,
                       "cg_mixed_precision_requests": n_mixed,
                       "plain": "one request at a time, lilac_spmv per vector / FP64 lilac_cg",
                       "matrices": len(pool), "pool_matrix_bytes": pool_bytes,
                       "request_vector_bytes": req_bytes,
                       "n_range": [1e3, args.served_nmax], "zipf": 1.1,
                       "spmv_vectors": f"1..{args.served_kmax}", "rtol": 1e-10,
                       "hbm_budget_gb": args.served_budget_gb, "tuned": bool(args.served_tune),
                       "iters_per_round": args.served_round,
                       "inputs": "per matrix one seeded block of SpMV vectors and one b, shared by "
                                 "its requests; request vectors and results in page-locked host "
                                 "memory (both arms); results checked against plain at 16 samples "
                                 "each"},
            "served": {"requests_per_s": value, "cg_solves_per_s": n_cg / served_makespan,
                       "saturated": sat_delta, "resident_bytes_end": st["resident_bytes"]},
            "plain": {"requests_per_s": cap, "cg_solves_per_s": n_cg / plain_makespan},
            "served_vs_plain_throughput": value / cap,
            "max_rel_diff_served_vs_plain": diff,
            "loads": loads,
            "budget_bound": bound, "clocks": clk,
            "roofline": None, "cpu_baseline": None,
            "e2e": {"value": value, "unit": "requests/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0, "note": "requests carry host buffers end to end"}}
    print(json.dumps(line), flush=True)
    return 0


# --- the two arms ---------------------------------------------------------------

def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def collectives(ws, device):
    """(barrier, max_over_ranks) for N replicas: with ws > 1 through the
    initialised process group (NCCL on the GPU, gloo on the CPU in tests)."""
    import torch

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        if device == "cuda":
            torch.cuda.synchronize()

    def max_over_ranks(v):
        if ws > 1:
            import torch.distributed as dist
            t = torch.tensor([float(v)], dtype=torch.float64, device=device)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return float(t.item())
        return v

    return barrier, max_over_ranks


def replica_value(ws, steps, work_per_step, total_ms):
    """Whole-job throughput of ws replicas: the units all ranks processed over
    the slowest rank's time."""
    return ws * steps * work_per_step / (total_ms / 1000.0)


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    wl = WORKLOADS["cg75k" if args.workload == "all" else args.workload](None, None)
    steps, warm = args.steps, args.warmup
    budget = max(0.05, args.ref_seconds / max(1, steps + warm))
    vals, sample = [], ""
    for i in range(warm + steps):
        v, sample = wl.cpu_sample(budget)
        if i >= warm:
            vals.append(v)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": wl.unit,
            "n_gpus": args.gpus, "steps": steps, "warmup": warm,
            "ms_per_step": 1000.0 * wl.work_per_step / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "n": wl.A.n, "nnz": wl.A.nnz},
            "cpu_baseline": {"value": value, "unit": wl.unit, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": wl.unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


VARIANT_NAMES = {v: k for k, v in VARIANT_CODES.items()}


def _tuner(wl):
    """The kernel the handle runs and the autotuner's trial (ms per call)."""
    M = getattr(wl, "M", None)
    if M is None:
        return None
    info = M.info()
    table = M.tune_table()
    return {"variant": VARIANT_NAMES.get(info["variant"], str(info["variant"])),
            "width": info["vector_width"],
            "forced": FORCED_VARIANT is not None,
            "trial_ms_per_call": {f"{VARIANT_NAMES.get(t['variant'], t['variant'])}:{t['width']}":
                                  round(t["ms"], 5) for t in table}}


def _cpu_baseline(wl, budget_s):
    """The oracle on one host core (the paper's sequential -O2 baseline kind),
    and the same oracle with its SpMV rows shared among all host cores."""
    import oracle
    v, sample = wl.cpu_sample(budget_s)
    out = {"value": v, "unit": wl.unit, "cores": 1, "kind": "oracle", "sample": sample}
    try:
        cores = oracle.threads(True)
        vp, sp = wl.cpu_sample(budget_s / 2, parallel=True)
        out["all_cores"] = {"value": vp, "unit": wl.unit, "cores": cores, "kind": "oracle",
                            "sample": sp + " (OpenMP build: SpMV rows on all cores, static "
                                           "schedule, results bitwise the sequential ones)"}
    except RuntimeError as e:
        out["all_cores"] = {"unavailable": str(e)}
    return out


def measure(wl, args, ctx, cpu_budget_s=20.0):
    """Warm up, time K steps with CUDA events (clocks sampled meanwhile), the
    dominant kernel's launches, the end-to-end form through the C ABI with
    host buffers, and the CPU oracle; returns the workload's JSON object
    (rank 0) or None."""
    torch, ws, rank = ctx["torch"], ctx["ws"], ctx["rank"]
    barrier, max_over_ranks = ctx["barrier"], ctx["max_over_ranks"]
    wl.setup()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda") if wl.flush_l2 else None
    for _ in range(args.warmup):
        wl.step()
    barrier()
    check = wl.check()
    barrier()

    K = args.steps
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    barrier()
    for k in range(K):
        if flush is not None:
            flush.fill_(k & 0xFF)  # L2 flush between timed steps, outside the step's events
        ev0[k].record(stream)
        wl.step()
        ev1[k].record(stream)
    barrier()
    clk = clocks.stop() if clocks else None
    step_ms = [ev0[k].elapsed_time(ev1[k]) for k in range(K)]
    total_ms = max_over_ranks(sum(step_ms))
    value = replica_value(ws, K, wl.work_per_step, total_ms)

    # dominant kernel: CUDA events on its own stream
    kern_ms, n_kern, kern_bytes, kname = wl.roofline_sample(min(K, 5))
    peak, peak_kind = _peaks()
    achieved = kern_bytes / (kern_ms / 1000.0) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": _ncu_traffic(wl.traffic_key), "kernel": kname,
                "algorithmic_bytes_per_launch": kern_bytes, "avg_launch_ms": kern_ms,
                "launches_timed": n_kern,
                "peak_kind": f"of {peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}
    roofline_hbm = None
    alu = wl.roofline_alu()
    if alu is not None:
        flops, what = alu
        tflops = flops / (kern_ms / 1000.0) / 1e12
        roofline_hbm = roofline
        roofline = {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": tflops / FP64_PEAK_TFLOPS,
                    "traffic": roofline_hbm["traffic"], "kernel": kname,
                    "algorithmic_flops_per_launch": flops, "flops": what,
                    "algorithmic_bytes_per_launch": kern_bytes, "avg_launch_ms": kern_ms,
                    "launches_timed": n_kern,
                    "peak_kind": "of the FP64 rate (152 SMs x 2 FMA/clk x 2.07 GHz, ncu's 304 "
                                 "DFMA/cycle peak; a DFMA loop measured 1.20 TFLOP/s)"}
    extra = wl.extra()

    # end to end through the C ABI with pinned host buffers
    wl.e2e_setup()
    for _ in range(2):
        wl.e2e_step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        wl.e2e_step()
    e1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1))
    e2e = {"value": ws * K * wl.work_per_step / (e2e_ms / 1000.0), "unit": wl.unit,
           "h2d_bytes_per_step": wl.e2e_bytes[0], "d2h_bytes_per_step": wl.e2e_bytes[1]}
    tuner = _tuner(wl)
    wl.close()
    if rank != 0:
        return None
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = _cpu_baseline(wl, cpu_budget_s)
    line = {"metric": METRIC, "value": value, "unit": wl.unit, "n_gpus": ws, "steps": K,
            "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": wl.dtype, "data": "synthetic",
            "config": wl.config() | {"parallelism": f"replicas{ws}"},
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                           "p99": float(np.percentile(step_ms, 99))},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            **({"roofline_hbm": roofline_hbm} if roofline_hbm else {}),
            "gpu_launches": wl.launches_per_step * K,
            "clocks": clk, "check": check, "tuner": tuner,
            "spmv": {"gbs": achieved, "hbm_frac": achieved / peak}}
    if extra:
        if "api_1000_calls" in extra:
            extra["api_1000_calls"] = {"us_per_call": 1000.0 * (total_ms / K) / wl.calls,
                                       "note": "1000 lilac_spmv API calls per step"}
        line.update(extra)
    return line


# The default run: the FP64 CG workload is the headline; the other configs
# of the benchmark suite ride along as keyed objects of the same line.
ALSO = [("spmv2d", "spmv2d", {}), ("pagerank22", "pagerank22", {}),
        ("pagerank22_unpermuted", "pagerank22", {"permute": False}), ("ir192", "ir192", {})]
SUB_KEYS_DROP = ("metric", "n_gpus", "scaling", "vs_baseline", "data", "higher_is_better")


def run_lilac(args):
    import torch
    from paper_2001_07938_gb300 import build as lbuild
    from paper_2001_07938_gb300 import lilac as L

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        lbuild.build()
    if ws > 1:
        dist.barrier()
    L.load()

    barrier, max_over_ranks = collectives(ws, "cuda")
    ctx = {"torch": torch, "ws": ws, "rank": rank, "barrier": barrier,
           "max_over_ranks": max_over_ranks}

    global FORCED_VARIANT
    if args.variant:
        name, _, width = args.variant.partition(":")
        FORCED_VARIANT = (VARIANT_CODES[name], int(width or 0))
    head = "cg75k" if args.workload == "all" else args.workload
    line = measure(WORKLOADS[head](L, torch), args, ctx)
    if args.workload == "all" and not args.variant:
        for key, wname, kw in ALSO:
            sub = measure(WORKLOADS[wname](L, torch, **kw), args, ctx, cpu_budget_s=10.0)
            if rank == 0:
                line[key] = {k: v for k, v in sub.items() if k not in SUB_KEYS_DROP}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["lilac", "reference"], default="lilac")
    ap.add_argument("--workload", choices=["all"] + sorted(WORKLOADS) + ["served", "marshal"],
                    default="all",
                    help="all (default): the FP64 CG headline with the 2D Laplacian SpMV, "
                         "PageRank (relabelled and unpermuted R-MAT) and mixed-precision CG "
                         "workloads as keyed objects of the same line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=120.0,
                    help="reference arm: total seconds of oracle work over all steps")
    ap.add_argument("--rmat-scale", type=int, default=22,
                    help="R-MAT scale of the pagerank22 workload (22 is the benchmark size)")
    ap.add_argument("--ir-precision", type=int, choices=[1, 2], default=2,
                    help="mixed-precision CG of the ir192 workload")
    ap.add_argument("--served-requests", type=int, default=2000,
                    help="served stream: requests (the full recipe: 10000)")
    ap.add_argument("--served-mats", type=int, default=32, help="matrices in the pool (full: 256)")
    ap.add_argument("--served-nmax", type=float, default=2e5, help="largest n (full: 2e6)")
    ap.add_argument("--served-kmax", type=int, default=8, help="vectors per SpMV (full: 32)")
    ap.add_argument("--served-loads", default="0.8",
                    help="arrival rates as fractions of the plain capacity (full: 0.5,0.8,0.95)")
    ap.add_argument("--served-budget-gb", type=float, default=120.0)
    ap.add_argument("--served-bind-gb", type=float, default=0.0,
                    help="also run the stream under this (binding) budget at load 0.8")
    ap.add_argument("--served-tune", type=int, default=0, help="1: timed tuning at upload")
    ap.add_argument("--served-round", type=int, default=16)
    ap.add_argument("--variant", default="",
                    help="force the SpMV kernel instead of the tuner's choice, e.g. slab:4")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    PageRank22.scale = args.rmat_scale
    IR192.precision = args.ir_precision
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "marshal":
        return run_marshal(args)
    return run_lilac(args)


if __name__ == "__main__":
    sys.exit(main())
