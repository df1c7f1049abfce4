#!/usr/bin/env python
"""Benchmark of the GB300 SpMV / CG / PageRank library.

Default workload (one JSON line on stdout): unpreconditioned FP64 CG, 75
iterations, on a random SPD CSR matrix with n = 75,000 and ~181 nonzeros per
row at uniformly random columns (values U[0,1), symmetrised, diagonal = row
sum + 20), b = ones, int32 indices.  One step = one full solve through
lilac_cg (device buffers, resident matrix).  The metric is solves/s;
the roofline object reports the fused SpMV kernel (q = A p with p.q) against
the measured HBM copy bandwidth.

Other workloads: --workload spmv2d (2D Laplacian 64x64, 1000 SpMV calls per
step), pagerank22 (R-MAT scale 22, 20 FP32 PageRank iterations), ir192
(3D Poisson 192^3, mixed-precision CG to 1e-10).

--impl reference times the CPU oracle (sequential FP64 C, the paper's
baseline kind: sequential code at -O2) on the same workload on the host
cores, one bounded sample per step.

Multi-GPU: replicas only (each rank solves its own copy; no collective on
the data path); value = solves of all ranks / max-over-ranks time.
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


def _kernel_src_hash():
    h = hashlib.sha256()
    for f in ("spmv_kernels.cuh", "ops.cuh", "lilac_device.cuh", "launch.cuh"):
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


# --- workloads ------------------------------------------------------------------

class CG75k:
    name = "cg_spd_n75000_75it"
    unit = "solves/s"
    dtype = "f64"

    def __init__(self, L, torch):
        from paper_2001_07938_gb300 import inputs
        self.L, self.torch = L, torch
        self.A, self.b = inputs.workload_spd_cg()
        self.iters = 75

    def config(self):
        A = self.A
        return {"workload": self.name, "matrix": "random SPD, ~181 nnz/row, uniform columns",
                "n": A.n, "nnz": A.nnz, "iterations": self.iters, "precision": "fp64",
                "index": "int32", "rhs": "ones",
                "l2": f"inputs larger than L2: matrix {self._mat_bytes() / 1e6:.0f} MB > "
                      f"{L2_BYTES / 1e6:.0f} MB L2, no flush"}

    def _mat_bytes(self):
        return self.A.nnz * 12 + (self.A.n + 1) * 4

    def spmv_bytes(self):
        A = self.A
        return A.nnz * (8 + 4) + (A.n + 1) * 4 + A.ncols * 8 + A.n * 8

    def setup(self):
        torch, L = self.torch, self.L
        self.M = L.CsrMatrix.from_csr(self.A)
        self.bd = torch.from_numpy(self.b).cuda()
        self.xd = torch.zeros(self.A.n, dtype=torch.float64, device="cuda")
        self.opts = L.lilac_cg_opts_default()
        self.opts.max_iter, self.opts.rtol, self.opts.true_residual = self.iters, 0.0, 0
        self.launches_per_step = 2 + 3 * self.iters

    def step(self):
        L = self.L
        L.lilac_cg(self.M.handle, self.bd.data_ptr(), self.xd.data_ptr(), L.LILAC_MEM_DEVICE,
                   self.opts, want_info=False)

    def check(self):
        st, info = self.M.cg(self.bd, self.xd, max_iter=self.iters, rtol=0.0, true_residual=True)
        return {"iters": info.iters, "true_rel_res": info.true_rel_res}

    def roofline_sample(self, k):
        """Average duration of the fused SpMV (q = A p, p.q) from CUDA events
        recorded on its stream inside the captured solve graph."""
        ms, n = 0.0, 0
        for _ in range(k):
            st, info = self.M.cg(self.bd, self.xd, max_iter=self.iters, rtol=0.0,
                                 true_residual=False, profile=True)
            ms += info.spmv_ms
            n += info.spmv_launches
        return ms / n, n

    def e2e_setup(self):
        torch = self.torch
        self.bh = torch.from_numpy(self.b).pin_memory()
        self.xh = torch.zeros(self.A.n, dtype=torch.float64).pin_memory()
        self.e2e_bytes = (self.A.n * 8, self.A.n * 8)

    def e2e_step(self):
        L = self.L
        L.lilac_cg(self.M.handle, self.bh.data_ptr(), self.xh.data_ptr(), L.LILAC_MEM_HOST,
                   self.opts, want_info=False)

    def cpu_sample(self, budget_s):
        """Oracle CG on the same system; a full 75-iteration solve if it fits
        the budget, else the first k iterations scaled to a solve."""
        import oracle
        A, b = self.A, self.b
        t0 = time.perf_counter()
        oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=2, rtol=0.0)
        t_it = (time.perf_counter() - t0) / 2
        k = int(max(1, min(self.iters, budget_s / max(t_it, 1e-9))))
        t0 = time.perf_counter()
        oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=k, rtol=0.0)
        t = time.perf_counter() - t0
        solve_s = t * self.iters / k
        sample = (f"one full {self.iters}-iteration oracle CG solve" if k == self.iters else
                  f"first {k} of {self.iters} oracle CG iterations, scaled to a solve")
        return 1.0 / solve_s, sample

    def close(self):
        self.M.close()


WORKLOADS = {"cg75k": CG75k}


# --- the two arms ---------------------------------------------------------------

def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_2001_07938_gb300 import inputs  # noqa: F401
    oracle.build()

    class _NoTorch:
        pass

    wl = WORKLOADS[args.workload](None, None)
    steps, warm = args.steps, args.warmup
    budget = max(0.5, 120.0 / max(1, steps + warm))
    vals, samples = [], ""
    for i in range(warm + steps):
        v, samples = wl.cpu_sample(budget)
        if i >= warm:
            vals.append(v)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": wl.unit,
            "n_gpus": args.gpus, "steps": steps, "warmup": warm,
            "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": wl.dtype, "data": "synthetic",
            "config": {"workload": wl.name, "n": wl.A.n, "nnz": wl.A.nnz},
            "cpu_baseline": {"value": value, "unit": wl.unit, "cores": 1, "kind": "oracle",
                             "sample": samples},
            "e2e": {"value": value, "unit": wl.unit, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


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

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    wl = WORKLOADS[args.workload](L, torch)
    wl.setup()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        wl.step()
    barrier()
    check = wl.check()
    barrier()

    K = args.steps
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    barrier()
    evs[0].record(stream)
    for k in range(K):
        wl.step()
        evs[k + 1].record(stream)
    barrier()
    clk = clocks.stop() if clocks else None
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(K)]
    total_ms = evs[0].elapsed_time(evs[K])
    if ws > 1:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = ws * K / (total_ms / 1000.0)

    # dominant kernel: fused SpMV, CUDA events on its own stream
    kr = min(K, 5)
    spmv_ms, n_spmv = wl.roofline_sample(kr)
    minfo = wl.M.info()
    kname = {1: "spmv_rows_kernel (scalar)", 2: f"spmv_rows_kernel (vector, {minfo['vector_width']} lanes/row)",
             3: f"spmv_staged_kernel ({minfo['vector_width']} lanes/row)",
             4: f"spmv_merge_kernel ({minfo['vector_width']} lanes/row)",
             5: "spmv_slab_kernel (x slabs in shared memory)"}.get(minfo["variant"], "spmv")
    peak, peak_kind = _peaks()
    achieved = wl.spmv_bytes() / (spmv_ms / 1000.0) / 1e9
    traffic = _ncu_traffic(f"spmv_cg_{args.workload}")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": kname + " with the CG epilogue (q = A p, p.q fused)",
                "algorithmic_bytes_per_launch": wl.spmv_bytes(),
                "avg_launch_ms": spmv_ms, "launches_timed": n_spmv,
                "peak_kind": f"of {peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}

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
    e2e_ms = e0.elapsed_time(e1)
    if ws > 1:
        t = torch.tensor([e2e_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e = {"value": ws * K / (e2e_ms / 1000.0), "unit": wl.unit,
           "h2d_bytes_per_step": wl.e2e_bytes[0], "d2h_bytes_per_step": wl.e2e_bytes[1]}

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and ws == 1:
            v, sample = wl.cpu_sample(budget_s=20.0)
            cpu = {"value": v, "unit": wl.unit, "cores": 1, "kind": "oracle", "sample": sample}
        line = {"metric": METRIC, "value": value, "unit": wl.unit, "n_gpus": ws, "steps": K,
                "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": wl.dtype, "data": "synthetic",
                "config": wl.config() | {"parallelism": f"replicas{ws}"},
                "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                               "p99": float(np.percentile(step_ms, 99))},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": wl.launches_per_step * K,
                "clocks": clk, "check": check,
                "spmv": {"gbs": achieved, "hbm_frac": achieved / peak}}
        print(json.dumps(line), flush=True)
    wl.close()
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
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cg75k")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_lilac(args)


if __name__ == "__main__":
    sys.exit(main())
