"""The N > 1 replica path of bench.py on the CPU: two gloo ranks take the
maximum of their times and report the whole job's throughput, and the
reference arm under torchrun prints one line from rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    barrier, max_over_ranks = bench.collectives(ws, "cpu")
    barrier()
    t = max_over_ranks(100.0 + 50.0 * rank)  # rank 1 is the slow one
    v = bench.replica_value(ws, 10, 2.0, t)
    barrier()
    dist.destroy_process_group()
    q.put((rank, t, v))


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 150.0
        # 2 ranks x 10 steps x 2 units over 0.15 s
        assert abs(v - 2 * 10 * 2.0 / 0.150) < 1e-9


def test_reference_arm_under_torchrun_prints_once():
    pytest.importorskip("torch.distributed.run")
    port = 30500 + os.getpid() % 1000
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--workload", "spmv2d", "--gpus", "2", "--steps", "1", "--warmup", "3",
           "--ref-seconds", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
