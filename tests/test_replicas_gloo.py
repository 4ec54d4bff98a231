"""Multi-process replica path of the benchmark on CPU (gloo, world size 2):
whole-job throughput = units of all ranks / slowest rank's time, and the
reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units = 1000.0 * (rank + 1)          # ranks may process different amounts
    ms = 10.0 + 5.0 * rank               # rank 1 is the slowest
    value, ms_max = bench.replica_throughput(units, ms, dist)
    out.put((rank, value, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms_max in res:
        assert ms_max == 15.0
        assert abs(value - 3000.0 / 15e-3) < 1e-6 * value


def test_replica_throughput_single_process():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.replica_throughput(500.0, 2.0, None)
    assert ms == 2.0 and abs(value - 250000.0) < 1e-9


def test_reference_arm_prints_once_under_two_ranks():
    port = _free_port()
    env = dict(os.environ, DJ_REF_BUDGET_S="0.5")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "2", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
