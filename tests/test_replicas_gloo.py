"""The multi-GPU path of bench.py is replicas only: each rank runs the whole
workload, the ranks line up around the timed region, and the job's time is the
slowest rank's. These tests run that logic as two gloo processes on the CPU
(no GPU), and the reference arm under torchrun (rank 0 prints, rank 1 exits)."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    g = bench.ReplicaGroup("gloo")
    g.barrier()
    t = g.max(1.5 + rank)                      # rank 1 is the slowest
    q.put((rank, g.rank, g.world, t, bench.whole_job_value(2e12, t, g.world)))
    g.barrier()
    g.close()


def test_replica_group_max_and_whole_job_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, grank, world, t, v in out:
        assert grank == rank and world == 2
        assert t == 2.5                         # the slowest rank's time, on every rank
        assert v == pytest.approx(2 * 2e12 / 2.5e-3 / 1e12)


def test_single_process_group():
    sys.path.insert(0, ROOT)
    import bench
    g = bench.ReplicaGroup(None)
    assert g.world == 1 and g.rank == 0 and g.max(3.0) == 3.0
    g.barrier()
    assert bench.whole_job_value(1e12, 1.0, 1) == pytest.approx(1000.0)


def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1                      # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
