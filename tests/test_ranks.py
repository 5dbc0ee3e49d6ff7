"""The N > 1 path of bench.py on CPU: replicas over a world-size-2 gloo
group (independent problems per rank, the job's time the slowest rank's,
whole-job throughput) and the reference arm under torchrun (rank 0 alone
measures and prints one line, the other rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank, ws, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        t = 1.0 + rank  # this rank's timed region (s)
        t_job = bench.max_over_ranks(t, ws)
        rate = bench.job_rate(ws, 3, 10.0, t_job)
        seeds = [None] * ws
        dist.all_gather_object(seeds, bench.rank_seed(rank))
        out.put((rank, t_job, rate, seeds))
    finally:
        dist.destroy_process_group()


def test_replicas_over_gloo():
    import torch.multiprocessing as mp

    ws, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_replica, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_job, rate, seeds in res:
        assert t_job == 2.0  # the slowest rank's time on every rank
        assert rate == pytest.approx(2 * 3 * 10.0 / 2.0)  # units of all ranks / job time
        assert len(set(seeds)) == ws  # every rank its own slice


def test_reference_arm_under_torchrun():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus",
           "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
