"""Multi-rank path of bench.py on CPU: two gloo ranks as replicas.

The method does not shard within a scene here: N GPUs run N independent
replicas, and the only cross-rank step is the throughput reduction (units of all
ranks over the slowest rank's time). This runs that reduction with world size 2.
"""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r ran r + 2 steps in 100 (r + 1) ms
        rate, slowest = bench.job_rate(rank + 2, 100.0 * (rank + 1))
        out[rank] = (rate, slowest)
    finally:
        dist.destroy_process_group()


def test_job_rate_sums_units_over_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # (2 + 3) steps over the slowest 200 ms = 25 steps/s, the same on every rank
    for r in range(world):
        assert res[r][1] == pytest.approx(200.0)
        assert res[r][0] == pytest.approx(25.0)


def test_job_rate_single_process_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    rate, t = bench.job_rate(3, 150.0)
    assert rate == pytest.approx(20.0) and t == 150.0


def test_reference_arm_under_torchrun_prints_once_from_rank_zero():
    """Launched like the multi-GPU bench (torchrun, two ranks), the oracle arm
    runs on rank 0 alone and prints exactly one JSON line; rank 1 exits 0
    without work."""
    import json
    import subprocess
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload", "droplet"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
