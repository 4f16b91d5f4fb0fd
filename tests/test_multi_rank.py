"""The N > 1 launch path of bench.py without a GPU (replicas only: the path
does not shard): two gloo ranks agree on the slowest rank's time and the
whole-job throughput, and the reference arm under torchrun prints one line
from rank 0 while the other rank exits without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r timed 10 (r + 1) ms for 100 units per step over 4 steps
    value, t_max = bench.job_throughput(10.0 * (rank + 1), 100, 4)
    q.put((rank, value, t_max))
    dist.destroy_process_group()


def test_job_throughput_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(2))
    for rank, value, t_max in out:
        assert t_max == 20.0  # the slowest rank's time, on every rank
        assert value == pytest.approx(2 * 100 * 4 / 0.020)


def test_job_throughput_single_process():
    sys.path.insert(0, ROOT)
    import bench
    value, t_max = bench.job_throughput(5.0, 10, 2)
    assert t_max == 5.0 and value == pytest.approx(10 * 2 / 0.005)


def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "2", "--warmup", "1", "--config", "plate_100x40"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
