"""Host logic of the benchmark's multi-GPU form (replicas, one per rank),
run as two gloo processes on the CPU: the job time is the slowest rank's,
the throughput counts every rank's bodies, and only rank 0 reports."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench  # noqa: PLC0415
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    value, ms = bench.replica_throughput(10.0 + 5.0 * rank, 1000, world, dist, torch.device("cpu"))
    out.put((rank, value, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_takes_the_slowest_rank():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # rank 0 took 10 ms, rank 1 15 ms: both see 15 ms and 2 x 1000 bodies / 15 ms
    for _, value, ms in res:
        assert ms == 15.0
        assert value == pytest.approx(2000 / 15e-3)


def test_single_rank_throughput():
    sys.path.insert(0, ROOT)
    import bench  # noqa: PLC0415
    value, ms = bench.replica_throughput(20.0, 4096, 1)
    assert ms == 20.0 and value == pytest.approx(4096 / 20e-3)


def test_reference_arm_reports_on_rank_0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


@pytest.mark.slow
def test_reference_arm_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    # the same oracle solve on one core, beside the all-core figure
    assert 0 < line["cpu_baseline"]["value_1_core"] <= line["value"] * 1.5
