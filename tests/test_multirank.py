"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks (replicas, no
data-path collective) reduce their timings to the slowest rank, and the job
throughput counts every rank's units; the reference arm prints on rank 0
only."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local = [10.0 + 5.0 * rank, 100.0 - rank]          # rank 1 is the slower one on the first entry
    tmax, emax = bench.max_over_ranks(local, dist, torch.device("cpu"))
    units, value = bench.job_throughput(1000, 4, ws, tmax)
    q.put((rank, tmax, emax, units, value))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo_ws2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, emax, units, value in res:
        assert tmax == 15.0 and emax == 100.0          # the maximum, on every rank
        assert units == 1000 * 4 * 2
        assert abs(value - units / 15e-3) < 1e-6 * value


def test_single_rank_is_identity():
    assert bench.max_over_ranks([3.0, 4.0], None, None) == [3.0, 4.0]
    units, value = bench.job_throughput(10, 2, 1, 5.0)
    assert units == 20 and abs(value - 4000.0) < 1e-9


def test_reference_arm_prints_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="2", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
