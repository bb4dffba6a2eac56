"""The multi-rank logic of bench.py on the CPU: world_size-2 gloo ranks run
independent replicas, the job time is the maximum over ranks and the value is
the total over ranks; the reference arm's non-zero ranks exit without work."""
import os
import subprocess
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    local_ms = [12.0, 20.0][rank]
    value, job_ms = bench.job_rate(world, 1000, local_ms)
    out[rank] = (value, job_ms)
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_is_total_over_ranks_at_the_slowest_rank():
    world = 2
    port = 29500 + os.getpid() % 1000
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        value, job_ms = out[r]
        assert job_ms == 20.0
        assert abs(value - 2 * 1000 / 0.020) < 1e-6


def test_single_rank_rate():
    sys.path.insert(0, ROOT)
    import bench
    value, job_ms = bench.job_rate(1, 1024 * 50, 12.5)
    assert job_ms == 12.5 and abs(value - 1024 * 50 / 0.0125) < 1e-6


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0
    assert p.stdout.strip() == ""
